// onepass.cuh -- single-pass launches in which a CTA reads what CTAs of
// lower index in the same launch publish (decoupled look-back).
//
// A CTA only ever waits on CTAs of lower index.  CTAs are dispatched in
// index order, so every CTA waited on has started and runs to the point
// where it publishes, whatever the grid size; every wait is also bounded
// (one second, then the device status bit is set and the CTA goes on).
//
// The published words live in the caller's workspace and carry a launch
// tag, so nothing has to be cleared between launches: the workspace holds
// the last launch's tag in its first word, a launch uses one more than
// that (1 .. 2^31 - 1, then 1 again) and only accepts words with its own
// tag.  The CTA that finishes last in dependency order (it has seen every
// other CTA publish, so every CTA has read the old tag) stores the new one.
// A workspace must be zero-filled once before its first launch (zero is
// the tag of no launch); afterwards every launch leaves it ready for the
// next, including one whose waits ran out.
#pragma once

#include <cstdint>

#include "ptx.cuh"

namespace fasthog {
namespace onepass {

// Bytes in front of the published words: the tag word, padded.
constexpr int kHeaderBytes = 64;

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// This launch's tag, from the last launch's (the header's first word).
__device__ __forceinline__ uint32_t launch_tag(const void* ws) {
    const uint32_t last = ld_relaxed(static_cast<const uint32_t*>(ws));
    return (last + 1u) >= 0x80000000u ? 1u : last + 1u;
}
__device__ __forceinline__ void end_launch(void* ws, uint32_t tag) { st_relaxed(static_cast<uint32_t*>(ws), tag); }

// Status word of a unit (one 64-bit store carries everything a reader
// needs, so no fence is required): tag and an inclusive bit in the high
// half, a 32-bit value in the low half.
__device__ __forceinline__ unsigned long long status_word(uint32_t tag, bool inclusive, uint32_t value) {
    return ((unsigned long long)((tag << 1) | (inclusive ? 1u : 0u)) << 32) | value;
}

// Spin until `slot` carries `tag`; returns false if the wait ran out.
__device__ __forceinline__ bool wait_status(const unsigned long long* slot, uint32_t tag, bool& inclusive,
                                            uint32_t& value, uint64_t limit_ns = kWaitLimitNs) {
    unsigned long long s = ld_relaxed(slot);
    if ((uint32_t)(s >> 33) != tag) {
        const uint64_t t0 = ptx::globaltimer_ns();
        do {
            if (ptx::globaltimer_ns() - t0 > limit_ns) return false;
            s = ld_relaxed(slot);
        } while ((uint32_t)(s >> 33) != tag);
    }
    inclusive = ((s >> 32) & 1u) != 0;
    value = (uint32_t)s;
    return true;
}

// Spin until the flag word `flag` equals `tag` (acquire: what its writer
// stored before its release becomes visible); false if the wait ran out.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t tag, uint64_t limit_ns = kWaitLimitNs) {
    if (ld_acquire(flag) == tag) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (ld_acquire(flag) != tag)
        if (ptx::globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

}  // namespace onepass
}  // namespace fasthog
