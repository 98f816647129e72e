// tcgen05.cuh -- inline-PTX pieces of the tensor-core score kernels
// (sm_103a): shared-memory and instruction descriptors, the bf16 MMA with
// its commit, TMEM loads, and the bf16 forms of the weights.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {
namespace tc {

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // tcgen05 shared-memory descriptor, no swizzle: start >> 4 in bits 0-13,
    // leading-dimension byte offset >> 4 in bits 16-29, stride-dimension byte
    // offset >> 4 in bits 32-45, fixed 0b001 in bits 46-48.
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D = f32, A = B = bf16, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     ptx::smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes; the registers are
// valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_load16_async(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Weights off .. off + 7 (off a multiple of 8) as 8 bf16 values.
template <typename WT>
__device__ __forceinline__ uint4 load_weight8(const WT* w, int off);
template <>
__device__ __forceinline__ uint4 load_weight8<uint16_t>(const uint16_t* w, int off) {
    const uint16_t* p = w + off;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) return __ldg(reinterpret_cast<const uint4*>(p));
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = (uint32_t)__ldg(p + 2 * k) | ((uint32_t)__ldg(p + 2 * k + 1) << 16);
    return make_uint4(h[0], h[1], h[2], h[3]);
}
template <>
__device__ __forceinline__ uint4 load_weight8<int8_t>(const int8_t* w, int off) {
    const int8_t* p = w + off;
    int8_t b[8];
    if ((reinterpret_cast<uintptr_t>(p) & 7) == 0) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            b[k] = (int8_t)(v.x >> (8 * k));
            b[k + 4] = (int8_t)(v.y >> (8 * k));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = __ldg(p + k);
    }
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)  // |w| <= 127: exact in bf16
        h[k] = (uint32_t)f32_to_bf16_exact_int((float)b[2 * k]) |
               ((uint32_t)f32_to_bf16_exact_int((float)b[2 * k + 1]) << 16);
    return make_uint4(h[0], h[1], h[2], h[3]);
}

// f32 weights: x = p0 + p1 + p2 exactly, each part the bf16 rounding of what
// the previous parts leave (every residual is exact in f32: it keeps the low
// bits of x, and 3 x 8 significand bits cover f32's 24).  Counts are exact
// in bf16 and a count times a bf16 part is exact in f32, so three MMAs per
// step into one accumulator give the f32 products; only the f32
// accumulation rounds.
__device__ __forceinline__ uint32_t bf16_part(float x, int part) {
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    for (int k = 0; k < part; ++k) {
        x = x - __bfloat162float(b);
        b = __float2bfloat16_rn(x);
    }
    return (uint32_t)__bfloat16_as_ushort(b);
}

// Part `part` of weights off .. off + 7 as 8 bf16 values (bf16 and int8
// weights have one part).
template <typename WT>
__device__ __forceinline__ uint4 load_weight8_part(const WT* w, int off, int part) {
    (void)part;
    return load_weight8<WT>(w, off);
}
template <>
__device__ __forceinline__ uint4 load_weight8_part<float>(const float* w, int off, int part) {
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        h[k] = bf16_part(__ldg(w + off + 2 * k), part) | (bf16_part(__ldg(w + off + 2 * k + 1), part) << 16);
    return make_uint4(h[0], h[1], h[2], h[3]);
}

// Part `part` of the 8 weights at w (any address space, read with plain
// loads) as 8 bf16 values.
template <typename WT>
__device__ __forceinline__ uint4 weight8_part(const WT* w, int part);
template <>
__device__ __forceinline__ uint4 weight8_part<float>(const float* w, int part) {
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = bf16_part(w[2 * k], part) | (bf16_part(w[2 * k + 1], part) << 16);
    return make_uint4(h[0], h[1], h[2], h[3]);
}
template <>
__device__ __forceinline__ uint4 weight8_part<uint16_t>(const uint16_t* w, int) {
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = (uint32_t)w[2 * k] | ((uint32_t)w[2 * k + 1] << 16);
    return make_uint4(h[0], h[1], h[2], h[3]);
}
template <>
__device__ __forceinline__ uint4 weight8_part<int8_t>(const int8_t* w, int) {
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)  // |w| <= 127: exact in bf16
        h[k] = (uint32_t)f32_to_bf16_exact_int((float)w[2 * k]) |
               ((uint32_t)f32_to_bf16_exact_int((float)w[2 * k + 1]) << 16);
    return make_uint4(h[0], h[1], h[2], h[3]);
}

// All PARTS parts of the 8 weights at w (any address space): part p is the
// bf16 rounding of what parts 0 .. p - 1 leave of each weight.
template <typename WT, int PARTS>
__device__ __forceinline__ void weight8_parts(const WT* w, uint4 (&out)[PARTS]) {
    if constexpr (std::is_same<WT, float>::value) {
        float x[8];
        const float4 a = reinterpret_cast<const float4*>(w)[0], b = reinterpret_cast<const float4*>(w)[1];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
#pragma unroll
        for (int p = 0; p < PARTS; ++p) {
            uint32_t h[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const __nv_bfloat16 r = __float2bfloat16_rn(x[k]);
                h[k] = (uint32_t)__bfloat16_as_ushort(r);
                x[k] -= __bfloat162float(r);  // exact: the residual keeps the low bits of x
            }
            out[p] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
    } else {
        out[0] = weight8_part<WT>(w, 0);
    }
}

template <typename WT>
__host__ __device__ constexpr int weight_parts() {
    return std::is_same<WT, float>::value ? 3 : 1;
}

}  // namespace tc
}  // namespace fasthog
