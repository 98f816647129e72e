"""Seeded synthetic inputs for the fast-HOG detection path.

This module is shared by the oracle side (tests, CPU baseline) and the CUDA
side (tests, benchmark).  It holds no step of the method: it only draws
images, weights and request streams from NumPy's PCG64 generator.

The paper measures on no public dataset (it quotes timings on an 800x600
image and on 352x288 video), so every input here is synthetic.  The
workloads, indexed as in the project's configuration list:

  0  one 320x240 gray image: uniform noise plus 20 filled rectangles;
     N_b = 8, stride 8, float32 weights N(0, 0.01) of length 1024, bias 0.
  1  one 800x600 RGB image: smooth multi-octave value noise plus random
     rectangles and ellipses; N_b = 8, stride 4, threshold 0.5.
  2  64 RGB images with sizes drawn from {640x480, 800x600, 1280x720,
     1920x1080}, each with a 3-level 2:1 pyramid; N_b in {8, 16}.
  3  32 RGB 1920x1080 images; N_b = 8, stride 4; bf16 and int8 weights.
  4  a Poisson stream of RGB requests with sizes uniform over multiples of
     8 from 320x240 to 3840x2160.

Seeds are 1703 + workload index unless the caller passes another.
"""

from __future__ import annotations

import numpy as np

BASE_SEED = 1703

WINDOW_CELLS_X = 8
WINDOW_CELLS_Y = 16
CELL = 8


def rng_for(index: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + index if seed is None else seed))


def gray_noise_rects(W: int, H: int, rng: np.random.Generator, n_rects: int = 20) -> np.ndarray:
    """Uniform [0, 255] noise with `n_rects` filled axis-aligned rectangles of random gray."""
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    for _ in range(n_rects):
        x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
        y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
        img[y0:y1, x0:x1] = rng.integers(0, 256, dtype=np.uint8)
    return img


def _value_noise_octave(W: int, H: int, cell: float, rng: np.random.Generator, ch: int) -> np.ndarray:
    """Random lattice values every `cell` pixels, smoothly interpolated (smoothstep)."""
    gw = int(np.ceil(W / cell)) + 2
    gh = int(np.ceil(H / cell)) + 2
    lat = rng.random((gh, gw, ch), dtype=np.float32)
    xs = np.arange(W, dtype=np.float32) / cell
    ys = np.arange(H, dtype=np.float32) / cell
    x0 = np.floor(xs).astype(np.int64)
    y0 = np.floor(ys).astype(np.int64)
    fx = xs - x0
    fy = ys - y0
    fx = fx * fx * (3 - 2 * fx)
    fy = fy * fy * (3 - 2 * fy)
    # interpolate along x once per lattice row, then pick and blend rows per
    # pixel row (the same float32 operations per pixel as blending the four
    # corners of every pixel directly)
    left = lat[:, x0]
    right = lat[:, x0 + 1]
    along_x = left + (right - left) * fx[None, :, None]
    top = along_x[y0]
    bot = along_x[y0 + 1]
    return top + (bot - top) * fy[:, None, None]


def rgb_smooth_shapes(W: int, H: int, rng: np.random.Generator, octaves: int = 4,
                      n_shapes: int = 24) -> np.ndarray:
    """Perlin-style smooth RGB noise (`octaves` octaves of value noise, the
    amplitude halving per octave) plus random filled rectangles and ellipses."""
    acc = np.zeros((H, W, 3), np.float32)
    amp, total = 1.0, 0.0
    base = max(W, H) / 4.0
    for o in range(octaves):
        acc += amp * _value_noise_octave(W, H, max(base / (2 ** o), 2.0), rng, 3)
        total += amp
        amp *= 0.5
    img = np.clip(acc / total * 255.0, 0, 255).astype(np.uint8)
    yy, xx = np.mgrid[0:H, 0:W]
    for _ in range(n_shapes):
        color = rng.integers(0, 256, size=3, dtype=np.uint8)
        cx, cy = rng.integers(0, W), rng.integers(0, H)
        rx = int(rng.integers(4, max(5, W // 6)))
        ry = int(rng.integers(4, max(5, H // 6)))
        if rng.random() < 0.5:
            img[max(cy - ry, 0):cy + ry, max(cx - rx, 0):cx + rx] = color
        else:
            # the ellipse lies inside its bounding box; test only the pixels there
            ya, yb = max(cy - ry, 0), min(cy + ry + 1, H)
            xa, xb = max(cx - rx, 0), min(cx + rx + 1, W)
            m = ((xx[ya:yb, xa:xb] - cx) / rx) ** 2 + ((yy[ya:yb, xa:xb] - cy) / ry) ** 2 <= 1.0
            img[ya:yb, xa:xb][m] = color
    return img


def weights_f32(n_bins: int, rng: np.random.Generator, sigma: float = 0.01) -> np.ndarray:
    """Window filter of 16 x 8 cells x n_bins, N(0, sigma^2), float32."""
    return rng.normal(0.0, sigma, size=WINDOW_CELLS_Y * WINDOW_CELLS_X * n_bins).astype(np.float32)


def weights_i8(n_bins: int, rng: np.random.Generator) -> np.ndarray:
    """Integer filter: uniform integers in [-127, 127], int8."""
    return rng.integers(-127, 128, size=WINDOW_CELLS_Y * WINDOW_CELLS_X * n_bins).astype(np.int8)


def config0(seed: int | None = None) -> dict:
    rng = rng_for(0, seed)
    img = gray_noise_rects(320, 240, rng)
    return dict(name="320x240 gray, N_b=8, stride 8", images=[img], n_bins=8, stride=8,
                w=weights_f32(8, rng), bias=0.0, thr=None)


def config1(seed: int | None = None) -> dict:
    rng = rng_for(1, seed)
    img = rgb_smooth_shapes(800, 600, rng)
    return dict(name="800x600 RGB, N_b=8, stride 4, thr 0.5", images=[img], n_bins=8, stride=4,
                w=weights_f32(8, rng), bias=0.0, thr=0.5)


BATCH_SIZES = [(640, 480), (800, 600), (1280, 720), (1920, 1080)]


def config2(seed: int | None = None, n_images: int = 64) -> dict:
    rng = rng_for(2, seed)
    sizes = [BATCH_SIZES[int(i)] for i in rng.integers(0, len(BATCH_SIZES), size=n_images)]
    images = [rgb_smooth_shapes(W, H, rng) for (W, H) in sizes]
    return dict(name=f"{n_images} RGB images of mixed sizes, 3-level pyramid", images=images,
                n_bins_options=(8, 16), stride=4, levels=3,
                w={8: weights_f32(8, rng), 16: weights_f32(16, rng)}, bias=0.0, thr=0.5)


def config3(seed: int | None = None, n_images: int = 32, W: int = 1920, H: int = 1080) -> dict:
    rng = rng_for(3, seed)
    images = [rgb_smooth_shapes(W, H, rng) for _ in range(n_images)]
    w = weights_f32(8, rng)
    return dict(name=f"{n_images} RGB {W}x{H}, N_b=8, stride 4", images=images, n_bins=8,
                stride=4, w=w, w_i8=weights_i8(8, rng), bias=0.0, thr=0.5)


def request_stream(n_requests: int, rate_per_s: float, seed: int | None = None,
                   min_wh=(320, 240), max_wh=(3840, 2160)) -> list[dict]:
    """Poisson arrivals; each request an RGB image whose width and height are
    uniform over multiples of 8 in [min, max].  Images are drawn lazily by the
    consumer from the recorded per-request seed."""
    rng = rng_for(4, seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps)
    ws = rng.integers(min_wh[0] // 8, max_wh[0] // 8 + 1, size=n_requests) * 8
    hs = rng.integers(min_wh[1] // 8, max_wh[1] // 8 + 1, size=n_requests) * 8
    seeds = rng.integers(0, 2 ** 31 - 1, size=n_requests)
    return [dict(t=float(t[i]), W=int(ws[i]), H=int(hs[i]), seed=int(seeds[i]))
            for i in range(n_requests)]


def request_image(req: dict) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(req["seed"]))
    return rgb_smooth_shapes(req["W"], req["H"], rng, n_shapes=8)
