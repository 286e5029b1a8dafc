"""Seeded synthetic grey images shared by the GPU-path tests, the oracle tests
and the benchmark.

This module only draws inputs; it holds none of the detector's or the
descriptor's arithmetic. The images stand in for the 640x480 test images of
the paper's evaluation (Sec. V-A), which are not available here: a flat
background, anisotropic Gaussian blobs of random size, angle and contrast, and
band-limited noise, clipped to 0..255.

Random numbers come from one counter-based generator, SplitMix64's output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``key + (counter + 1) * 0x9E3779B97F4A7C15``,
so every value is a pure function of (seed, stream, counter) on any machine.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (xor-ed into the image seed)
_STREAM_BLOBS = 1
_STREAM_NOISE = 2
_STREAM_WARP = 3
_STREAM_SIZE = 4


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def mix64(x: int) -> int:
    """SplitMix64 output function of one integer."""
    return int(_mix(np.array([x & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0])


def raw64(key: int, start: int, n: int) -> np.ndarray:
    """n 64-bit draws of stream ``key`` at counters start .. start+n-1."""
    c = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + c * _GAMMA
    return _mix(z)


def uniform(key: int, start: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of each draw."""
    return (raw64(key, start, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(key: int, start: int, n: int) -> np.ndarray:
    """n standard normals by the Box-Muller transform of paired uniforms."""
    m = (n + 1) // 2
    u = uniform(key, start, 2 * m)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
    return z[:n]


def image_seed(base: int, i: int) -> int:
    """Seed of image i of a batch drawn from base seed ``base``."""
    return (base ^ mix64(i)) & 0xFFFFFFFFFFFFFFFF


def _stream(seed: int, stream: int) -> int:
    return mix64(seed ^ (stream * 0x632BE59BD9B4E019))


def _smooth_noise(z: np.ndarray, sigma: float = 1.0) -> np.ndarray:
    """Separable Gaussian smoothing (edge-clamped) of the white noise field."""
    r = int(math.ceil(4 * sigma))
    t = np.exp(-(np.arange(-r, r + 1) ** 2) / (2 * sigma * sigma))
    t /= t.sum()
    H, W = z.shape
    zp = np.pad(z, ((r, r), (0, 0)), mode="edge")
    v = sum(t[i] * zp[i:i + H, :] for i in range(2 * r + 1))
    vp = np.pad(v, ((0, 0), (r, r)), mode="edge")
    out = sum(t[i] * vp[:, i:i + W] for i in range(2 * r + 1))
    # std of unit white noise after the 2-D kernel = sum of squared 1-D taps
    return out / float((t * t).sum())


def blob_image(seed: int, width: int = 640, height: int = 480, n_blobs: int = 200,
               sigma_range=(1.5, 20.0), amp_range=(20.0, 120.0), noise_std: float = 4.0,
               background: float = 128.0) -> np.ndarray:
    """One synthetic uint8 image (height x width).

    ``n_blobs`` anisotropic Gaussian blobs: centre uniform over the image, two
    standard deviations uniform in ``sigma_range`` (the larger is the major
    axis), angle uniform in [0, pi), amplitude uniform in ``amp_range`` with a
    random sign; plus white noise smoothed by a Gaussian of std 1 px and scaled
    to ``noise_std``; clipped to [0, 255] and rounded half to even.
    """
    kb = _stream(seed, _STREAM_BLOBS)
    u = uniform(kb, 0, 7 * n_blobs).reshape(n_blobs, 7)
    img = np.full((height, width), background, dtype=np.float64)
    lo, hi = sigma_range
    for b in range(n_blobs):
        cx = u[b, 0] * width
        cy = u[b, 1] * height
        s1 = lo + (hi - lo) * u[b, 2]
        s2 = lo + (hi - lo) * u[b, 3]
        smaj, smin = max(s1, s2), min(s1, s2)
        ang = math.pi * u[b, 4]
        amp = amp_range[0] + (amp_range[1] - amp_range[0]) * u[b, 5]
        if u[b, 6] < 0.5:
            amp = -amp
        ext = 4.0 * smaj
        x0, x1 = max(0, int(math.floor(cx - ext))), min(width, int(math.ceil(cx + ext)) + 1)
        y0, y1 = max(0, int(math.floor(cy - ext))), min(height, int(math.ceil(cy + ext)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        xs = np.arange(x0, x1, dtype=np.float64) - cx
        ys = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
        c, s = math.cos(ang), math.sin(ang)
        xr = xs * c + ys * s
        yr = -xs * s + ys * c
        img[y0:y1, x0:x1] += amp * np.exp(-0.5 * (xr * xr / (smaj * smaj) + yr * yr / (smin * smin)))
    if noise_std > 0:
        kn = _stream(seed, _STREAM_NOISE)
        z = normal(kn, 0, width * height).reshape(height, width)
        img += noise_std * _smooth_noise(z)
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)


def blob_batch(n: int, base_seed: int = 1, width: int = 640, height: int = 480, **kw) -> np.ndarray:
    """n images (n x height x width, uint8); image i uses image_seed(base_seed, i)."""
    out = np.empty((n, height, width), dtype=np.uint8)
    for i in range(n):
        out[i] = blob_image(image_seed(base_seed, i), width, height, **kw)
    return out


def warp_params(seed: int):
    """Rotation (rad, 0..45 deg) and scale (0.7..1.4) of the paired warped copy."""
    u = uniform(_stream(seed, _STREAM_WARP), 0, 2)
    return math.radians(45.0 * u[0]), 0.7 + 0.7 * u[1]


def warp_image(img: np.ndarray, angle: float, scale: float, fill: float = 128.0) -> np.ndarray:
    """Rotate by ``angle`` and scale by ``scale`` about the image centre, bilinear,
    ``fill`` outside; returns the warped uint8 image and the 2x3 forward map."""
    H, W = img.shape
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    c, s = math.cos(angle), math.sin(angle)
    # forward: p' = scale * R (p - c) + c ; inverse for sampling
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    dx, dy = (xx - cx) / scale, (yy - cy) / scale
    sx = c * dx + s * dy + cx
    sy = -s * dx + c * dy + cy
    x0 = np.floor(sx).astype(np.int64)
    y0 = np.floor(sy).astype(np.int64)
    fx, fy = sx - x0, sy - y0
    src = img.astype(np.float64)

    def tap(yi, xi):
        ok = (xi >= 0) & (xi < W) & (yi >= 0) & (yi < H)
        v = np.full(xi.shape, fill)
        v[ok] = src[yi[ok], xi[ok]]
        return v

    out = ((1 - fx) * (1 - fy) * tap(y0, x0) + fx * (1 - fy) * tap(y0, x0 + 1)
           + (1 - fx) * fy * tap(y0 + 1, x0) + fx * fy * tap(y0 + 1, x0 + 1))
    A = np.array([[scale * c, -scale * s, 0.0], [scale * s, scale * c, 0.0]])
    A[:, 2] = np.array([cx, cy]) - A[:, :2] @ np.array([cx, cy])
    return np.rint(np.clip(out, 0, 255)).astype(np.uint8), A


def uneven_sizes(n: int, base_seed: int = 3, lo: int = 240, hi: int = 1280):
    """Sizes (width, height) of an uneven batch: width uniform in [lo, hi],
    aspect uniform in [0.5, 2], height = clamp(round(width / aspect), lo, hi)."""
    u = uniform(_stream(base_seed, _STREAM_SIZE), 0, 2 * n).reshape(n, 2)
    out = []
    for i in range(n):
        w = int(lo + math.floor((hi - lo + 1) * u[i, 0]))
        aspect = 0.5 + 1.5 * u[i, 1]
        h = int(min(hi, max(lo, round(w / aspect))))
        out.append((w, h))
    return out
