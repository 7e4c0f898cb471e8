"""Seeded synthetic rectified stereo pairs (shared input generator).

The paper's laparoscopy videos are not available, so these generators stand in
for them: textured left images, a smooth ground-truth disparity field, and a
right image rendered from the left one through that field.  This module holds
none of the matching method's arithmetic; it only makes inputs, which both the
CUDA path and the CPU oracle consume.

Workloads (seed = 20070000 + 100 * config + pair index):
  * ``perlin_pair``   320x240 gray, Perlin-style texture with two 40x40
                      low-texture patches, disparity 2..28 from three Gaussian
                      bumps, right-view noise sigma 1.
  * ``tissue_pair``   RGB tissue-like texture (vessel ridges on band-limited
                      noise, 30 % low-texture blobs), disparity from a random
                      quadratic surface plus bumps, right view with gain
                      0.9..1.1, offset -8..8 and noise sigma 2.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

SEED_BASE = 20070000


def seed_for(config: int, pair: int = 0) -> int:
    return SEED_BASE + 100 * config + pair


# ------------------------------------------------------------------ textures

def _perlin(rng, H, W, period):
    """One octave of 2-D gradient noise with lattice spacing ``period``."""
    gy, gx = int(np.ceil(H / period)) + 2, int(np.ceil(W / period)) + 2
    ang = rng.uniform(0, 2 * np.pi, (gy, gx))
    gvx, gvy = np.cos(ang), np.sin(ang)
    ys = np.arange(H) / period
    xs = np.arange(W) / period
    y0 = np.floor(ys).astype(int)
    x0 = np.floor(xs).astype(int)
    fy = (ys - y0)[:, None]
    fx = (xs - x0)[None, :]

    def dot(iy, ix, oy, ox):
        return gvx[iy[:, None], ix[None, :]] * ox + gvy[iy[:, None], ix[None, :]] * oy

    n00 = dot(y0, x0, fy, fx)
    n01 = dot(y0, x0 + 1, fy, fx - 1)
    n10 = dot(y0 + 1, x0, fy - 1, fx)
    n11 = dot(y0 + 1, x0 + 1, fy - 1, fx - 1)
    sy = fy * fy * fy * (fy * (fy * 6 - 15) + 10)
    sx = fx * fx * fx * (fx * (fx * 6 - 15) + 10)
    a = n00 + sx * (n01 - n00)
    b = n10 + sx * (n11 - n10)
    return a + sy * (b - a)


def perlin_texture(rng, H, W, base_period=32, octaves=4):
    t = np.zeros((H, W))
    amp = 1.0
    for o in range(octaves):
        t += amp * _perlin(rng, H, W, base_period / (2 ** o))
        amp *= 0.5
    return t


def _normalise(a, lo, hi):
    a = a - a.min()
    m = a.max()
    return lo + (hi - lo) * (a / m if m > 0 else a)


def _bumps(rng, H, W, n, sig_lo, sig_hi):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    f = np.zeros((H, W))
    for _ in range(n):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        s = rng.uniform(sig_lo, sig_hi)
        a = rng.uniform(0.5, 1.0)
        f += a * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
    return f


# ------------------------------------------------------------ right view

def render_right(left: np.ndarray, disp: np.ndarray, iters: int = 12) -> np.ndarray:
    """Backward-warp the left view into the right view.

    A left pixel x with disparity d(x) appears at x - d(x) in the right view, so
    R(u) = L(u + t(u)) where t solves t(u) = d(u + t(u)); t is found by
    fixed-point iteration and L, d are sampled with 1-D linear interpolation.
    ``left`` is float (H, W) or (H, W, C); returns float of the same shape.
    """
    H, W = disp.shape
    u = np.arange(W, dtype=np.float64)[None, :].repeat(H, 0)
    rows = np.arange(H)[:, None]

    def sample_row(img, xs):
        xs = np.clip(xs, 0, W - 1)
        x0 = np.floor(xs).astype(np.int64)
        x1 = np.minimum(x0 + 1, W - 1)
        f = xs - x0
        if img.ndim == 3:
            f = f[..., None]
        return img[rows, x0] * (1 - f) + img[rows, x1] * f

    t = disp.copy()
    for _ in range(iters):
        t = sample_row(disp, u + t)
    return sample_row(left, u + t)


# ------------------------------------------------------------------- pairs

def perlin_pair(seed: int, W: int = 320, H: int = 240):
    """Gray pair: band-limited Perlin texture (20..235), two 40x40 near-constant
    patches, disparity 2..28 from three Gaussian bumps (sigma 30..60 px),
    right view with N(0, 1) noise.  Returns (L u8, R u8, gt float64)."""
    rng = np.random.default_rng(seed)
    tex = _normalise(perlin_texture(rng, H, W, 32, 4), 20.0, 235.0)
    for _ in range(2):
        py = int(rng.integers(0, max(1, H - 40)))
        px = int(rng.integers(0, max(1, W - 40)))
        tex[py:py + 40, px:px + 40] = 128.0 + rng.uniform(-1, 1, (min(40, H - py), min(40, W - px)))
    gt = 2.0 + 26.0 * _normalise(_bumps(rng, H, W, 3, 30, 60), 0.0, 1.0)
    right = render_right(tex, gt) + rng.normal(0.0, 1.0, (H, W))
    L = np.clip(np.rint(tex), 0, 255).astype(np.uint8)
    R = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return L, R, gt


def _smooth_coarse(a, sigma, f=4):
    """Gaussian blur of width sigma computed on an f-times coarser grid."""
    H, W = a.shape
    Hc, Wc = (H + f - 1) // f, (W + f - 1) // f
    pad = np.pad(a, ((0, Hc * f - H), (0, Wc * f - W)), mode="edge")
    c = pad.reshape(Hc, f, Wc, f).mean(axis=(1, 3))
    c = ndimage.gaussian_filter(c, sigma / f)
    return ndimage.zoom(c, f, order=1)[:H, :W]


def tissue_texture(rng, H, W):
    """Gray tissue-like texture in [0, 255]: band-limited noise with 40..80
    smooth vessel ridges (Gaussian cross-section, amplitude -40..-80) and 30 %
    of the area blended to smooth shading (low texture)."""
    base = _normalise(perlin_texture(rng, H, W, max(8, W // 24), 4), -1, 1)
    fine = ndimage.gaussian_filter(rng.normal(0, 1, (H, W)), 1.2)
    fine /= fine.std() + 1e-12
    tex = 150.0 + 35.0 * base + 12.0 * fine
    nves = int(rng.integers(40, 81))
    scale = np.sqrt(H * W / (960.0 * 540.0))
    for wclass in range(3):
        mask = np.zeros((H, W))
        width = (1.0 + 1.5 * wclass) * max(scale, 0.5)
        for _ in range(nves // 3 + (1 if wclass < nves % 3 else 0)):
            n = 600
            t = np.linspace(0, 1, n)
            p0 = rng.uniform([0, 0], [W, H])
            ang = rng.uniform(0, 2 * np.pi)
            length = rng.uniform(0.3, 0.9) * max(W, H)
            k1, k2 = rng.normal(0, 1.5, 2)
            ph = rng.uniform(0, 2 * np.pi)
            theta = ang + k1 * t + 0.6 * np.sin(2 * np.pi * k2 * t + ph)
            dx = np.cos(theta) * length / n
            dy = np.sin(theta) * length / n
            xs = p0[0] + np.cumsum(dx)
            ys = p0[1] + np.cumsum(dy)
            amp = rng.uniform(40, 80)
            ok = (xs >= 0) & (xs < W) & (ys >= 0) & (ys < H)
            np.maximum.at(mask, (ys[ok].astype(int), xs[ok].astype(int)), amp)
        if mask.any():
            # a one-pixel line of height A blurred with sigma w has a Gaussian
            # cross-section of peak A / (sqrt(2 pi) w); rescale to peak A.
            tex -= ndimage.gaussian_filter(mask, width) * np.sqrt(2 * np.pi) * width
    # low-texture blobs covering 30 % of the area, blended to smooth shading
    # (the wide blurs run on a 4x coarser grid and are upsampled)
    blob = _smooth_coarse(rng.normal(0, 1, (H, W)), max(6.0, 25.0 * scale))
    thr = np.quantile(blob, 0.70)
    wgt = np.clip((blob - thr) / (blob.std() * 0.15 + 1e-12), 0, 1)
    smooth = _smooth_coarse(tex, max(4.0, 12.0 * scale))
    tex = tex * (1 - wgt) + smooth * wgt
    return np.clip(tex, 0, 255)


def tissue_disparity(rng, H, W, lo, hi):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    u = xx / W - 0.5
    v = yy / H - 0.5
    c = rng.normal(0, 1, 6)
    quad = c[0] * u + c[1] * v + c[2] * u * u + c[3] * v * v + c[4] * u * v
    bumps = _bumps(rng, H, W, int(rng.integers(3, 7)), 0.05 * max(W, H), 0.15 * max(W, H))
    f = _normalise(quad, 0, 1) + 0.8 * _normalise(bumps, 0, 1)
    return _normalise(f, lo, hi)


def tissue_pair(seed: int, W: int = 960, H: int = 540, disp_lo: float = 10.0,
                disp_hi: float = 110.0):
    """RGB pair of the tissue generator.  Returns (L_rgb u8 HxWx3, R_rgb u8,
    gt float64 HxW)."""
    rng = np.random.default_rng(seed)
    g = tissue_texture(rng, H, W)
    tint = np.array([1.0, 0.62, 0.55]) * rng.uniform(0.9, 1.1, 3)
    chan = np.stack([g * tint[0], g * tint[1] + 8.0, g * tint[2] + 4.0], axis=-1)
    chan = np.clip(chan, 0, 255)
    gt = tissue_disparity(rng, H, W, disp_lo, disp_hi)
    gain = rng.uniform(0.9, 1.1)
    offset = rng.uniform(-8.0, 8.0)
    right = render_right(chan, gt) * gain + offset + rng.normal(0.0, 2.0, (H, W, 3))
    L = np.clip(np.rint(chan), 0, 255).astype(np.uint8)
    R = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return L, R, gt


# ------------------------------------------------------------ batch workload

BATCH_SIZES = ((640, 480), (960, 540), (1280, 720), (1920, 1080))


def batch_pair_spec(i: int):
    """Pair i of the 64-pair mixed batch: 16 pairs of each size, disparity
    range drawn from {64, 128, 192} and window radius from {4, 5, 7} by the
    pair's seed, ground truth mapped to [0.08 D, 0.86 D]."""
    W, H = BATCH_SIZES[(i // 16) % 4]
    rng = np.random.default_rng(seed_for(3, i))
    D = int(rng.choice([64, 128, 192]))
    r = int(rng.choice([4, 5, 7]))
    return dict(W=W, H=H, D=D, r=r, seed=seed_for(3, i), lo=0.08 * D, hi=0.86 * D)


def batch_pair(i: int):
    sp = batch_pair_spec(i)
    L, R, gt = tissue_pair(sp["seed"], sp["W"], sp["H"], sp["lo"], sp["hi"])
    return L, R, gt, sp


def feature_matches(seed: int, n: int = 2000, inlier_frac: float = 0.15, shift=(6.0, -3.0),
                    noise: float = 1.0, W: int = 960, H: int = 540, max_disp: float = 120.0):
    """Synthetic feature matches between two adjacent frames: keypoints
    uniform in the image; inliers move by `shift` plus N(0, noise) per
    coordinate, outliers by a uniform displacement in [-max_disp, max_disp)^2.
    Returns (uv1 [n, 2], uv2 [n, 2], is_inlier [n]) as float32 / bool."""
    rng = np.random.default_rng(seed)
    uv1 = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n)], -1)
    inl = rng.random(n) < inlier_frac
    d = rng.uniform(-max_disp, max_disp, (n, 2))
    d[inl] = np.asarray(shift) + rng.normal(0.0, noise, (int(inl.sum()), 2))
    return uv1.astype(np.float32), (uv1 + d).astype(np.float32), inl
