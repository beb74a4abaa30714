"""Seeded synthetic stereo pairs shaped like the paper's workloads.

The paper evaluates on KITTI 2015 (about 1242x375, D = 128; Sec. V) and on 1280x384 images
(Sec. V-A, V-B). No dataset is available here, so these generators stand in for it:

* left image: uniform noise, Gaussian blur (sigma 1.5 px), min-max scaled to 0..255, uint8;
* disparity map on the left grid: piecewise-constant rectangles ("rects") or slanted planes
  over a Voronoi partition ("planes"), or a constant ("const");
* right image: the left image forward-warped to x - d (the larger d wins where several
  pixels land on one target), holes and optional vertical occlusion bands filled with fresh
  blurred noise, then a photometric change right = clip(rint(gain*right + offset + N(0,
  noise^2)), 0, 255).

Nothing here computes any part of the matching method.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.ndimage import gaussian_filter


@dataclass
class StereoPair:
    left: np.ndarray      # uint8 [H][W], reference image I_R
    right: np.ndarray     # uint8 [H][W], target image I_T
    gt: np.ndarray        # int32 [H][W], ground-truth disparity on the left grid
    valid: np.ndarray     # bool  [H][W], False where occluded / warped outside / band
    max_disp: int
    seed: int

    @property
    def shape(self):
        return self.left.shape


def blurred_noise(rng: np.random.Generator, h: int, w: int, sigma: float = 1.5) -> np.ndarray:
    """Uniform noise, Gaussian blur, min-max scaled to 0..255, rounded to uint8."""
    u = rng.random((h, w))
    b = gaussian_filter(u, sigma, mode="reflect")
    lo, hi = float(b.min()), float(b.max())
    if hi <= lo:
        return np.zeros((h, w), np.uint8)
    return np.rint((b - lo) * (255.0 / (hi - lo))).astype(np.uint8)


def _disp_rects(rng, h, w, max_disp):
    d = np.full((h, w), int(rng.integers(0, max_disp)), np.int32)
    for _ in range(int(rng.integers(4, 9))):
        rw = int(rng.integers(max(1, w // 8), max(2, w // 3) + 1))
        rh = int(rng.integers(max(1, h // 8), max(2, h // 2) + 1))
        x0 = int(rng.integers(0, max(1, w - rw + 1)))
        y0 = int(rng.integers(0, max(1, h - rh + 1)))
        d[y0:y0 + rh, x0:x0 + rw] = int(rng.integers(0, max_disp))
    return d


def _disp_planes(rng, h, w, max_disp):
    n = int(rng.integers(3, 7))
    sx = rng.uniform(0, w, n)
    sy = rng.uniform(0, h, n)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    dist = (xx[None] - sx[:, None, None]) ** 2 + (yy[None] - sy[:, None, None]) ** 2
    region = np.argmin(dist, axis=0)
    d = np.zeros((h, w), np.float64)
    for k in range(n):
        c = rng.uniform(0.15 * max_disp, 0.85 * max_disp)
        a = rng.uniform(-0.25, 0.25) * max_disp / max(w, 1)
        b = rng.uniform(-0.25, 0.25) * max_disp / max(h, 1)
        plane = a * (xx - sx[k]) + b * (yy - sy[k]) + c
        d = np.where(region == k, plane, d)
    return np.clip(np.rint(d), 0, max_disp - 1).astype(np.int32)


def make_pair(h: int, w: int, max_disp: int, seed: int, disp: str = "rects",
              const_disp: int = 7, occlusion_frac: float = 0.0,
              gain: float = 0.9, offset: float = 10.0, noise: float = 2.0) -> StereoPair:
    """Draw one seeded stereo pair; see the module docstring for the recipe."""
    rng = np.random.default_rng(seed)
    left = blurred_noise(rng, h, w)
    if disp == "rects":
        d = _disp_rects(rng, h, w, max_disp)
    elif disp == "planes":
        d = _disp_planes(rng, h, w, max_disp)
    elif disp == "const":
        d = np.full((h, w), int(const_disp), np.int32)
    else:
        raise ValueError(f"unknown disparity model {disp!r}")

    # forward warp: left (x, y) lands on right (x - d, y); the larger d (closer) wins
    right = np.zeros((h, w), np.float64)
    owner_d = np.full((h, w), -1, np.int32)
    ys, xs = np.mgrid[0:h, 0:w]
    tx = xs - d
    inside = tx >= 0
    order = np.argsort(d[inside], kind="stable")          # ascending d: later writes win
    sy, sx, stx, sd = ys[inside][order], xs[inside][order], tx[inside][order], d[inside][order]
    right[sy, stx] = left[sy, sx]
    owner_d[sy, stx] = sd
    holes = owner_d < 0
    fill = blurred_noise(rng, h, w).astype(np.float64)
    right = np.where(holes, fill, right)

    band = np.zeros(w, bool)
    if occlusion_frac > 0.0:
        total = max(1, int(round(occlusion_frac * w)))
        nb = int(rng.integers(2, 4))
        widths = np.full(nb, total // nb)
        widths[: total % nb] += 1
        for bw in widths:
            x0 = int(rng.integers(0, max(1, w - bw)))
            band[x0:x0 + bw] = True
        right[:, band] = blurred_noise(rng, h, w).astype(np.float64)[:, band]

    right = np.clip(np.rint(gain * right + offset + rng.normal(0.0, noise, (h, w))
                            if noise > 0 else np.rint(gain * right + offset)), 0, 255).astype(np.uint8)

    # valid ground truth: the left pixel lands inside, wins its target, target not in a band
    valid = np.zeros((h, w), bool)
    ok = tx >= 0
    txc = np.clip(tx, 0, w - 1)
    valid[ok] = (owner_d[ys[ok], txc[ok]] == d[ok]) & (~band[txc[ok]])
    return StereoPair(left=left, right=right, gt=d, valid=valid, max_disp=max_disp, seed=seed)


# --- the workloads: sizes, seeds and knobs of the five benchmark configurations -------------

def config_pair(name: str, seed: int | None = None) -> StereoPair:
    """The seeded pair of a named workload.

    plain_320x96     : 320x96, D = 32, rectangles, seed 1 (ZNCC + WTA only)
    paper_1280x384   : 1280x384, D = 128, slanted planes, 5% occlusion bands, seed 2
    precision_1920x1080 : 1920x1080, D = 256, slanted planes, 5% bands, seed 4
    """
    if name == "plain_320x96":
        return make_pair(96, 320, 32, 1 if seed is None else seed, disp="rects")
    if name == "paper_1280x384":
        return make_pair(384, 1280, 128, 2 if seed is None else seed, disp="planes",
                         occlusion_frac=0.05)
    if name == "precision_1920x1080":
        return make_pair(1080, 1920, 256, 4 if seed is None else seed, disp="planes",
                         occlusion_frac=0.05)
    raise ValueError(f"unknown workload {name!r}")


BATCH_SIZES = [(192, 640), (384, 1280), (375, 1242), (1080, 1920)]   # (H, W)
BATCH_DISPS = [64, 128, 192]
BATCH_WINS = [7, 9, 11]


def batch_specs(n: int = 16, seed0: int = 300):
    """Uneven batch: pair i uses seed seed0 + i; size, D and window drawn from that seed."""
    specs = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        h, w = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        d = BATCH_DISPS[int(rng.integers(0, len(BATCH_DISPS)))]
        win = BATCH_WINS[int(rng.integers(0, len(BATCH_WINS)))]
        specs.append(dict(h=h, w=w, max_disp=d, win=win, seed=seed0 + i))
    return specs


SERVE_SIZES = [(192, 640), (384, 1280), (1080, 1920)]
SERVE_DISPS = [64, 128, 256]


def serving_requests(n: int, rate_hz: float, seed: int = 5, win: int = 9):
    """Poisson arrival stream: request k has arrival time t_k, a size, D and seed 500000 + k."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for k in range(n):
        h, w = SERVE_SIZES[int(rng.integers(0, len(SERVE_SIZES)))]
        d = SERVE_DISPS[int(rng.integers(0, len(SERVE_DISPS)))]
        reqs.append(dict(t=float(t[k]), h=h, w=w, max_disp=d, win=win, seed=500000 + k))
    return reqs
