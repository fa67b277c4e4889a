"""Seeded synthetic inputs for lost-block extrapolation workloads.

This module only draws pictures, loss patterns and block lists.  It contains
none of the extrapolation arithmetic (no weighting, no transforms, no
iterations), so the FP64 oracle and the CUDA path can both be fed from it
without sharing any of the method.

The paper evaluates on natural test images that are not available here
(Sec. 4); these generators stand in for them with content that exercises the
same behaviour: smooth gradients, oriented periodic texture, straight edges of
piecewise-constant regions, and sensor-like noise, quantised to 8 bit.

All generators use ``numpy.random.Generator(PCG64(seed))``; the default seed of
workload ``i`` is ``220701205 + i``.

Coordinates: ``m`` is the row (y), ``n`` the column (x).  Frames are float32
arrays holding 8-bit values (exact in float32) unless noted.  Availability
masks are uint8 (1 = usable sample, 0 = lost).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 220701205


def rng_for(index: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index if seed is None else seed))


# ----------------------------------------------------------------------------
# single block (small FP64 case)
# ----------------------------------------------------------------------------

def single_block_area(rng: np.random.Generator, size: int = 48, center: float = 23.5):
    """A ``size``x``size`` area: 128 + 40 sin(2pi(0.07m + 0.03n)) + a +50 step
    edge through the centre at a random angle + N(0, 2^2), clipped to
    [0, 255], not rounded.  Returns float64."""
    m, n = np.meshgrid(np.arange(size, dtype=np.float64), np.arange(size, dtype=np.float64),
                       indexing="ij")
    theta = rng.uniform(0.0, math.pi)
    f = 128.0 + 40.0 * np.sin(2.0 * math.pi * (0.07 * m + 0.03 * n))
    f += 50.0 * (((m - center) * math.cos(theta) + (n - center) * math.sin(theta)) > 0)
    f += rng.normal(0.0, 2.0, size=f.shape)
    return np.clip(f, 0.0, 255.0)


# ----------------------------------------------------------------------------
# natural-image stand-in
# ----------------------------------------------------------------------------

def _star_polygon(rng, cx, cy, extent):
    k = int(rng.integers(3, 9))
    ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, size=k))
    rad = rng.uniform(0.25 * extent, 0.5 * extent, size=k)
    return np.stack([cy + rad * np.sin(ang), cx + rad * np.cos(ang)], axis=1)  # (k, 2) rows, cols


def _fill_polygon(img, poly, value):
    """Even-odd rule rasterisation of a simple polygon into ``img`` (adds value)."""
    h, w = img.shape
    y0 = max(int(math.floor(poly[:, 0].min())), 0)
    y1 = min(int(math.ceil(poly[:, 0].max())) + 1, h)
    x0 = max(int(math.floor(poly[:, 1].min())), 0)
    x1 = min(int(math.ceil(poly[:, 1].max())) + 1, w)
    if y0 >= y1 or x0 >= x1:
        return
    yy, xx = np.meshgrid(np.arange(y0, y1) + 0.5, np.arange(x0, x1) + 0.5, indexing="ij")
    inside = np.zeros(yy.shape, dtype=bool)
    k = len(poly)
    for i in range(k):
        ay, ax = poly[i]
        by, bx = poly[(i + 1) % k]
        cond = (ay > yy) != (by > yy)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = ax + (yy - ay) * (bx - ax) / (by - ay)
        inside ^= cond & (xx < xint)
    img[y0:y1, x0:x1] += value * inside


def natural_frame(rng: np.random.Generator, height: int, width: int, *, n_sines: int = 12,
                  n_polys: int = 30, noise_sigma: float = 2.0, canvas_margin: int = 0):
    """8-bit grayscale stand-in for a natural image.

    base 128; ``n_sines`` oriented sinusoids (period log-uniform in [4, 64] px,
    orientation U[0, pi), phase U[0, 2pi), amplitude U[5, 20]);
    ``n_polys`` random simple (star-shaped) polygons with 3-8 vertices, extent
    20-300 px, constant offset U[-40, 40]; noise N(0, sigma^2); clipped to
    [0, 255] and rounded.  Returns float32 of shape (height + 2*margin,
    width + 2*margin).
    """
    H, W = height + 2 * canvas_margin, width + 2 * canvas_margin
    img = np.full((H, W), 128.0, dtype=np.float64)
    m = np.arange(H, dtype=np.float64)[:, None]
    n = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(n_sines):
        period = math.exp(rng.uniform(math.log(4.0), math.log(64.0)))
        phi = rng.uniform(0.0, math.pi)
        psi = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.uniform(5.0, 20.0)
        img += amp * np.sin(2.0 * math.pi * (m * math.cos(phi) + n * math.sin(phi)) / period + psi)
    for _ in range(n_polys):
        extent = rng.uniform(20.0, 300.0)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        _fill_polygon(img, _star_polygon(rng, cx, cy, extent), rng.uniform(-40.0, 40.0))
    img += rng.normal(0.0, noise_sigma, size=img.shape)
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.float32)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class PlanSpec:
    """Extrapolation parameters of one block class (Sec. 4 notation:
    lost block b x b, support border width, T x T FFT, rho-hat, gamma, I)."""
    block: int
    border: int
    fft_size: int
    rho: float
    gamma: float
    iters: int
    support: int = 0  # 0 = full frame around B, 1 = causal L shape (top/left)
    compensation: int = 0  # 0 = constant gamma (FOFSE, Eq. 14), 1 = OFSE's (Eq. 10-12)
    basis: int = 0  # 0 = 2-D DFT, 1 = 2-D DCT-II

    def __post_init__(self):
        # rho and gamma cross the C ABI as single-precision numbers: hold the
        # single-precision values so that every consumer of the spec sees the
        # same parameters
        self.rho = float(np.float32(self.rho))
        self.gamma = float(np.float32(self.gamma))


@dataclasses.dataclass
class Workload:
    name: str
    frame: np.ndarray          # (H, W) float32 observed frame (lost samples hold `fill`)
    truth: np.ndarray          # (H, W) float32 ground truth
    avail: np.ndarray          # (H, W) uint8
    blocks: np.ndarray         # (n, 3) int32: y, x (top-left of B), plan index
    plans: list                # list[PlanSpec]
    precision: str = "fp32"

    @property
    def n_blocks(self):
        return int(self.blocks.shape[0])


def _mark_lost(frame, avail, blocks, plans, fill):
    for (y, x, p) in blocks:
        b = plans[p].block
        avail[y:y + b, x:x + b] = 0
        frame[y:y + b, x:x + b] = fill


def single_block(seed: int | None = None, *, iters: int = 100, gamma: float = 0.5,
                 rho: float = 0.8, fill: float = 0.0) -> Workload:
    """One 16x16 lost block inside a 48x48 area (border 16), 64x64 FFT."""
    rng = rng_for(0, seed)
    truth = single_block_area(rng).astype(np.float64)
    plans = [PlanSpec(16, 16, 64, rho, gamma, iters)]
    blocks = np.array([[16, 16, 0]], dtype=np.int32)
    avail = np.ones(truth.shape, dtype=np.uint8)
    frame = truth.copy()
    _mark_lost(frame, avail, blocks, plans, fill)
    return Workload("single-16x16-T64-fp64", frame, truth, avail, blocks, plans, "fp64")


def frame_concealment(seed: int | None = None, *, height: int = 1080, width: int = 1920,
                      loss: float = 0.10, iters: int = 200, gamma: float = 0.5, rho: float = 0.8,
                      fill: float = 0.0) -> Workload:
    """10 % of the full 16x16 tiles of a 1920x1080 frame lost uniformly at
    random (exactly round(loss * tiles), without replacement); border 16,
    64x64 FFT; lost neighbours are unavailable."""
    rng = rng_for(1, seed)
    truth = natural_frame(rng, height, width)
    ty, tx = height // 16, width // 16
    n_lost = int(round(loss * ty * tx))
    pick = np.sort(rng.choice(ty * tx, size=n_lost, replace=False))
    blocks = np.stack([(pick // tx) * 16, (pick % tx) * 16, np.zeros_like(pick)], axis=1).astype(np.int32)
    plans = [PlanSpec(16, 16, 64, rho, gamma, iters)]
    avail = np.ones(truth.shape, dtype=np.uint8)
    frame = truth.copy()
    _mark_lost(frame, avail, blocks, plans, fill)
    return Workload(f"conceal-{width}x{height}-16x16-T64-I{iters}", frame, truth, avail, blocks,
                    plans)


MIXED_CLASSES = (  # (block, border, fft, iters)
    (4, 4, 32, 50),
    (8, 8, 32, 100),
    (16, 16, 64, 200),
    (32, 16, 128, 400),
)


def uneven_batch(seed: int | None = None, *, height: int = 2160, width: int = 3840,
                 loss: float = 0.20, gamma: float = 0.5, rho: float = 0.8, fill: float = 0.0,
                 classes=MIXED_CLASSES) -> Workload:
    """Burst losses until ``loss`` of the frame area is gone.  Each burst picks
    a class uniformly and a length U{1..8}; the burst runs in raster order on
    that class's block grid from a random start and only takes blocks that do
    not overlap earlier losses."""
    rng = rng_for(2, seed)
    truth = natural_frame(rng, height, width)
    plans = [PlanSpec(b, br, t, rho, gamma, it) for (b, br, t, it) in classes]
    lost = np.zeros((height, width), dtype=bool)
    blocks = []
    target = loss * height * width
    area = 0
    while area < target:
        c = int(rng.integers(0, len(plans)))
        b = plans[c].block
        gy, gx = height // b, width // b
        length = int(rng.integers(1, 9))
        start = int(rng.integers(0, gy * gx))
        for j in range(start, min(start + length, gy * gx)):
            y, x = (j // gx) * b, (j % gx) * b
            if lost[y:y + b, x:x + b].any():
                continue
            lost[y:y + b, x:x + b] = True
            blocks.append((y, x, c))
            area += b * b
            if area >= target:
                break
    blocks = np.array(blocks, dtype=np.int32)
    avail = (~lost).astype(np.uint8)
    frame = truth.copy()
    frame[lost] = fill
    return Workload(f"uneven-{width}x{height}-4/8/16/32", frame, truth, avail, blocks, plans)


def prediction_sequence(seed: int | None = None, *, n_frames: int = 64, height: int = 720,
                        width: int = 1280, iters: int = 64, gamma: float = 0.5, rho: float = 0.8,
                        max_step: int = 4):
    """Frames for causal block prediction: crops of one larger canvas, each
    translated by a cumulative random integer offset of 0..max_step px per
    axis.  Every 8x8 block of every frame is predicted from its causal
    L-shaped support (top/left, border 8, 24x24 area, 32x32 FFT).

    Returns (frames (n_frames, H, W) float32, blocks (n, 3) int32, plans)."""
    rng = rng_for(4, seed)
    margin = n_frames * max_step + 8
    canvas = natural_frame(rng, height + margin, width + margin)
    steps = rng.integers(0, max_step + 1, size=(n_frames, 2))
    offs = np.cumsum(steps, axis=0) - steps[0]
    frames = np.stack([canvas[oy:oy + height, ox:ox + width] for (oy, ox) in offs]).astype(np.float32)
    by, bx = np.meshgrid(np.arange(0, height, 8), np.arange(0, width, 8), indexing="ij")
    blocks = np.stack([by.ravel(), bx.ravel(), np.zeros(by.size, dtype=np.int64)], axis=1).astype(np.int32)
    plans = [PlanSpec(8, 8, 32, rho, gamma, iters, support=1)]
    return frames, blocks, plans


def small_frame(seed: int, *, height: int = 96, width: int = 128, n_lost: int = 6,
                plan: PlanSpec | None = None, fill: float = 0.0, edge_blocks: bool = True) -> Workload:
    """A small frame with a handful of lost blocks, including blocks at the
    frame border (partial support) when ``edge_blocks``; for tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    plan = plan or PlanSpec(16, 16, 64, 0.8, 0.5, 50)
    b = plan.block
    truth = natural_frame(rng, height, width, n_sines=6, n_polys=4)
    gy, gx = height // b, width // b
    cells = rng.choice(gy * gx, size=n_lost, replace=False)
    if edge_blocks:
        cells[0] = 0                      # top-left corner
        if n_lost > 1:
            cells[1] = gy * gx - 1        # bottom-right corner
    cells = np.unique(cells)
    blocks = np.stack([(cells // gx) * b, (cells % gx) * b, np.zeros_like(cells)], axis=1).astype(np.int32)
    avail = np.ones(truth.shape, dtype=np.uint8)
    frame = truth.copy()
    _mark_lost(frame, avail, blocks, [plan], fill)
    return Workload(f"small-{width}x{height}", frame, truth, avail, blocks, [plan])


# ----------------------------------------------------------------------------
# video volumes
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class VolumePlanSpec:
    """Parameters of extrapolation over video volumes: lost block b x b in one
    frame, spatial border, ``depth`` frames on each side of it, a
    T x T x Tt DFT grid (T = fft_size, Tt = fft_time), rho-hat, gamma, I."""
    block: int
    border: int
    depth: int
    fft_size: int
    fft_time: int
    rho: float
    gamma: float
    iters: int

    def __post_init__(self):
        self.rho = float(np.float32(self.rho))
        self.gamma = float(np.float32(self.gamma))


@dataclasses.dataclass
class VideoWorkload:
    name: str
    video: np.ndarray          # (F, H, W) float32 observed frames (lost samples hold `fill`)
    truth: np.ndarray          # (F, H, W) float32 ground truth
    avail: np.ndarray          # (F, H, W) uint8
    blocks: np.ndarray         # (n, 3) int32: frame t, y, x (top-left of B)
    plan: VolumePlanSpec

    @property
    def n_blocks(self):
        return int(self.blocks.shape[0])


def moving_frames(rng: np.random.Generator, n_frames: int, height: int, width: int, *,
                  max_step: int = 2, noise_sigma: float = 2.0, **frame_kw) -> np.ndarray:
    """Frames of a camera pan: crops of one natural_frame canvas, frame i
    offset from frame i-1 by a random integer step of 0..max_step px per axis,
    each with its own sensor noise N(0, sigma^2), clipped and rounded to 8 bit.
    Returns float32 (n_frames, height, width)."""
    margin = n_frames * max_step
    canvas = natural_frame(rng, height + margin, width + margin, noise_sigma=0.0, **frame_kw)
    steps = rng.integers(0, max_step + 1, size=(n_frames, 2))
    offs = np.cumsum(steps, axis=0) - steps[0]
    out = np.empty((n_frames, height, width), dtype=np.float32)
    for i, (oy, ox) in enumerate(offs):
        f = canvas[oy:oy + height, ox:ox + width].astype(np.float64)
        f += rng.normal(0.0, noise_sigma, size=f.shape)
        out[i] = np.rint(np.clip(f, 0.0, 255.0))
    return out


def _lose_tiles(rng, avail, frame_index, b, loss):
    """Pick round(loss * tiles) of frame frame_index's full b x b tiles."""
    _, H, W = avail.shape
    ty, tx = H // b, W // b
    n = int(round(loss * ty * tx))
    pick = np.sort(rng.choice(ty * tx, size=n, replace=False))
    return np.stack([np.full_like(pick, frame_index), (pick // tx) * b, (pick % tx) * b], axis=1)


def video_concealment(seed: int | None = None, *, n_frames: int = 3, height: int = 1080,
                      width: int = 1920, loss: float = 0.10, plan: VolumePlanSpec | None = None,
                      fill: float = 0.0) -> VideoWorkload:
    """A camera pan of ``n_frames`` 1920x1080 frames; in every frame 10 % of
    the full 16x16 tiles are lost uniformly at random and independently of
    the other frames.  The blocks to conceal are the centre frame's; those of
    the other frames only make samples of the volumes unusable.  Plan: border
    8 (32x32 spatial area), one frame on each side (depth 1), 32x32x4 DFT,
    rho 0.8, gamma 0.5, 200 iterations."""
    rng = rng_for(5, seed)
    plan = plan or VolumePlanSpec(16, 8, 1, 32, 4, 0.8, 0.5, 200)
    b = plan.block
    truth = moving_frames(rng, n_frames, height, width)
    avail = np.ones(truth.shape, dtype=np.uint8)
    video = truth.copy()
    tc = n_frames // 2
    lost = [_lose_tiles(rng, avail, t, b, loss) for t in range(n_frames)]
    for tiles in lost:
        for (t, y, x) in tiles:
            avail[t, y:y + b, x:x + b] = 0
            video[t, y:y + b, x:x + b] = fill
    blocks = lost[tc].astype(np.int32)
    return VideoWorkload(f"video-{n_frames}x{width}x{height}-16x16-T{plan.fft_size}x{plan.fft_time}"
                         f"-I{plan.iters}", video, truth, avail, blocks, plan)


def small_video(seed: int, *, n_frames: int = 3, height: int = 64, width: int = 96,
                n_lost: int = 5, plan: VolumePlanSpec | None = None,
                fill: float = 0.0) -> VideoWorkload:
    """A few frames with a handful of lost blocks in every frame; the blocks to
    conceal include the corners of the first and last frames (volumes that
    reach beyond the video in space and time); for tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    plan = plan or VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 40)
    b = plan.block
    truth = moving_frames(rng, n_frames, height, width, n_sines=6, n_polys=4)
    gy, gx = height // b, width // b
    avail = np.ones(truth.shape, dtype=np.uint8)
    video = truth.copy()
    blocks = []
    for t in range(n_frames):
        cells = rng.choice(gy * gx, size=min(n_lost, gy * gx), replace=False)
        if t == 0:
            cells[0] = 0
        if t == n_frames - 1:
            cells[0] = gy * gx - 1
        for c in np.unique(cells):
            y, x = (c // gx) * b, (c % gx) * b
            avail[t, y:y + b, x:x + b] = 0
            video[t, y:y + b, x:x + b] = fill
            blocks.append((t, y, x))
    return VideoWorkload(f"small-video-{n_frames}x{width}x{height}", video, truth, avail,
                         np.array(blocks, dtype=np.int32), plan)
