"""Seeded synthetic inputs for the rasterizer: Gaussian sets, cameras, block AABBs.

This module only draws random numbers and builds camera poses. It holds none of
the rasterizer's arithmetic (no projection, no compositing, no gradients), so the
FP64 oracle (``oracle/``) and the CUDA path (``paper_2510_01767_b300``) can both
consume exactly the same bytes without sharing any method code.

The paper's datasets (MatrixCity-Aerial, Mill19, UrbanScene3D; Sec. 5.1) are not
available, so every workload here is synthetic. Each generator reproduces the
*shape* of one workload: Gaussian counts, spatial layout, scale and opacity
distributions, image resolutions and camera poses.

All arrays are float32 (the rasterizer's parameter precision). Layouts:
  means [N,3], log_scales [N,3], quats [N,4] as (w,x,y,z) un-normalised,
  opacity_logits [N], sh [N,16,3] (real SH, band-major, DC first).
Cameras are dicts with a 4x4 row-major world->camera ``viewmat`` (OpenCV axes:
x right, y down, +z forward), pinhole ``fx, fy, cx, cy``, ``width, height``,
``near``, ``far``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_COEFFS = 16


@dataclass
class GaussianSet:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    crop_mask: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "GaussianSet":
        idx = np.asarray(idx)
        return GaussianSet(
            self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
            self.opacity_logits[idx].copy(), self.sh[idx].copy(),
            None if self.crop_mask is None else self.crop_mask[idx].copy())

    def arrays(self):
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logits=self.opacity_logits, sh=self.sh)


@dataclass
class Camera:
    viewmat: np.ndarray  # [4,4] float32 row-major world->camera
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01
    far: float = 1e10

    def as_dict(self):
        return dict(viewmat=self.viewmat, fx=self.fx, fy=self.fy, cx=self.cx, cy=self.cy,
                    width=self.width, height=self.height, near=self.near, far=self.far)


@dataclass
class AABB:
    lo: tuple = (-math.inf, -math.inf, -math.inf)
    hi: tuple = (math.inf, math.inf, math.inf)


@dataclass
class Workload:
    """A set of render items: (gaussian set, camera, block) triples."""
    name: str
    sets: list
    cameras: list
    blocks: list
    items: list  # list of (set_index, camera_index, block_index)
    tile: tuple = (16, 16)
    extra: dict = field(default_factory=dict)

    @property
    def pixels(self) -> int:
        return sum(self.cameras[c].width * self.cameras[c].height for _, c, _ in self.items)

    @property
    def gaussians(self) -> int:
        return sum(self.sets[s].n for s, _, _ in self.items)


# --------------------------------------------------------------------------- poses

def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera matrix (OpenCV axes) for a camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:  # looking straight along up: pick any right vector
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = -R @ eye
    return V.astype(np.float32)


def pinhole(width, height, fx, fy=None, cx=None, cy=None, viewmat=None, near=0.01, far=1e10) -> Camera:
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    vm = np.eye(4, dtype=np.float32) if viewmat is None else np.asarray(viewmat, np.float32)
    return Camera(vm, float(fx), float(fy), float(cx), float(cy), int(width), int(height), near, far)


# --------------------------------------------------------------------------- appearance

def random_quats(rng, n) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def random_sh(rng, n, dc_mean=0.5, dc_std=0.2, rest_std=0.05) -> np.ndarray:
    sh = np.empty((n, SH_COEFFS, 3), np.float32)
    sh[:, 0, :] = rng.normal(dc_mean, dc_std, (n, 3))
    sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, SH_COEFFS - 1, 3))
    return sh


def uniform_gaussians(rng, n, xy_half, z_lo, z_hi, logscale_lo=-4.0, logscale_hi=-2.0,
                      logscale_shift=0.0) -> GaussianSet:
    means = np.empty((n, 3), np.float32)
    means[:, 0] = rng.uniform(-xy_half, xy_half, n)
    means[:, 1] = rng.uniform(-xy_half, xy_half, n)
    means[:, 2] = rng.uniform(z_lo, z_hi, n)
    log_scales = (rng.uniform(logscale_lo, logscale_hi, (n, 3)) + logscale_shift).astype(np.float32)
    quats = random_quats(rng, n)
    logits = rng.standard_normal(n).astype(np.float32)
    sh = random_sh(rng, n)
    return GaussianSet(means, log_scales, quats, logits, sh)


# --------------------------------------------------------------------------- workloads

def small_scene(seed=0, n=1000) -> Workload:
    """1,000 Gaussians in front of a 128x128 pinhole (fx=fy=128, identity pose), 16x16 tiles.

    means x,y ~ U(-1,1), z ~ U(2,6); log-scales ~ U(-4,-2); random unit quaternions;
    opacity = sigmoid(N(0,1)); SH DC ~ N(0.5,0.2), higher bands ~ N(0,0.05).
    """
    rng = np.random.default_rng(seed)
    g = uniform_gaussians(rng, n, 1.0, 2.0, 6.0)
    cam = pinhole(128, 128, 128.0, cx=64.0, cy=64.0)
    return Workload("small_1k_128px", [g], [cam], [AABB()], [(0, 0, 0)], (16, 16))


def medium_scene(seed=0, n=200_000) -> Workload:
    """200k Gaussians in a 20 m box (x,y ~ U(-10,10), z ~ U(5,50)), 1600x1066 pinhole, fx=fy=1200.

    Log-scales are the small-scene distribution shifted by ln(10) (scaled with the box).
    """
    rng = np.random.default_rng(seed)
    g = uniform_gaussians(rng, n, 10.0, 5.0, 50.0, logscale_shift=math.log(10.0))
    cam = pinhole(1600, 1066, 1200.0, cx=800.0, cy=533.0)
    return Workload("medium_200k_1600x1066", [g], [cam], [AABB()], [(0, 0, 0)], (16, 16))


def perturbed_copy(g: GaussianSet, seed=2, sigma=0.01) -> GaussianSet:
    rng = np.random.default_rng(seed)
    h = g.subset(np.arange(g.n))
    h.means = (h.means + rng.normal(0.0, sigma, h.means.shape)).astype(np.float32)
    return h


def _quat_from_rotmat(R) -> np.ndarray:
    """Batch rotation matrices [n,3,3] -> quaternions (w,x,y,z)."""
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    w = np.sqrt(np.maximum(0.0, 1.0 + tr)) / 2
    x = np.sqrt(np.maximum(0.0, 1.0 + R[:, 0, 0] - R[:, 1, 1] - R[:, 2, 2])) / 2
    y = np.sqrt(np.maximum(0.0, 1.0 - R[:, 0, 0] + R[:, 1, 1] - R[:, 2, 2])) / 2
    z = np.sqrt(np.maximum(0.0, 1.0 - R[:, 0, 0] - R[:, 1, 1] + R[:, 2, 2])) / 2
    x = np.copysign(x, R[:, 2, 1] - R[:, 1, 2])
    y = np.copysign(y, R[:, 0, 2] - R[:, 2, 0])
    z = np.copysign(z, R[:, 1, 0] - R[:, 0, 1])
    q[:, 0], q[:, 1], q[:, 2], q[:, 3] = w, x, y, z
    return q


def city_layout(seed=0, n=4_000_000, extent=500.0, n_boxes=200) -> GaussianSet:
    """Synthetic city: 60% of Gaussians on the ground plane z=0, 40% on the faces of
    ``n_boxes`` axis-aligned boxes (footprint U(10,40) m, height U(10,80) m) over a
    ``extent`` x ``extent`` m area. Density along x rises 10x across the area
    (pdf proportional to 1 + 9 (x + extent/2) / extent). Surface Gaussians are flattened along
    the surface normal (normal-axis log-scale 2.3 below the in-plane ones);
    in-plane log-scales ~ U(ln 0.05, ln 0.5).
    """
    rng = np.random.default_rng(seed)
    half = extent / 2.0

    def sample_x(k):
        # inverse CDF of p(t) ~ 1 + 9 t on t in [0,1]:  F(t) = (t + 4.5 t^2) / 5.5
        u = rng.uniform(0.0, 1.0, k)
        t = (-1.0 + np.sqrt(1.0 + 4 * 4.5 * 5.5 * u)) / (2 * 4.5)
        return -half + extent * t

    n_ground = int(round(0.6 * n))
    n_facade = n - n_ground
    means = np.empty((n, 3))
    normal_axis = np.empty(n, np.int64)
    means[:n_ground, 0] = sample_x(n_ground)
    means[:n_ground, 1] = rng.uniform(-half, half, n_ground)
    means[:n_ground, 2] = 0.0
    normal_axis[:n_ground] = 2

    # boxes: centres follow the same density gradient
    bx = sample_x(n_boxes)
    by = rng.uniform(-half, half, n_boxes)
    bw = rng.uniform(10.0, 40.0, n_boxes)
    bd = rng.uniform(10.0, 40.0, n_boxes)
    bh = rng.uniform(10.0, 80.0, n_boxes)
    # facade Gaussians per box proportional to lateral area
    area = 2 * (bw + bd) * bh
    box_of = rng.choice(n_boxes, n_facade, p=area / area.sum())
    # choose a face proportional to its width: faces 0,1 -> normal x (width bd), 2,3 -> normal y (width bw)
    wx = bd[box_of]
    wy = bw[box_of]
    face_is_x = rng.uniform(0, 1, n_facade) < wx / (wx + wy)
    side = np.where(rng.uniform(0, 1, n_facade) < 0.5, -1.0, 1.0)
    s_along = rng.uniform(-0.5, 0.5, n_facade)
    h = rng.uniform(0.0, 1.0, n_facade) * bh[box_of]
    fx_ = np.where(face_is_x, bx[box_of] + side * bw[box_of] / 2, bx[box_of] + s_along * bw[box_of])
    fy_ = np.where(face_is_x, by[box_of] + s_along * bd[box_of], by[box_of] + side * bd[box_of] / 2)
    means[n_ground:, 0] = fx_
    means[n_ground:, 1] = fy_
    means[n_ground:, 2] = h
    normal_axis[n_ground:] = np.where(face_is_x, 0, 1)

    log_scales = rng.uniform(math.log(0.05), math.log(0.5), (n, 3))
    # local frame: local z is the flattened axis; rotate local z onto the surface normal,
    # then spin randomly about the normal.
    log_scales[:, 2] -= 2.3
    theta = rng.uniform(0, 2 * math.pi, n)
    c, s = np.cos(theta), np.sin(theta)
    Rspin = np.zeros((n, 3, 3))
    Rspin[:, 0, 0], Rspin[:, 0, 1], Rspin[:, 1, 0], Rspin[:, 1, 1], Rspin[:, 2, 2] = c, -s, s, c, 1.0
    # columns of Ralign map local (x,y,z) to world; local z -> normal
    Ralign = np.zeros((n, 3, 3))
    m0 = normal_axis == 0  # normal = world x: local x->world y, local y->world z, local z->world x
    Ralign[m0] = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], float)
    m1 = normal_axis == 1  # normal = world y: local x->world z, local y->world x, local z->world y
    Ralign[m1] = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], float)
    m2 = normal_axis == 2
    Ralign[m2] = np.eye(3)
    R = Ralign @ Rspin
    quats = _quat_from_rotmat(R)

    logits = rng.standard_normal(n)
    sh = random_sh(rng, n)
    perm = rng.permutation(n)  # interleave ground and facades in memory
    return GaussianSet(means[perm].astype(np.float32), log_scales[perm].astype(np.float32),
                       quats[perm].astype(np.float32), logits[perm].astype(np.float32), sh[perm])


def block_aabb_fraction(means, frac=0.25, center=(0.0, 0.0)) -> AABB:
    """Axis-aligned x,y box around ``center`` holding about ``frac`` of ``means`` (z unbounded)."""
    d = np.maximum(np.abs(means[:, 0] - center[0]), np.abs(means[:, 1] - center[1]))
    r = float(np.quantile(d, frac))
    return AABB((center[0] - r, center[1] - r, -math.inf), (center[0] + r, center[1] + r, math.inf))


def aerial_camera(target, altitude, pitch_deg, heading_deg, width, height, f, distance=None) -> Camera:
    """Oblique aerial camera at ``altitude`` above ground, pitched ``pitch_deg`` down, looking at ``target``."""
    target = np.asarray(target, np.float64)
    pitch = math.radians(pitch_deg)
    heading = math.radians(heading_deg)
    horiz = altitude / math.tan(pitch) if distance is None else distance
    eye = target + np.array([-horiz * math.cos(heading), -horiz * math.sin(heading), altitude - target[2]])
    return pinhole(width, height, f, viewmat=look_at(eye, target))


def city_block_scene(seed=0, n=4_000_000) -> Workload:
    """4M-Gaussian city; one block AABB holding ~25% of Gaussians; one 1920x1080
    oblique aerial view (fx=fy=1400, 150 m altitude, 45 deg pitch) at the block centre."""
    g = city_layout(seed, n)
    block = block_aabb_fraction(g.means, 0.25)
    c = ((block.lo[0] + block.hi[0]) / 2, (block.lo[1] + block.hi[1]) / 2, 0.0)
    cam = aerial_camera(c, 150.0, 45.0, 30.0, 1920, 1080, 1400.0)
    return Workload("city_4M_1920x1080", [g], [cam], [block], [(0, 0, 0)], (16, 16))


BATCH_RESOLUTIONS = [(640, 480), (800, 600), (1024, 768), (1280, 720),
                     (1280, 960), (1600, 900), (1600, 1066), (1920, 1080)]


def kd_median_leaves(means, depth=2):
    """Median KD split on x then y (``depth`` levels) -> list of (index array, AABB)."""
    leaves = [(np.arange(means.shape[0]), AABB())]
    for level in range(depth):
        axis = level % 2
        nxt = []
        for idx, box in leaves:
            cut = float(np.median(means[idx, axis]))
            left = idx[means[idx, axis] < cut]
            right = idx[means[idx, axis] >= cut]
            lo, hi = list(box.lo), list(box.hi)
            hl = list(hi)
            hl[axis] = cut
            lr = list(lo)
            lr[axis] = cut
            nxt.append((left, AABB(tuple(lo), tuple(hl))))
            nxt.append((right, AABB(tuple(lr), tuple(hi))))
        leaves = nxt
    return leaves


def multi_block_scene(seed=0, block_sizes=(500_000, 1_000_000, 2_000_000, 3_000_000),
                      views_per_block=4, city_n=None) -> Workload:
    """Four KD blocks of the city layout subsampled to 0.5/1/2/3 M Gaussians and 16 views
    (4 per block) of uneven resolution (640x480 ... 1920x1080, each size twice) from random
    oblique poses at 120-180 m altitude looking at the block."""
    rng = np.random.default_rng(seed + 1)
    total = sum(block_sizes)
    # median KD leaves hold ~1/4 of the city each: the largest block needs 4x its size
    city = city_layout(seed, city_n if city_n is not None else int(max(block_sizes) * 4 * 1.05))
    leaves = kd_median_leaves(city.means, 2)
    order = np.argsort([len(ix) for ix, _ in leaves])
    sets, blocks, cams, items = [], [], [], []
    res = BATCH_RESOLUTIONS * 2
    rng.shuffle(res)
    for b, (size, li) in enumerate(zip(block_sizes, order)):
        idx, box = leaves[li]
        take = rng.choice(idx, size=min(size, len(idx)), replace=False)
        take.sort()
        sets.append(city.subset(take))
        blocks.append(box)
        cxy = city.means[take, :2].mean(axis=0)
        for v in range(views_per_block):
            w, h = res[len(cams) % len(res)]
            cam = aerial_camera((cxy[0], cxy[1], 0.0), rng.uniform(120, 180), rng.uniform(35, 60),
                                rng.uniform(0, 360), w, h, 1.1 * w)
            items.append((b, len(cams), b))
            cams.append(cam)
    return Workload("multi_block_4x_16views", sets, cams, blocks, items, (16, 16))


def training_scene(seed=0, n=2_000_000, n_views=64, width=1280, height=720):
    """Hidden ground-truth 2M-Gaussian city block, 64 views around it, and a perturbed init
    (means + N(0, 0.1 m), SH DC reset to 0.5 + N(0, 0.05), opacity logit 0)."""
    rng = np.random.default_rng(seed + 7)
    city = city_layout(seed, int(n * 4.2))
    block = block_aabb_fraction(city.means, n / city.n)
    inside = np.nonzero((city.means[:, 0] >= block.lo[0]) & (city.means[:, 0] < block.hi[0]) &
                        (city.means[:, 1] >= block.lo[1]) & (city.means[:, 1] < block.hi[1]))[0]
    take = np.sort(rng.choice(inside, size=min(n, len(inside)), replace=False))
    gt = city.subset(take)
    c = gt.means[:, :2].mean(axis=0)
    cams = []
    for k in range(n_views):
        cams.append(aerial_camera((c[0], c[1], 0.0), rng.uniform(120, 180), rng.uniform(35, 60),
                                  360.0 * k / n_views, width, height, 1.1 * width))
    init = gt.subset(np.arange(gt.n))
    init.means = (init.means + rng.normal(0, 0.1, init.means.shape)).astype(np.float32)
    init.sh[:, 0, :] = rng.normal(0.5, 0.05, (init.n, 3)).astype(np.float32)
    init.sh[:, 1:, :] = 0.0
    init.opacity_logits[:] = 0.0
    return gt, init, cams, block


def random_upstream(rng, workload: Workload) -> list:
    """Seeded dL/dC images, one planar [3,H,W] float32 array per item."""
    out = []
    for _, c, _ in workload.items:
        cam = workload.cameras[c]
        out.append(rng.standard_normal((3, cam.height, cam.width)).astype(np.float32))
    return out
