"""Shared test helpers: moving oracle data to the GPU path's layouts and comparing results.

Tolerances (the parity bar): image max-abs error 1e-4 on pixels whose compositing decisions
are not marginal; gradient relative error 1e-3, measured per element as
|gpu - oracle| / max(|oracle|, 1e-3 * max|oracle of that tensor|) -- the floor keeps
near-zero elements of a float32 sum over thousands of pixels from dominating the ratio.
"""
from __future__ import annotations

import numpy as np

import oracle

IMG_ATOL = 1e-4
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-3

# largest error seen per named check in this session (printed at the end of the run)
REPORT: dict = {}


def record(name, value):
    REPORT[name] = max(REPORT.get(name, 0.0), float(value))
    return value


def assert_img_close(gpu, orc, name):
    """Max-abs image error (parity bar 1e-4), recorded under `name`."""
    d = float(np.abs(np.asarray(gpu, np.float64) - np.asarray(orc, np.float64)).max()) if np.size(orc) else 0.0
    record(name, d)
    assert d <= IMG_ATOL, f"{name}: max-abs error {d:.3e} > {IMG_ATOL}"
    return d


def rect_tiles(mean2d, radius, cam, tile):
    """Tile rectangle area of each splat, computed exactly from float32 u, v and integer r."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    gx = -(-c["width"] // tile[0])
    gy = -(-c["height"] // tile[1])
    u = mean2d[:, 0].astype(np.float32).astype(np.float64)
    v = mean2d[:, 1].astype(np.float32).astype(np.float64)
    r = radius.astype(np.float64)
    x0 = np.clip(np.floor((u - r) / tile[0]), 0, gx)
    x1 = np.clip(np.ceil((u + r) / tile[0]), 0, gx)
    y0 = np.clip(np.floor((v - r) / tile[1]), 0, gy)
    y1 = np.clip(np.ceil((v + r) / tile[1]), 0, gy)
    t = ((x1 - x0) * (y1 - y0)).astype(np.int32)
    t[radius <= 0] = 0
    return t


def rect_of(mean2d, radius, cam, tile):
    """[n,4] tile rectangles (x0, y0, x1, y1) from float32 u, v and integer r (exact)."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    gx = -(-c["width"] // tile[0])
    gy = -(-c["height"] // tile[1])
    u = mean2d[:, 0].astype(np.float32).astype(np.float64)
    v = mean2d[:, 1].astype(np.float32).astype(np.float64)
    r = radius.astype(np.float64)
    out = np.stack([np.clip(np.floor((u - r) / tile[0]), 0, gx), np.clip(np.floor((v - r) / tile[1]), 0, gy),
                    np.clip(np.ceil((u + r) / tile[0]), 0, gx), np.clip(np.ceil((v + r) / tile[1]), 0, gy)], 1)
    out[radius <= 0] = 0
    return out.astype(np.int32)


def differing_rects(p: oracle.Projection, gpu_mean2d, gpu_radius, cam, tile) -> np.ndarray:
    """Gaussians whose tile rectangle differs between the GPU projection and the oracle's
    (float32 took a marginal radius / rectangle / culling decision the other way)."""
    a = rect_of(gpu_mean2d, gpu_radius, cam, tile)
    b = np.where((p.radius > 0)[:, None], p.rect, 0)
    return np.any(a != b, axis=1)


def splat_array(p: oracle.Projection) -> np.ndarray:
    s = np.zeros((p.n, 12), np.float32)
    s[:, 0:2] = p.mean2d
    s[:, 2:5] = p.conic
    s[:, 5] = p.opacity
    s[:, 6:9] = p.color
    s[:, 9] = p.depth
    return s


def grad_rel_err(gpu, orc):
    gpu = np.asarray(gpu, np.float64)
    orc = np.asarray(orc, np.float64)
    if orc.size == 0:
        return 0.0
    floor = GRAD_FLOOR * max(np.abs(orc).max(), 1e-30)
    return float((np.abs(gpu - orc) / np.maximum(np.abs(orc), floor)).max())


SUM_FLOOR = 3e-3


def sum_rel_err(gpu, orc, abs_sum):
    """Relative error of a float32 sum: |gpu - oracle| / max(|oracle|, 3e-3 * sum|terms|).
    Where the terms cancel (|oracle| much smaller than sum|terms|) float32 arithmetic can only
    resolve the result to some ulps of sum|terms|; the floor grants 3e-6 of it (about 25 ulps)
    at the 1e-3 tolerance, and nothing more."""
    gpu = np.asarray(gpu, np.float64)
    orc = np.asarray(orc, np.float64)
    den = np.maximum(np.abs(orc), SUM_FLOOR * np.asarray(abs_sum, np.float64))
    den = np.maximum(den, 1e-30)
    return float((np.abs(gpu - orc) / den).max()) if orc.size else 0.0


def assert_grad_close(gpu, orc, name, rtol=GRAD_RTOL):
    err = grad_rel_err(gpu, orc)
    record("grad rel " + name, err)
    assert err <= rtol, f"{name}: relative error {err:.3e} > {rtol}"
    return err


def oracle_grad2d_array(g2d: oracle.Grad2D) -> np.ndarray:
    a = np.zeros((g2d.mean2d.shape[0], 12))
    a[:, 0:2] = g2d.mean2d
    a[:, 2:5] = g2d.conic
    a[:, 5] = g2d.opacity
    a[:, 6:9] = g2d.color
    return a
