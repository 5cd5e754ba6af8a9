"""FP64 CPU oracle of the differentiable tile rasterizer (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package. It wraps ``lobe_oracle.c`` (plain C, double precision, compiled
with ``-ffp-contract=off``) through ctypes and shares no code with the CUDA library.

Every function takes float64 numpy arrays (float32 inputs are widened exactly) and
returns float64 / int32 arrays. One call handles one (Gaussian set, camera) item; a
batch of items is a Python loop over items.

Parity-unpinned parts: none of the functions below is unpinned; the pins live in
``tests/test_oracle_*.py`` (closed forms, library routines, invariants, brute force and
central finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lobe_oracle.c")
_LIB = os.path.join(_HERE, "liblobe_oracle.so")

# margin order: rel (alpha/T/clamp), px (rect edges), rad (3 sqrt(lambda) near integer),
# col (colour clamp), sig (sigma near 0), guard (fov guard, relative)
MARGINS_NONE = np.zeros(6)
# same float32 inputs on both sides: only the renderer's float32 arithmetic differs
MARGINS_STAGE = np.array([2e-5, 1e-4, 2e-6, 1e-6, 1e-5, 1e-6])
# end to end: the GPU's float32 projection feeds its renderer
MARGINS_E2E = np.array([5e-4, 2e-3, 2e-5, 2e-5, 1e-4, 2e-5])

F_GUARD, F_RADIUS, F_RECT, F_COLOR, F_GUARD_OUT = 1, 2, 4, 8, 16


def marginal_visibility(p: "Projection") -> np.ndarray:
    """Gaussians whose culling decision float32 may take the other way: a marginal fov-guard
    decision, or (not culled by the guard) a marginal radius / rectangle edge, which may make
    the tile rectangle empty or not at the image border."""
    g = (p.flags & F_GUARD) != 0
    r = ((p.flags & (F_RADIUS | F_RECT)) != 0) & ((p.flags & F_GUARD_OUT) == 0)
    return (g | r) & (p.radius_all > 0)


def marginal_rect(p: "Projection") -> np.ndarray:
    """Gaussians whose tile rectangle a marginal decision may change (as orc_bin_ext reads it)."""
    m = (p.flags & F_GUARD) != 0
    m |= ((p.flags & (F_RADIUS | F_RECT)) != 0) & ((p.flags & F_GUARD_OUT) == 0)
    return m & (p.radius_all > 0)


def build(force: bool = False) -> str:
    """Compile lobe_oracle.c into liblobe_oracle.so (gcc, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        # compile to a private file and rename it into place, so that processes building at
        # the same time (spawned test ranks) never load a half-written library
        tmp = f"{_LIB}.{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.orc_bin.restype = ctypes.c_int64
        _lib.orc_depth_key.restype = ctypes.c_uint32
        _lib.orc_depth_key.argtypes = [ctypes.c_double]
        _lib.orc_round_f32.restype = ctypes.c_float
        _lib.orc_round_f32.argtypes = [ctypes.c_double]
        _lib.orc_bin_ext.restype = ctypes.c_int64
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _u8(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def cam_vector(cam) -> np.ndarray:
    """[viewmat(16), fx, fy, cx, cy, width, height, near, far] as float64 (from float32 values)."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    v = np.empty(24)
    v[:16] = np.asarray(c["viewmat"], np.float32).astype(np.float64).reshape(16)
    v[16:20] = np.float32([c["fx"], c["fy"], c["cx"], c["cy"]]).astype(np.float64)
    v[20], v[21] = c["width"], c["height"]
    v[22], v[23] = np.float32(c["near"]), np.float32(c["far"])
    return v


@dataclass
class Projection:
    mean2d: np.ndarray
    conic: np.ndarray
    color: np.ndarray
    opacity: np.ndarray
    depth: np.ndarray
    radius: np.ndarray
    rect: np.ndarray
    flags: np.ndarray
    radius_all: np.ndarray
    color_raw: np.ndarray | None = None  # [n,3] SH colour + 0.5 before the clamp at 0

    @property
    def n(self):
        return self.radius.shape[0]

    def rounded(self) -> "Projection":
        """The same projection with every float rounded to float32 (what a float32 stage sees)."""
        r = lambda a: a.astype(np.float32).astype(np.float64)
        return Projection(r(self.mean2d), r(self.conic), r(self.color), r(self.opacity),
                          self.depth.copy(), self.radius.copy(), self.rect.copy(), self.flags.copy(),
                          self.radius_all.copy(), None if self.color_raw is None else self.color_raw.copy())


def project(g, cam, tile=(16, 16), sh_degree=3, crop=None, margins=MARGINS_NONE) -> Projection:
    L = lib()
    n = g["means"].shape[0]
    means, pm = _d(g["means"])
    ls, pls = _d(g["log_scales"])
    q, pq = _d(g["quats"])
    lo, plo = _d(g["opacity_logits"])
    sh, psh = _d(g["sh"])
    cr, pcr = _u8(crop)
    cv, pcv = _d(cam_vector(cam))
    mg, pmg = _d(margins)
    out = Projection(np.zeros((n, 2)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n), np.zeros(n),
                     np.zeros(n, np.int32), np.zeros((n, 4), np.int32), np.zeros(n, np.int32),
                     np.zeros(n, np.int32), np.zeros((n, 3)))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    L.orc_project(ctypes.c_int64(n), pm, pls, pq, plo, psh, ctypes.c_int(sh_degree), pcr, pcv,
                  ctypes.c_int(tile[0]), ctypes.c_int(tile[1]), pmg,
                  ptr(out.mean2d), ptr(out.conic), ptr(out.color), ptr(out.opacity), ptr(out.depth),
                  ptr(out.radius), ptr(out.rect), ptr(out.flags), ptr(out.radius_all), ptr(out.color_raw))
    return out


def grid(cam, tile):
    c = cam if isinstance(cam, dict) else cam.as_dict()
    return (c["width"] + tile[0] - 1) // tile[0], (c["height"] + tile[1] - 1) // tile[1]


def bin_sort(p: Projection, cam, tile=(16, 16)):
    """(ids, tile_start): Gaussian index of every pair in (tile, depth, index) order, and the
    first pair of every tile (n_tiles + 1 entries)."""
    L = lib()
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    m2, pm2 = _d(p.mean2d)
    rad, pr = _i(p.radius)
    dep, pd = _d(p.depth)
    total = L.orc_bin(ctypes.c_int64(p.n), pm2, pr, pd, W, H, tile[0], tile[1], None, None)
    gx, gy = grid(c, tile)
    ids = np.zeros(max(total, 1), np.int32)
    ts = np.zeros(gx * gy + 1, np.int32)
    L.orc_bin(ctypes.c_int64(p.n), pm2, pr, pd, W, H, tile[0], tile[1],
              ids.ctypes.data_as(ctypes.c_void_p), ts.ctypes.data_as(ctypes.c_void_p))
    return ids[:total], ts


def flag_pixels(p: Projection, cam, tile=(16, 16)) -> np.ndarray:
    """int32 [H*W]: pixels a marginal Gaussian decision could change."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    pxf = np.zeros(W * H, np.int32)
    fl, pfl = _i(p.flags)
    m2, pm2 = _d(p.mean2d)
    r, pr = _i(p.radius)
    ra, pra = _i(p.radius_all)
    lib().orc_flag_marginal_gaussians(ctypes.c_int64(p.n), pfl, pm2, pr, pra, W, H, tile[0], tile[1],
                                      pxf.ctypes.data_as(ctypes.c_void_p))
    return pxf


@dataclass
class Image:
    rgb: np.ndarray       # [3,H,W]
    T_final: np.ndarray   # [H,W]
    n_contrib: np.ndarray  # [H,W] int32
    flags: np.ndarray     # [H,W] int32, 1 = some decision on this pixel is marginal
    wsum: np.ndarray      # [H,W] sum_i alpha_i T_i


def render_fwd(p: Projection, ids, tile_start, cam, tile=(16, 16), bg=(0.0, 0.0, 0.0),
               margins=MARGINS_NONE, pixel_flags=None) -> Image:
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    rgb = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    fl = np.zeros((H, W), np.int32) if pixel_flags is None else \
        np.ascontiguousarray(pixel_flags, np.int32).reshape(H, W).copy()
    ws = np.zeros((H, W))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m2, _ = _d(p.mean2d)
    cn, _ = _d(p.conic)
    co, _ = _d(p.color)
    op, _ = _d(p.opacity)
    ids_, _ = _i(ids if len(ids) else np.zeros(1, np.int32))
    ts, _ = _i(tile_start)
    bgv, _ = _d(np.asarray(bg, np.float64))
    mg, _ = _d(margins)
    lib().orc_render_fwd(W, H, tile[0], tile[1], ptr(m2), ptr(cn), ptr(co), ptr(op), ptr(ids_), ptr(ts),
                         ptr(bgv), ptr(mg), ptr(rgb), ptr(T), ptr(nc), ptr(fl), ptr(ws))
    return Image(rgb, T, nc, fl, ws)


def render_untiled(p: Projection, cam, tile=(16, 16), respect_rect=True, bg=(0.0, 0.0, 0.0),
                   margins=MARGINS_NONE):
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    rgb = np.zeros((3, H, W))
    T = np.zeros((H, W))
    fl = np.zeros((H, W), np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m2, _ = _d(p.mean2d)
    cn, _ = _d(p.conic)
    co, _ = _d(p.color)
    op, _ = _d(p.opacity)
    r, _ = _i(p.radius)
    dp, _ = _d(p.depth)
    bgv, _ = _d(np.asarray(bg, np.float64))
    mg, _ = _d(margins)
    lib().orc_render_untiled(ctypes.c_int64(p.n), W, H, tile[0], tile[1], ptr(m2), ptr(cn), ptr(co),
                             ptr(op), ptr(r), ptr(dp), int(respect_rect), ptr(bgv), ptr(mg), ptr(rgb),
                             ptr(T), ptr(fl))
    return rgb, T, fl


@dataclass
class Grad2D:
    mean2d: np.ndarray
    conic: np.ndarray
    color: np.ndarray
    opacity: np.ndarray


def render_bwd(p: Projection, ids, tile_start, cam, dL_drgb, tile=(16, 16), bg=(0.0, 0.0, 0.0)) -> Grad2D:
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    n = p.n
    out = Grad2D(np.zeros((n, 2)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m2, _ = _d(p.mean2d)
    cn, _ = _d(p.conic)
    co, _ = _d(p.color)
    op, _ = _d(p.opacity)
    ids_, _ = _i(ids if len(ids) else np.zeros(1, np.int32))
    ts, _ = _i(tile_start)
    bgv, _ = _d(np.asarray(bg, np.float64))
    gr, _ = _d(np.asarray(dL_drgb).reshape(3, H, W))
    lib().orc_render_bwd(W, H, tile[0], tile[1], ptr(m2), ptr(cn), ptr(co), ptr(op), ptr(ids_), ptr(ts),
                         ptr(bgv), ptr(gr), ptr(out.mean2d), ptr(out.conic), ptr(out.color),
                         ptr(out.opacity))
    return out


@dataclass
class ParamGrads:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sd_acc: np.ndarray
    sd_cnt: np.ndarray


def zero_param_grads(n) -> ParamGrads:
    return ParamGrads(np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n),
                      np.zeros((n, 16, 3)), np.zeros(n), np.zeros(n, np.int32))


def project_bwd(g, cam, g2d: Grad2D, tile=(16, 16), sh_degree=3, crop=None, aabb=None,
                out: ParamGrads | None = None) -> ParamGrads:
    L = lib()
    n = g["means"].shape[0]
    out = zero_param_grads(n) if out is None else out
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    means, _ = _d(g["means"])
    ls, _ = _d(g["log_scales"])
    q, _ = _d(g["quats"])
    lo, _ = _d(g["opacity_logits"])
    sh, _ = _d(g["sh"])
    cr, pcr = _u8(crop)
    cv, _ = _d(cam_vector(cam))
    if aabb is None:
        box = np.array([-np.inf, -np.inf, -np.inf, np.inf, np.inf, np.inf])
    else:
        box = np.array(list(aabb.lo) + list(aabb.hi), np.float64)
    box = box.astype(np.float32).astype(np.float64)
    dm, _ = _d(g2d.mean2d)
    dc, _ = _d(g2d.conic)
    dcol, _ = _d(g2d.color)
    dop, _ = _d(g2d.opacity)
    L.orc_project_bwd(ctypes.c_int64(n), ptr(means), ptr(ls), ptr(q), ptr(lo), ptr(sh), sh_degree, pcr,
                      ptr(cv), tile[0], tile[1], ptr(box), ptr(dm), ptr(dc), ptr(dcol), ptr(dop),
                      ptr(out.means), ptr(out.log_scales), ptr(out.quats), ptr(out.opacity_logits),
                      ptr(out.sh), ptr(out.sd_acc), ptr(out.sd_cnt))
    return out


def visibility_crop(g, cams, tile=(16, 16), sh_degree=3) -> np.ndarray:
    """uint8 mask: 1 where the Gaussian is visible from at least one of ``cams`` (Sec. 3.3)."""
    L = lib()
    n = g["means"].shape[0]
    mask = np.zeros(n, np.uint8)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    means, _ = _d(g["means"])
    ls, _ = _d(g["log_scales"])
    q, _ = _d(g["quats"])
    lo, _ = _d(g["opacity_logits"])
    sh, _ = _d(g["sh"])
    for cam in cams:
        cv, _ = _d(cam_vector(cam))
        L.orc_visibility_crop(ctypes.c_int64(n), ptr(means), ptr(ls), ptr(q), ptr(lo), ptr(sh), sh_degree,
                              ptr(cv), tile[0], tile[1], ptr(mask))
    return mask


def render_depth(p: Projection, ids, tile_start, cam, tile=(16, 16), margins=MARGINS_NONE,
                 pixel_flags=None) -> Image:
    """Composite depth of fast camera selection (Sec. 3.2): D = sum_i d_i alpha_i T_i, the
    blending equation with each Gaussian's camera-space depth d_i in place of its colour.
    Returned as an Image whose rgb[0] (= rgb[1] = rgb[2]) is D, with the background 0."""
    q = Projection(p.mean2d, p.conic, np.repeat(p.depth[:, None], 3, axis=1), p.opacity, p.depth, p.radius,
                   p.rect, p.flags, p.radius_all)
    return render_fwd(q, ids, tile_start, cam, tile, (0.0, 0.0, 0.0), margins, pixel_flags)


def backproject(D, T, cam, normalize=False):
    """World points of the pixels some Gaussian reached (T < 1), from the depth map D (divided
    by the accumulated opacity 1 - T when normalize): camera-space (x, y, z) =
    ((px + 0.5 - cx) D / fx, (py + 0.5 - cy) D / fy, D), world = the inverse of the
    world->camera viewmat applied to it (R^T (p_c - t) for an orthonormal R). Returns
    (points [H, W, 3], mask [H, W])."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    H, W = D.shape
    mask = T < 1.0
    d = D / np.where(mask, 1.0 - T, 1.0) if normalize else D
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    pc = np.stack([(px + 0.5 - c["cx"]) / c["fx"] * d, (py + 0.5 - c["cy"]) / c["fy"] * d, d], axis=-1)
    Vinv = np.linalg.inv(np.asarray(c["viewmat"], np.float64).reshape(4, 4))
    return pc @ Vinv[:3, :3].T + Vinv[:3, 3], mask


def fcs_coverage(D, T, cam, blocks, normalize=False, rel_margin=0.0):
    """Fast camera selection counts (Sec. 3.2): per block box, the number of back-projected
    points inside it (lo <= p < hi per axis), and the number of points N_p. With rel_margin >
    0 also returns a per-pixel flag for points within rel_margin * (|coordinate| + 1) of a face
    of some box (a float32 evaluation may put them on either side)."""
    pts, mask = backproject(D, T, cam, normalize)
    counts, flags = [], np.zeros(mask.shape, bool)
    for b in blocks:
        lo, hi = np.asarray(b.lo, np.float64), np.asarray(b.hi, np.float64)
        inside = mask & np.all((pts >= lo) & (pts < hi), axis=-1)
        counts.append(int(inside.sum()))
        if rel_margin > 0:
            tol = rel_margin * (np.abs(pts) + 1.0)
            near = np.isfinite(lo) & (np.abs(pts - lo) < tol) | np.isfinite(hi) & (np.abs(pts - hi) < tol)
            flags |= mask & np.any(near, axis=-1)
    return np.array(counts, np.int64), int(mask.sum()), flags


def densify(params, acc, cnt, normals, grad_threshold, max_clone_log_scale, prune_logit, n_split,
            split_log_shrink):
    """Selective densification (Sec. 3.3) with the adaptive density control of the 3DGS
    procedure (appendix "3DGS Training"). Per Gaussian: pruned when its opacity logit is below
    prune_logit; else, when it has SD views (cnt > 0, so its mean was inside the block) and
    its mean gradient acc / cnt reaches grad_threshold, cloned (an exact copy follows it) if
    its largest log-scale is at most max_clone_log_scale, split otherwise into n_split
    children with means mu + R(q) (exp(log_s) * z_k) (z_k = normals[g, k]) and log-scales
    log_s - split_log_shrink; else kept. Outputs follow their sources' order. The decisions
    are taken in float32, the precision of the statistic and the parameters; the children's
    geometry in FP64. Returns (dict of float64 arrays, source index per output)."""
    f32 = np.float32
    ls = np.asarray(params["log_scales"], f32)
    lg = np.asarray(params["opacity_logits"], f32)
    acc32 = np.asarray(acc, f32)
    cnt = np.asarray(cnt, np.int64)
    n = lg.shape[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        mean_grad = np.where(cnt > 0, acc32 / np.maximum(cnt, 1).astype(f32), f32(0))
    prune = lg < f32(prune_logit)
    dens = ~prune & (cnt > 0) & (mean_grad >= f32(grad_threshold))
    clone = dens & (ls.max(axis=1) <= f32(max_clone_log_scale))
    split = dens & ~clone
    k_out = np.where(prune, 0, np.where(clone, 2, np.where(split, n_split, 1)))
    source = np.repeat(np.arange(n), k_out)
    first = np.concatenate([[0], np.cumsum(k_out)[:-1]])
    k = np.arange(source.shape[0]) - first[source]
    out = {key: np.asarray(params[key], np.float64)[source].copy() for key in
           ("means", "log_scales", "quats", "opacity_logits", "sh")}
    child = split[source]
    if child.any():
        g = source[child]
        q = np.asarray(params["quats"], np.float64)[g]
        q = q / np.linalg.norm(q, axis=1, keepdims=True)
        r, x, y, z = q.T
        R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - r * z), 2 * (x * z + r * y),
                      2 * (x * y + r * z), 1 - 2 * (x * x + z * z), 2 * (y * z - r * x),
                      2 * (x * z - r * y), 2 * (y * z + r * x), 1 - 2 * (x * x + y * y)], axis=1).reshape(-1, 3, 3)
        s = np.exp(np.asarray(params["log_scales"], np.float64)[g])
        zk = np.asarray(normals, np.float64)[g, k[child]]
        out["means"][child] = np.asarray(params["means"], np.float64)[g] + np.einsum("nij,nj->ni", R, s * zk)
        out["log_scales"][child] = np.asarray(params["log_scales"], np.float64)[g] - split_log_shrink
    return out, source


# ----------------------------------------------------------------------------- admissible branches

MAX_LEAVES = 64  # leaves per pixel an enumeration keeps (a uint64 bitmask names the admissible ones)


@dataclass
class ExtBins:
    """Per-tile lists with every possible member: ``unc[k]`` is 0 for a certain member, 1 for
    a member only if a marginal projection decision went the other way, 2 for a member that
    such a flip would remove."""
    ids: np.ndarray
    unc: np.ndarray
    tile_start: np.ndarray


def bin_ext(p: Projection, cam, tile=(16, 16), win=None) -> ExtBins:
    """Extended per-tile lists of the tiles touching ``win`` = (x0, y0, x1, y1) (None: the
    sampling window(s) in effect, by default the whole image):
    the certain members as ``bin_sort`` lists them, plus the Gaussians whose membership a
    marginal radius, rectangle or guard decision (``p.flags``) could flip."""
    L = lib()
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    m2, _ = _d(p.mean2d)
    r, _ = _i(p.radius)
    ra, _ = _i(p.radius_all)
    fl, _ = _i(p.flags)
    dp, _ = _d(p.depth)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    gx, gy = grid(c, tile)
    ctx = window(*win) if win is not None else _NoWindowChange()
    with ctx:
        total = L.orc_bin_ext(ctypes.c_int64(p.n), ptr(m2), ptr(r), ptr(ra), ptr(fl), ptr(dp), W, H, tile[0],
                              tile[1], None, None, None)
        ids = np.zeros(max(total, 1), np.int32)
        unc = np.zeros(max(total, 1), np.uint8)
        ts = np.zeros(gx * gy + 1, np.int32)
        L.orc_bin_ext(ctypes.c_int64(p.n), ptr(m2), ptr(r), ptr(ra), ptr(fl), ptr(dp), W, H, tile[0], tile[1],
                      ptr(ids), ptr(unc), ptr(ts))
    return ExtBins(ids[:total], unc[:total], ts)


class _NoWindowChange:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


@dataclass
class Leaves:
    """Every admissible composite of each pixel of a window (see ``render_leaves``)."""
    win: tuple            # (x0, y0, x1, y1)
    n: np.ndarray         # [h, w] leaves per pixel; 0 = more than the cap (pixel not checkable)
    C: np.ndarray         # [h, w, L, 3] colour, background included
    T: np.ndarray         # [h, w, L] final transmittance
    nc: np.ndarray        # [h, w, L] n_contrib


def _win(cam, win):
    c = cam if isinstance(cam, dict) else cam.as_dict()
    if win is None:
        return (0, 0, c["width"], c["height"])
    x0, y0, x1, y1 = win
    return (x0, y0, min(x1, c["width"]), min(y1, c["height"]))


def render_leaves(p: Projection, eb: ExtBins, cam, tile=(16, 16), bg=(0.0, 0.0, 0.0), margins=MARGINS_NONE,
                  win=None, max_leaves=MAX_LEAVES, certain=False) -> Leaves:
    """Enumerates, per pixel of ``win``, every composite reachable by flipping decisions that
    are marginal under ``margins`` (membership of uncertain list members, sigma < 0, the 1/255
    skip, the 0.99 clamp, the 1e-4 stop), depth first with the FP64 outcome first: leaf 0 is
    the FP64 composite. ``certain`` treats every list member as certain (stage inputs)."""
    if not 1 <= max_leaves <= 64:
        raise ValueError("max_leaves must be in [1, 64]")
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    x0, y0, x1, y1 = _win(c, win)
    h, w = y1 - y0, x1 - x0
    n = np.zeros((h, w), np.int32)
    C = np.zeros((h, w, max_leaves, 3))
    T = np.zeros((h, w, max_leaves))
    nc = np.zeros((h, w, max_leaves), np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m2, _ = _d(p.mean2d)
    cn, _ = _d(p.conic)
    co, _ = _d(p.color)
    op, _ = _d(p.opacity)
    ids, _ = _i(eb.ids if len(eb.ids) else np.zeros(1, np.int32))
    unc = np.ascontiguousarray(eb.unc if len(eb.unc) else np.zeros(1, np.uint8), np.uint8)
    ts, _ = _i(eb.tile_start)
    bgv, _ = _d(np.asarray(bg, np.float64))
    mg, _ = _d(margins)
    lib().orc_render_leaves(W, H, tile[0], tile[1], ptr(m2), ptr(cn), ptr(co), ptr(op), ptr(ids),
                            None if certain else ptr(unc), ptr(ts), ptr(bgv), ptr(mg), x0, y0, x1, y1,
                            max_leaves, ptr(n), ptr(C), ptr(T), ptr(nc))
    return Leaves((x0, y0, x1, y1), n, C, T, nc)


def render_bwd_envelope(p: Projection, eb: ExtBins, cam, dL_drgb, admissible, tile=(16, 16), bg=(0.0, 0.0, 0.0),
                        margins=MARGINS_NONE, win=None, max_leaves=MAX_LEAVES, certain=False):
    """Bounds of the composite adjoint when each pixel of ``win`` may have taken any of its
    ``admissible`` leaves (uint64 [h, w], bit l = leaf l of ``render_leaves`` with the same
    arguments): (lo, hi, absmax), each [n, 12] in the grad2d layout (u, v, conic a, b, c,
    opacity, r, g, b, 0, 0, 0). Any one choice of an admissible leaf per pixel gives per-splat
    gradients inside [lo, hi]; with one admissible leaf per pixel lo = hi = the plain
    adjoint. absmax sums, per pixel, the largest absolute per-pixel term over the admissible
    leaves (the scale a float32 sum of the terms resolves to)."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    W, H = c["width"], c["height"]
    x0, y0, x1, y1 = _win(c, win)
    adm = np.ascontiguousarray(admissible, np.uint64).reshape(y1 - y0, x1 - x0)
    lo = np.zeros((p.n, 12))
    hi = np.zeros((p.n, 12))
    ab = np.zeros((p.n, 12))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    m2, _ = _d(p.mean2d)
    cn, _ = _d(p.conic)
    co, _ = _d(p.color)
    op, _ = _d(p.opacity)
    ids, _ = _i(eb.ids if len(eb.ids) else np.zeros(1, np.int32))
    unc = np.ascontiguousarray(eb.unc if len(eb.unc) else np.zeros(1, np.uint8), np.uint8)
    ts, _ = _i(eb.tile_start)
    bgv, _ = _d(np.asarray(bg, np.float64))
    mg, _ = _d(margins)
    gr, _ = _d(np.asarray(dL_drgb).reshape(3, H, W))
    lib().orc_render_bwd_envelope(W, H, tile[0], tile[1], ptr(m2), ptr(cn), ptr(co), ptr(op), ptr(ids),
                                  None if certain else ptr(unc), ptr(ts), ptr(bgv), ptr(mg), x0, y0, x1, y1,
                                  max_leaves, ptr(adm), ptr(gr), ptr(lo), ptr(hi), ptr(ab))
    return lo, hi, ab


class branch_flips:
    """Context manager: while active, ``project_bwd`` inverts the culling decision of every
    Gaussian with ``vis[g] != 0`` and the colour clamp of channel ch where bit ch of
    ``color[g]`` is set (the other outcome of a decision float32 could take either way)."""

    def __init__(self, vis=None, color=None):
        self.vis = None if vis is None else np.ascontiguousarray(vis, np.uint8)
        self.color = None if color is None else np.ascontiguousarray(color, np.uint8)

    def __enter__(self):
        ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        lib().orc_set_branch_flips(ptr(self.vis), ptr(self.color))
        return self

    def __exit__(self, *exc):
        lib().orc_set_branch_flips(None, None)


def sh_basis(dirs, degree=3):
    """Real SH basis [n,16] and its derivative [n,16,3] for each row of ``dirs``."""
    L = lib()
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    Y = np.zeros((dirs.shape[0], 16))
    dY = np.zeros((dirs.shape[0], 16, 3))
    for i in range(dirs.shape[0]):
        L.orc_sh_basis(degree, dirs[i].ctypes.data_as(ctypes.c_void_p),
                       Y[i].ctypes.data_as(ctypes.c_void_p), dY[i].ctypes.data_as(ctypes.c_void_p))
    return Y, dY


class abs_sums:
    """Context manager: while active, render_bwd also accumulates, per Gaussian, the sum of
    the absolute values of the per-pixel terms of each 2D gradient into ``self.a``
    ([n,12], grad2d layout: u, v, conic a, b, c, opacity, r, g, b)."""

    def __init__(self, n):
        self.a = np.zeros((n, 12))

    def __enter__(self):
        lib().orc_set_abs_out(self.a.ctypes.data_as(ctypes.c_void_p))
        return self

    def __exit__(self, *exc):
        lib().orc_set_abs_out(None)


class window:
    """Context manager restricting bin/render/render_bwd to the pixel window [x0,x1) x [y0,y1)
    (a bounded sample of a large image for timing; per-pixel work is unchanged)."""

    def __init__(self, x0, y0, x1, y1):
        self.w = (int(x0), int(y0), int(x1), int(y1))

    def __enter__(self):
        lib().orc_set_window(*self.w)
        return self

    def __exit__(self, *exc):
        lib().orc_set_window(0, 0, 1 << 30, 1 << 30)


class windows:
    """Context manager restricting bin/render/render_bwd (and bin_ext) to the union of several
    pixel windows [(x0, y0, x1, y1), ...] (at most 64): tiles touching any of them, pixels
    inside any of them. Changes no arithmetic."""

    def __init__(self, rects):
        self.r = np.ascontiguousarray(np.asarray(rects, np.int32).reshape(-1, 4))
        if not 1 <= len(self.r) <= 64:
            raise ValueError("1 to 64 windows")

    def __enter__(self):
        lib().orc_set_windows(len(self.r), self.r.ctypes.data_as(ctypes.c_void_p))
        return self

    def __exit__(self, *exc):
        lib().orc_set_window(0, 0, 1 << 30, 1 << 30)


def depth_key(z: float) -> int:
    return int(lib().orc_depth_key(float(z)))


# ----------------------------------------------------------------------------- pipelines

@dataclass
class Forward:
    proj: Projection
    ids: np.ndarray
    tile_start: np.ndarray
    image: Image
    pixel_flags: np.ndarray  # [H,W] int32: union of pixel and Gaussian marginal flags


def forward(g, cam, tile=(16, 16), sh_degree=3, crop=None, bg=(0.0, 0.0, 0.0), margins=MARGINS_NONE,
            proj: Projection | None = None) -> Forward:
    """Full forward of one item: project -> bin/sort -> composite."""
    p = project(g, cam, tile, sh_degree, crop, margins) if proj is None else proj
    ids, ts = bin_sort(p, cam, tile)
    pxf = flag_pixels(p, cam, tile)
    img = render_fwd(p, ids, ts, cam, tile, bg, margins, pxf)
    return Forward(p, ids, ts, img, img.flags)


def backward(g, cam, fwd: Forward, dL_drgb, tile=(16, 16), sh_degree=3, crop=None, aabb=None,
             bg=(0.0, 0.0, 0.0)):
    g2d = render_bwd(fwd.proj, fwd.ids, fwd.tile_start, cam, dL_drgb, tile, bg)
    pg = project_bwd(g, cam, g2d, tile, sh_degree, crop, aabb)
    return g2d, pg


def set_dict(gs) -> dict:
    """Widen a scenes.GaussianSet (or dict of float32 arrays) to float64 arrays."""
    if hasattr(gs, "arrays"):
        gs = gs.arrays()
    return {k: np.asarray(v, np.float64) for k, v in gs.items()}


# ----------------------------------------------------------------------------- Adam

ADAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def adam(params, grads, exp_avg, exp_avg_sq, step, lr, beta1=0.9, beta2=0.999, eps=1e-15, rows=None):
    """One Adam update (Kingma and Ba, Algorithm 1) of a Gaussian set, the optimizer of the
    3DGS procedure the fine-training follows (appendix "3DGS Training"). With g the gradient
    and t = step (>= 1, the index of this update), per element:
        m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
        p <- p - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
    lr is a dict of per-group rates: means, log_scales, quats, opacity_logits, sh_dc (the
    degree-0 coefficients sh[:, 0, :]) and sh_rest (sh[:, 1:, :]). With ``rows`` (bool [n])
    only those Gaussians change, parameters and moments alike (the sparse variant of coarse
    training, appendix "3DGS Training"); without, every Gaussian does (standard Adam, a zero
    gradient still decays the moments and moves the parameter). All dicts map ADAM_KEYS to
    arrays of the set's shapes. Returns new float64 dicts (params, exp_avg, exp_avg_sq)."""
    t = int(step)
    if t < 1:
        raise ValueError("step must be >= 1")
    bc1 = 1.0 - beta1 ** t
    bc2 = 1.0 - beta2 ** t
    out_p, out_m, out_v = {}, {}, {}
    for key in ADAM_KEYS:
        p = np.asarray(params[key], np.float64)
        g = np.asarray(grads[key], np.float64)
        m = beta1 * np.asarray(exp_avg[key], np.float64) + (1.0 - beta1) * g
        v = beta2 * np.asarray(exp_avg_sq[key], np.float64) + (1.0 - beta2) * g * g
        if key == "sh":
            rate = np.full(p.shape[1:], float(lr["sh_rest"]))
            rate[0, :] = float(lr["sh_dc"])
        else:
            rate = float(lr[key])
        p_new = p - rate * (m / bc1) / (np.sqrt(v / bc2) + eps)
        if rows is not None:
            keep = ~np.asarray(rows, bool).reshape((-1,) + (1,) * (p.ndim - 1))
            p_new = np.where(keep, p, p_new)
            m = np.where(keep, np.asarray(exp_avg[key], np.float64), m)
            v = np.where(keep, np.asarray(exp_avg_sq[key], np.float64), v)
        out_p[key], out_m[key], out_v[key] = p_new, m, v
    return out_p, out_m, out_v


# ----------------------------------------------------------------------------- KD partition

def kd_partition(centers, root, n_blocks, cams_points, tau=0.1, q_lo=0.1, q_hi=0.9, steps=3):
    """Load-balanced KD-tree partition with cutline refinement (Alg. 1, Sec. 3.1), written as
    plain loops. ``centers`` [N, 3] are the coarse Gaussian centres, ``root`` the scene box,
    ``cams_points`` one entry per camera: the world points back-projected from its depth map
    (fast camera selection, Sec. 3.2). A box's camera set holds the cameras of its parent with
    V = (points inside the box) / (all the camera's points) >= tau; its workload is the set's
    size. The leaf with the largest workload (earliest created among equals) is split along
    the longer of its x / y extents (of the centres inside it) at a percentile q of those
    centres' coordinates, starting at the median and moved by bisection toward the lighter
    side for ``steps`` rounds inside [q_lo, q_hi]; the children of the last evaluated cut are
    kept. Boxes are half-open: lo <= p < hi. Returns [(lo, hi, camera index list)] in
    creation order of the leaves."""
    centers = np.asarray(centers, np.float64)

    def inside(pts, lo, hi):
        return np.all((pts >= lo) & (pts < hi), axis=-1)

    def cams_of(lo, hi, parent_cams):
        out = []
        for c in parent_cams:
            pts = cams_points[c]
            if len(pts) and inside(pts, lo, hi).sum() / len(pts) >= tau:
                out.append(c)
        return out

    lo0 = np.array(root.lo, np.float64)
    hi0 = np.array(root.hi, np.float64)
    leaves = [(lo0, hi0, cams_of(lo0, hi0, list(range(len(cams_points)))), 0)]
    serial = 1
    while len(leaves) < n_blocks:
        best = 0
        for i in range(1, len(leaves)):
            if len(leaves[i][2]) > len(leaves[best][2]) or \
                    (len(leaves[i][2]) == len(leaves[best][2]) and leaves[i][3] < leaves[best][3]):
                best = i
        lo, hi, cams, _ = leaves.pop(best)
        pts = centers[inside(centers, lo, hi)]
        ext = [pts[:, d].max() - pts[:, d].min() if len(pts) else 0.0 for d in (0, 1)]
        a = 0 if ext[0] >= ext[1] else 1
        coords = np.sort(pts[:, a])
        qlo, qhi, q = q_lo, q_hi, 0.5
        for _ in range(steps):
            cut = float(np.quantile(coords, q)) if len(coords) else 0.5 * (lo[a] + hi[a])
            hl, lr = hi.copy(), lo.copy()
            hl[a] = cut
            lr[a] = cut
            cl, cr = cams_of(lo, hl, cams), cams_of(lr, hi, cams)
            if len(cl) > len(cr):
                qhi, q = q, 0.5 * (qlo + q)
            elif len(cr) > len(cl):
                qlo, q = q, 0.5 * (qhi + q)
            else:
                break
        leaves.append((lo, hl, cl, serial))
        leaves.append((lr, hi, cr, serial + 1))
        serial += 2
    return [(lo, hi, cams) for lo, hi, cams, _ in leaves]
