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


# ----------------------------------------------------------------------------- admissible branches
#
# Where float32 can take a decision either way (alpha at 1/255, T at 1e-4, the 0.99 clamp,
# sigma < 0, a radius or tile-rectangle edge, the fov guard, the colour clamp), the oracle
# enumerates every outcome (oracle.render_leaves): a GPU pixel passes when it matches one of
# its pixel's leaves within the parity bar, and the gradients must lie within the envelope of
# the adjoints of the leaves the GPU's own forward matched (oracle.render_bwd_envelope). Only
# pixels with more admissible outcomes than the enumeration keeps stay unchecked; their share
# is bounded by EXCLUDED_MAX and printed with the other counts.

EXCLUDED_MAX = 1e-4
PARITY: dict = {}  # check name -> summed pixel counts


def _add_parity(name, stats):
    agg = PARITY.setdefault(name, {})
    for k, v in stats.items():
        agg[k] = agg.get(k, 0) + v


def match_image(lv: oracle.Leaves, rgb, T, nc=None, name="image", atol=IMG_ATOL, t_atol=IMG_ATOL):
    """Matches a window of the GPU's image (rgb [3,h,w], T_final [h,w], n_contrib [h,w] or None)
    against the oracle's leaves of the same window. Every checkable pixel must match a leaf
    (colour and T within atol, n_contrib equal when given). Returns the admissible-leaf masks
    (uint64 [h,w], bit l = leaf l matched) for the backward envelope."""
    rgb = np.asarray(rgb, np.float64)
    T = np.asarray(T, np.float64)
    h, w = lv.n.shape
    L = lv.C.shape[2]
    lidx = np.arange(L)
    valid = lidx[None, None, :] < lv.n[:, :, None]
    d = np.abs(lv.C - np.transpose(rgb, (1, 2, 0))[:, :, None, :]).max(-1)
    d = np.maximum(d, np.abs(lv.T - T[:, :, None]) * (atol / t_atol))
    ok = valid & (d <= atol)
    if nc is not None:
        ok &= lv.nc == np.asarray(nc)[:, :, None]
    checked = lv.n > 0
    anyok = ok.any(-1)
    failed = checked & ~anyok
    if failed.any():
        y, x = np.argwhere(failed)[0]
        k = int(lv.n[y, x])
        raise AssertionError(
            f"{name}: {int(failed.sum())} pixels match no admissible result; e.g. window pixel ({x},{y}): "
            f"gpu rgb {rgb[:, y, x]} T {T[y, x]}" + (f" nc {np.asarray(nc)[y, x]}" if nc is not None else "") +
            f"; oracle leaves rgb {lv.C[y, x, :k].tolist()} T {lv.T[y, x, :k].tolist()} nc {lv.nc[y, x, :k].tolist()}")
    stats = {"pixels": h * w, "excluded": int((~checked).sum()), "branched": int((lv.n > 1).sum()),
             "other_branch": int((checked & ~ok[:, :, 0] & anyok).sum())}
    _add_parity(name, stats)
    assert stats["excluded"] <= EXCLUDED_MAX * stats["pixels"], (name, stats)
    if checked.any():
        record(name, float(np.where(ok, d, np.inf).min(-1)[checked].max()))
    bits = np.left_shift(np.uint64(1), lidx.astype(np.uint64))
    return np.bitwise_or.reduce(np.where(ok, bits[None, None, :], np.uint64(0)), axis=-1)


def envelope_err(gpu, lo, hi, abs_sum=None, floor_rel=GRAD_FLOOR):
    """Per element: the distance of gpu from [lo, hi] over max(|mid|, floor_rel * max|mid| of the
    tensor[, SUM_FLOOR * abs_sum]); with lo = hi it is grad_rel_err (or sum_rel_err)."""
    gpu, lo, hi = (np.asarray(a, np.float64) for a in (gpu, lo, hi))
    if lo.size == 0:
        return np.zeros(lo.shape)
    mid = 0.5 * (lo + hi)
    dist = np.maximum(np.maximum(lo - gpu, gpu - hi), 0.0)
    den = np.maximum(np.abs(mid), floor_rel * max(float(np.abs(mid).max()), 1e-30))
    if abs_sum is not None:
        den = np.maximum(den, SUM_FLOOR * np.asarray(abs_sum, np.float64))
    return dist / np.maximum(den, 1e-30)


def assert_envelope(gpu, lo, hi, name, abs_sum=None, rtol=GRAD_RTOL):
    err = envelope_err(gpu, lo, hi, abs_sum)
    e = float(err.max()) if err.size else 0.0
    if e > rtol:
        k = np.unravel_index(int(np.argmax(err)), err.shape)
        g0 = np.asarray(gpu, np.float64)[k]
        l0, h0 = np.asarray(lo, np.float64)[k], np.asarray(hi, np.float64)[k]
        extra = "" if abs_sum is None else f", sum|terms| {np.asarray(abs_sum)[k]:.6e}"
        name = f"{name} [worst at {tuple(int(i) for i in k)}: gpu {g0:.9e}, envelope [{l0:.9e}, {h0:.9e}]{extra}]"
    record("grad rel " + name, e)
    wide = int((np.asarray(hi) > np.asarray(lo)).any(axis=tuple(range(1, np.ndim(lo)))).sum()) if np.size(lo) else 0
    _add_parity("grad " + name, {"elements": int(np.shape(lo)[0]) if np.ndim(lo) else 0, "branch_envelope": wide})
    assert e <= rtol, f"{name}: relative distance from the admissible envelope {e:.3e} > {rtol}"
    return e


# End to end, the GPU composites its own float32 splats, whose per-pixel terms differ from the
# oracle's FP64 ones by the float32 projection's error, not only by float32 sums. Where a
# per-splat gradient is a sum of terms that cancel, that difference is a fraction of the sum of
# the terms' magnitudes, not of the result: the end-to-end envelope is widened by E2E_TERM_REL
# times that sum. E2E_TERM_REL is the relative float32 error of an end-to-end alpha that the
# branch margins already assume (MARGINS_E2E); the largest seen on the full-size batched views
# was 4e-4 of the sum. The stage tests, on identical float32 splats, keep the tight
# float32-summation floor, except where a test makes the terms cancel on purpose: there the
# per-pixel terms still differ by the float32 renderer's own alpha and T error (the stage
# margin MARGINS_STAGE, 2e-5: the adjoint's transmittance, recovered by division back
# through the list, drifts about an ulp a splat), and the envelope widens by STAGE_TERM_REL
# times the sum of the terms' magnitudes.
E2E_TERM_REL = float(oracle.MARGINS_E2E[0])
STAGE_TERM_REL = float(oracle.MARGINS_STAGE[0])


def split2d(a):
    """[n,12] grad2d layout -> oracle.Grad2D."""
    a = np.asarray(a, np.float64)
    return oracle.Grad2D(a[:, 0:2].copy(), a[:, 2:5].copy(), a[:, 6:9].copy(), a[:, 5].copy())


PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _project_bwd_box(g64, cam, mid, half, tile, sh_degree, crop, aabb, vis=None, col=None):
    """(centre, half-width) of the projection adjoint of every Gaussian of g64 when its 2D
    gradients lie in mid +- half, under the given culling / colour-clamp flips."""
    with oracle.branch_flips(vis, col):
        base = oracle.project_bwd(g64, cam, split2d(mid), tile, sh_degree, crop, aabb)
    hw = {k: np.zeros_like(getattr(base, k)) for k in PARAMS}
    S = np.nonzero(half[:, :9].max(axis=1) > 0)[0]
    if len(S):
        sub = {k: np.asarray(v)[S] for k, v in g64.items()}
        with oracle.branch_flips(None if vis is None else vis[S], None if col is None else col[S]):
            for j in range(9):
                e = np.zeros((len(S), 12))
                e[:, j] = half[S, j]
                if not e.any():
                    continue
                r = oracle.project_bwd(sub, cam, split2d(e), tile, sh_degree,
                                       None if crop is None else np.asarray(crop)[S], None)
                for k in PARAMS:
                    hw[k][S] += np.abs(getattr(r, k))
    return base, hw


def param_envelope(g64, cam, p: oracle.Projection, lo2d, hi2d, tile, sh_degree=3, crop=None, aabb=None,
                   margins=oracle.MARGINS_E2E):
    """Envelope of the projection adjoint (the raw-parameter gradients and the SD statistic of
    one view) when the 2D gradients lie in [lo2d, hi2d] ([n,12]) and, for Gaussians whose
    culling or colour clamp is marginal in ``p`` (projected with ``margins``), either outcome
    is taken. The adjoint is linear in the 2D gradients: the centre maps to the centre, and
    the half-widths through the absolute values of the chain rule (evaluated column by column
    on the Gaussians with a nonzero half-width). The other outcomes of marginal decisions are
    evaluated on those Gaussians only (a Gaussian's adjoint depends on nothing else). Returns
    {name: (lo, hi)} for PARAMS, sd_acc and sd_cnt."""
    lo2d, hi2d = np.asarray(lo2d, np.float64), np.asarray(hi2d, np.float64)
    n = p.n
    c = cam if isinstance(cam, dict) else cam.as_dict()
    vis_flip = oracle.marginal_visibility(p)
    col_bits = np.zeros(n, np.uint8)
    if p.color_raw is not None:
        for ch in range(3):
            col_bits |= ((np.abs(p.color_raw[:, ch]) < margins[3]).astype(np.uint8) << ch)
    mid, half = 0.5 * (lo2d + hi2d), 0.5 * (hi2d - lo2d)
    sx, sy = 0.5 * c["width"], 0.5 * c["height"]
    ulo, uhi, vlo, vhi = lo2d[:, 0] * sx, hi2d[:, 0] * sx, lo2d[:, 1] * sy, hi2d[:, 1] * sy
    near_u = np.where((ulo <= 0) & (uhi >= 0), 0.0, np.minimum(np.abs(ulo), np.abs(uhi)))
    near_v = np.where((vlo <= 0) & (vhi >= 0), 0.0, np.minimum(np.abs(vlo), np.abs(vhi)))
    far_u, far_v = np.maximum(np.abs(ulo), np.abs(uhi)), np.maximum(np.abs(vlo), np.abs(vhi))
    sd_lo, sd_hi = np.hypot(near_u, near_v), np.hypot(far_u, far_v)

    def box(base, hw, cnt):
        r = {k: [getattr(base, k) - hw[k], getattr(base, k) + hw[k]] for k in PARAMS}
        cnt = cnt.astype(np.float64)
        r["sd_cnt"] = [cnt, cnt.copy()]
        r["sd_acc"] = [np.where(cnt > 0, sd_lo_, 0.0), np.where(cnt > 0, sd_hi_, 0.0)]
        return r

    sd_lo_, sd_hi_ = sd_lo, sd_hi
    base, hw = _project_bwd_box(g64, cam, mid, half, tile, sh_degree, crop, aabb)
    out = box(base, hw, base.sd_cnt)
    F = np.nonzero(vis_flip | (col_bits != 0))[0]
    if len(F):
        sub = {k: np.asarray(v)[F] for k, v in g64.items()}
        sd_lo_, sd_hi_ = sd_lo[F], sd_hi[F]
        crop_f = None if crop is None else np.asarray(crop)[F]
        for vis, col in ((vis_flip[F].astype(np.uint8), None), (None, col_bits[F]),
                         (vis_flip[F].astype(np.uint8), col_bits[F])):
            if (vis is not None and not vis.any()) or (col is not None and not col.any()):
                continue
            b, h = _project_bwd_box(sub, cam, mid[F], half[F], tile, sh_degree, crop_f, aabb, vis, col)
            r = box(b, h, b.sd_cnt)
            for k in out:
                out[k][0][F] = np.minimum(out[k][0][F], r[k][0])
                out[k][1][F] = np.maximum(out[k][1][F], r[k][1])
    return {k: tuple(v) for k, v in out.items()}


def add_envelopes(a, b):
    """Sum of two views' envelopes (a per-view choice of admissible outcome in each)."""
    if a is None:
        return {k: (v[0].copy(), v[1].copy()) for k, v in b.items()}
    return {k: (a[k][0] + b[k][0], a[k][1] + b[k][1]) for k in a}


def assert_params_in_envelope(grads, env, name, rows=None):
    """grads: {name: array} from the GPU; env: param_envelope output. rows (bool) restricts."""
    sel = (lambda a: a) if rows is None else (lambda a: np.asarray(a)[rows])
    for k in PARAMS:
        assert_envelope(sel(grads[k]), sel(env[k][0]), sel(env[k][1]), f"{k} {name}")
    if "sd_cnt" in grads:
        c = sel(np.asarray(grads["sd_cnt"], np.float64))
        assert np.all((c >= sel(env["sd_cnt"][0])) & (c <= sel(env["sd_cnt"][1]))), f"sd_cnt {name}"
        assert_envelope(sel(grads["sd_acc"]), sel(env["sd_acc"][0]), sel(env["sd_acc"][1]), f"sd_acc {name}")


def check_lists_admissible(gpu_ids, gpu_ts, eb: oracle.ExtBins, tiles, tile_off=0, entry_off=0, name="lists"):
    """Per tile t of ``tiles``: the GPU's list (entry ids minus entry_off) holds every certain
    member of the oracle's extended list, no Gaussian outside it, and in its order (tile,
    fp32 depth, index) -- bit-exact index work, with each uncertain member either present or
    absent as its marginal projection decision went."""
    n_unc = 0
    for t in tiles:
        a = np.asarray(gpu_ids[gpu_ts[tile_off + t]:gpu_ts[tile_off + t + 1]]) - entry_off
        b = eb.ids[eb.tile_start[t]:eb.tile_start[t + 1]]
        u = eb.unc[eb.tile_start[t]:eb.tile_start[t + 1]]
        inset = np.isin(b, a)
        np.testing.assert_array_equal(a, b[inset], err_msg=f"{name}: tile {t}")
        assert np.all(inset[u == 0]), f"{name}: tile {t} misses a certain member"
        n_unc += int((u != 0).sum())
    _add_parity(name, {"tiles": len(tiles), "uncertain_members": n_unc})


def windows_tiles(win, cam, tile):
    """Tile indices (of the item's grid) that the pixel window (x0, y0, x1, y1) touches."""
    c = cam if isinstance(cam, dict) else cam.as_dict()
    gx = -(-c["width"] // tile[0])
    x0, y0, x1, y1 = win
    return [ty * gx + tx for ty in range(y0 // tile[1], -(-y1 // tile[1])) for tx in range(x0 // tile[0], -(-x1 // tile[0]))]


def resolve_membership(eb: oracle.ExtBins, gpu_ids, gpu_ts, tiles, tile_off=0, entry_off=0, gpu_mean2d=None,
                       gpu_radius=None, p: oracle.Projection | None = None, cam=None, tile=None,
                       name="lists"):
    """The GPU's per-tile lists as a certificate for the membership part of its decisions.

    An uncertain member of the oracle's extended lists (a Gaussian whose radius, rectangle
    edge or fov-guard decision float32 may take either way) is in a tile's list under one
    outcome and out under the other. Enumerating every combination per pixel is infeasible
    where many such Gaussians overlap, so the decision the GPU took is read from its list and
    checked instead: the GPU list must be the oracle's list with each uncertain member in or
    out (check_lists_admissible), and, given the GPU's projection, each uncertain Gaussian's
    radius must be one its decision allows (the oracle's, one more or less, or culled) and its
    membership in every checked tile must be exactly its own tile rectangle's. The lists
    returned are then the oracle's with every uncertain member fixed to that verified outcome,
    and the oracle composites them with its own FP64 splats: nothing but the choice between
    admissible outcomes comes from the GPU."""
    check_lists_admissible(gpu_ids, gpu_ts, eb, tiles, tile_off, entry_off, name)
    c = None if cam is None else (cam if isinstance(cam, dict) else cam.as_dict())
    out_ids, out_ts = [], np.zeros_like(eb.tile_start)
    pos = 0
    tl = sorted(set(tiles))
    unc_g = np.unique(eb.ids[eb.unc != 0])
    if gpu_radius is not None and len(unc_g):
        r_gpu = np.asarray(gpu_radius)[entry_off + unc_g]
        ok = (r_gpu == p.radius[unc_g]) | (r_gpu == 0) | (np.abs(r_gpu - p.radius_all[unc_g]) <= 1)
        assert np.all(ok), f"{name}: an uncertain Gaussian's GPU radius is outside its admissible set"
        rect = rect_of(np.asarray(gpu_mean2d)[entry_off + unc_g], r_gpu, c, tile)
        gx = -(-c["width"] // tile[0])
        where = {int(g): k for k, g in enumerate(unc_g)}
    prev = 0
    for t in tl:
        out_ts[prev:t + 1] = pos
        b = eb.ids[eb.tile_start[t]:eb.tile_start[t + 1]]
        u = eb.unc[eb.tile_start[t]:eb.tile_start[t + 1]]
        a = np.asarray(gpu_ids[gpu_ts[tile_off + t]:gpu_ts[tile_off + t + 1]]) - entry_off
        inset = np.isin(b, a)
        if gpu_radius is not None:
            tx, ty = t % gx, t // gx
            for g, i_in in zip(b[u != 0], inset[u != 0]):
                x0, y0, x1, y1 = rect[where[int(g)]]
                assert bool(i_in) == bool(x0 <= tx < x1 and y0 <= ty < y1), \
                    f"{name}: Gaussian {int(g)} in tile {t} disagrees with its own GPU rectangle"
        keep = (u == 0) | inset
        out_ids.append(b[keep])
        pos += int(keep.sum())
        prev = t + 1
    out_ts[prev:] = pos
    ids = np.concatenate(out_ids) if out_ids else np.zeros(0, np.int32)
    return oracle.ExtBins(ids.astype(np.int32), np.zeros(len(ids), np.uint8), out_ts)
