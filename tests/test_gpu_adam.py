"""Adam on the GPU (appendix "3DGS Training": the 3DGS optimizer of the fine-training, and the
sparse variant of the coarse training) against the FP64 oracle.

* The standalone update (lobe_adam) on seeded parameters, gradients and moments, over several
  steps, dense and sparse, at ragged sizes: each side evolves its own state; the bound is a few
  float32 roundings per step of each term (derived in ``adam_bounds``).
* The update fused into the projection adjoint (lobe_project_bwd_adam) against the oracle's
  projection adjoint followed by its Adam, on the oracle's float32-rounded splats and 2D
  gradients: the moments within the gradient bar carried through the moment equations, the
  parameters inside the interval the moment bounds allow.
* Fused against unfused on the GPU (the adjoint's gradients through lobe_adam), sparse and
  standard, on a multi-set, multi-view batch.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import GRAD_FLOOR, GRAD_RTOL, oracle_grad2d_array, record

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe

KEYS = oracle.ADAM_KEYS
LR = dict(means=1.6e-4 * 20.0, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20)
B1, B2, EPS = 0.9, 0.999, 1e-15
U32 = 2.0 ** -24  # unit roundoff of float32


def shapes(n):
    return dict(means=(n, 3), log_scales=(n, 3), quats=(n, 4), opacity_logits=(n,), sh=(n, 16, 3))


def f32(d):
    return {k: np.asarray(v, np.float32) for k, v in d.items()}


def random_grads(rng, n):
    """Gradients with magnitudes spread log-uniformly over 1e-8 .. 1 and random signs."""
    return f32({k: rng.choice([-1.0, 1.0], s) * 10.0 ** rng.uniform(-8, 0, s) for k, s in shapes(n).items()})


def rate_array(key, shape):
    if key == "sh":
        r = np.full(shape[1:], LR["sh_rest"])
        r[0, :] = LR["sh_dc"]
        return r
    return LR[key]


def to_dev(d):
    return {k: torch.as_tensor(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def to_host(d):
    return {k: v.cpu().numpy().astype(np.float64) for k, v in d.items()}


def adam_bounds(m_abs, v, t, key, shape):
    """Float32 bound of one step's parameter change: ss m / (sqrt(v) rsb2 + eps) evaluated with
    |m| at most m_abs (the moment's sum of absolute terms, so cancellation in m is covered),
    times 16 unit roundoffs: the constants ss and rsb2 (1 each), m (2), half of v's 3, the
    approximate square root (2^-23: 2), the fma (1), the approximate division (2 ulp: 4), the
    product with ss (1), with the rest left for the moments' error carried from earlier steps."""
    ss = rate_array(key, shape) / (1 - B1 ** t)
    return 16 * U32 * ss * m_abs / (np.sqrt(v / (1 - B2 ** t)) + EPS)


@pytest.mark.parametrize("n, sparse", [(1001, False), (1001, True), (70_001, False), (70_001, True)])
def test_adam_kernel_matches_oracle(n, sparse):
    rng = np.random.default_rng(n + sparse)
    p0 = f32({k: rng.standard_normal(s) for k, s in shapes(n).items()})
    zeros = {k: np.zeros(s, np.float32) for k, s in shapes(n).items()}
    rows = (rng.uniform(size=n) < 0.4).astype(np.uint8) if sparse else None
    g_state = lobe.GaussianSet(**to_dev(p0))
    opt = lobe.Adam(g_state, lr=LR, betas=(B1, B2), eps=EPS)
    ctx = lobe.Context()
    p, m, v = p0, zeros, zeros
    m_abs = {k: np.zeros(s) for k, s in shapes(n).items()}  # sum of |terms| of each m
    p_tol = {k: np.zeros(s) for k, s in shapes(n).items()}
    sel = np.ones(n, bool) if rows is None else rows.astype(bool)
    for t in range(1, 4):
        g = random_grads(rng, n)
        opt.step(ctx, to_dev(g), None if rows is None else torch.as_tensor(rows).cuda())
        p, m, v = oracle.adam(p, g, m, v, t, LR, B1, B2, EPS, rows=None if rows is None else sel)
        for k in KEYS:
            shp = shapes(n)[k]
            m_abs[k][sel] = B1 * m_abs[k][sel] + (1 - B1) * np.abs(np.asarray(g[k], np.float64)[sel])
            step_tol = adam_bounds(m_abs[k], np.maximum(v[k], 1e-300), t, k, shp)
            p_tol[k][sel] += step_tol[sel] + 2 * U32 * np.abs(p[k][sel])
    gp = to_host({k: getattr(g_state, k) for k in KEYS})
    gm, gv = to_host(opt.exp_avg), to_host(opt.exp_avg_sq)
    worst = 0.0
    for k in KEYS:
        em = np.abs(gm[k] - m[k]) / np.maximum(m_abs[k], 1e-300)
        ev = np.abs(gv[k] - v[k]) / np.maximum(v[k], 1e-300)
        # moments: at most 4 roundings of each term per step, over 3 steps (v has no cancellation)
        assert float(em[sel].max()) <= 12 * U32, (k, float(em[sel].max()))
        assert float(ev[sel].max()) <= 12 * U32, (k, float(ev[sel].max()))
        ep = np.abs(gp[k] - p[k]) / np.maximum(p_tol[k], 1e-300)
        worst = max(worst, float(ep[sel].max()))
        assert float(ep[sel].max()) <= 1.0, (k, float(ep[sel].max()))
        if rows is not None:  # untouched rows keep their bits
            np.testing.assert_array_equal(gp[k][~sel], p0[k][~sel])
            assert np.all(gm[k][~sel] == 0) and np.all(gv[k][~sel] == 0)
    record("adam param error / bound", worst)


def test_adam_rejects_bad_arguments():
    ctx = lobe.Context()
    g = lobe.GaussianSet(**to_dev(f32({k: np.zeros(s) for k, s in shapes(4).items()})))
    opt = lobe.Adam(g, lr=LR)
    grads = to_dev(f32({k: np.zeros(s) for k, s in shapes(4).items()}))
    opt.t = -1  # step 0 is not an Adam step
    with pytest.raises(lobe.raster.A.LobeError):
        opt.step(ctx, grads)
    opt.t = 0
    opt.betas = (1.0, 0.999)
    with pytest.raises(lobe.raster.A.LobeError):
        opt.step(ctx, grads)
    opt.betas = (0.9, 0.999)
    opt.step(ctx, grads)  # zero gradients from zero moments: nothing moves
    assert torch.equal(g.means, torch.zeros_like(g.means)) and opt.t == 1


# ----------------------------------------------------------------------------- fused with the adjoint

def interval_of_update(m, dm, v, dv, ss, rsb2):
    """[lo, hi] of ss m' / (sqrt(v') rsb2 + eps) over m' in [m - dm, m + dm], v' in [v - dv, v + dv]
    (monotone in m', decreasing in v')."""
    vlo = np.maximum(v - dv, 0.0)
    vhi = v + dv
    den_lo = np.sqrt(vlo) * rsb2 + EPS
    den_hi = np.sqrt(vhi) * rsb2 + EPS
    cands = [ss * (m - dm) / den_lo, ss * (m - dm) / den_hi, ss * (m + dm) / den_lo, ss * (m + dm) / den_hi]
    return np.minimum.reduce(cands), np.maximum.reduce(cands)


@pytest.mark.parametrize("sparse", [True, False])
def test_fused_adjoint_adam_matches_oracle(sparse):
    """Small scene (a tenth of it behind the camera), one view: the oracle's 2D gradients
    (float32) through the fused GPU adjoint + Adam, against the oracle's adjoint + Adam, from a
    seeded state at step t = 5."""
    wl = scenes.small_scene()
    # every tenth Gaussian moved behind the camera: culled, so no view sees it
    wl.sets[0].means[::10, 2] *= -1.0
    g64 = oracle.set_dict(wl.sets[0])
    cam = wl.cameras[0].as_dict()
    f = oracle.forward(g64, cam, wl.tile, margins=oracle.MARGINS_STAGE)
    dL = np.random.default_rng(4).standard_normal((3, 128, 128)) * (f.pixel_flags == 0)[None]
    g2d = oracle.render_bwd(f.proj, f.ids, f.tile_start, cam, dL, wl.tile)
    g2d_r = oracle.Grad2D(*(a.astype(np.float32).astype(np.float64) for a in
                            (g2d.mean2d, g2d.conic, g2d.color, g2d.opacity)))
    want_g = oracle.project_bwd(g64, cam, g2d_r, wl.tile)
    n = g64["means"].shape[0]
    rng = np.random.default_rng(11)
    gm = {k: getattr(want_g, k) for k in KEYS}
    # a seeded state consistent with earlier steps: |m| <= sqrt(v)
    m0 = f32({k: rng.standard_normal(s) * np.abs(gm[k]).max() for k, s in shapes(n).items()})
    v0 = f32({k: (np.asarray(m0[k], np.float64) ** 2) * rng.uniform(1.0, 4.0, s) for k, s in shapes(n).items()})
    t = 5
    seen = f.proj.radius > 0
    want_p, want_m, want_v = oracle.adam(g64, gm, m0, v0, t, LR, B1, B2, EPS, rows=seen if sparse else None)

    gs = lobe.GaussianSet.from_numpy(wl.sets[0])
    batch = lobe.Batch([gs], wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=wl.tile)
    proj = lobe.project(ctx, batch)  # the fused kernel recomputes its forward from the parameters
    opt = lobe.Adam(gs, lr=LR, betas=(B1, B2), eps=EPS)
    opt.exp_avg = to_dev(m0)
    opt.exp_avg_sq = to_dev(v0)
    opt.t = t - 1
    lobe.project_bwd_adam(ctx, batch, proj, torch.as_tensor(oracle_grad2d_array(g2d_r), dtype=torch.float32).cuda(),
                          [opt], sparse=sparse)
    got_p = to_host({k: getattr(gs, k) for k in KEYS})
    got_m, got_v = to_host(opt.exp_avg), to_host(opt.exp_avg_sq)
    ok = (f.proj.flags == 0)
    gpu_seen = (proj.radius.cpu().numpy() > 0)
    assert np.array_equal(gpu_seen[ok], seen[ok])
    rsb2 = 1 / math.sqrt(1 - B2 ** t)
    worst = 0.0
    for k in KEYS:
        g = gm[k]
        # the gradient bar per element (relative 1e-3 with the floor 1e-3 max|g|)
        dg = GRAD_RTOL * np.maximum(np.abs(g), GRAD_FLOOR * max(np.abs(g).max(), 1e-30))
        dg = np.where(seen.reshape((-1,) + (1,) * (g.ndim - 1)), dg, 0.0)
        m0k, v0k = np.asarray(m0[k], np.float64), np.asarray(v0[k], np.float64)
        dm = (1 - B1) * dg + 4 * U32 * (B1 * np.abs(m0k) + (1 - B1) * np.abs(g))
        dv = (1 - B2) * (2 * np.abs(g) * dg + dg * dg) + 4 * U32 * (B2 * v0k + (1 - B2) * g * g)
        sl = ok.reshape((-1,) + (1,) * (g.ndim - 1)) & np.ones_like(g, bool)
        assert np.all(np.abs(got_m[k] - want_m[k])[sl] <= dm[sl]), k
        assert np.all(np.abs(got_v[k] - want_v[k])[sl] <= dv[sl]), k
        ss = rate_array(k, g.shape) / (1 - B1 ** t)
        lo, hi = interval_of_update(want_m[k], dm, want_v[k], dv, ss, rsb2)
        slack = 16 * U32 * np.maximum(np.abs(lo), np.abs(hi)) + 2 * U32 * np.abs(want_p[k])
        p0k = np.asarray(g64[k], np.float64)
        step = p0k - got_p[k]
        moved = seen.reshape((-1,) + (1,) * (g.ndim - 1)) | (not sparse)
        inside = (step >= lo - slack) & (step <= hi + slack)
        assert np.all(inside[sl & moved]), (k, int((~inside[sl & moved]).sum()))
        if sparse:
            stay = sl & ~seen.reshape((-1,) + (1,) * (g.ndim - 1))
            np.testing.assert_array_equal(got_p[k][stay], p0k[stay])
            np.testing.assert_array_equal(got_m[k][stay], m0k[stay])
        # how far into its allowance the parameter step went (0: the oracle's step)
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo) + slack
        worst = max(worst, float((np.abs(step - mid) / np.maximum(half, 1e-300))[sl & moved].max()))
    record("fused adam step / allowance", worst)
    assert seen.sum() > 100 and (~seen).sum() > 0  # both kinds of Gaussians present


@pytest.mark.parametrize("sparse", [True, False])
def test_fused_equals_adjoint_then_adam(sparse):
    """Two sets of two views each (uneven sizes and resolutions): the fused step against
    lobe_project_bwd followed by lobe_adam (rows = Gaussians some item sees when sparse)."""
    rng = np.random.default_rng(5)
    sets_np = [scenes.uniform_gaussians(rng, 30_001, 10.0, 5.0, 50.0, logscale_shift=math.log(10.0)),
               scenes.uniform_gaussians(rng, 12_345, 10.0, 5.0, 50.0, logscale_shift=math.log(10.0))]
    cams = [scenes.pinhole(320, 240, 240.0), scenes.pinhole(256, 200, 200.0, cx=40.0),
            scenes.pinhole(200, 160, 150.0), scenes.pinhole(180, 150, 140.0, cy=10.0)]
    items = [(0, 0, -1), (0, 1, -1), (1, 2, -1), (1, 3, -1)]

    # one forward and render adjoint for both paths (its atomics sum in no fixed order)
    ctx = lobe.Context(tile=(16, 16))
    batch0 = lobe.Batch([lobe.GaussianSet.from_numpy(s) for s in sets_np], cams, items)
    proj, bins, img = lobe.forward(ctx, batch0)
    dL = torch.as_tensor(np.random.default_rng(9).standard_normal(3 * batch0.n_pixels), dtype=torch.float32).cuda()
    g2d = lobe.render_bwd(ctx, batch0, proj, bins, img, dL)

    def run(fused):
        sets = [lobe.GaussianSet.from_numpy(s) for s in sets_np]
        batch = lobe.Batch(sets, cams, items)
        opts = [lobe.Adam(s, lr=LR, betas=(B1, B2), eps=EPS) for s in sets]
        for o, s in zip(opts, sets):  # a nonzero state at step 3
            r = np.random.default_rng(s.n)
            o.exp_avg = {k: torch.as_tensor(r.standard_normal(shapes(s.n)[k]) * 1e-3, dtype=torch.float32).cuda()
                         for k in KEYS}
            o.exp_avg_sq = {k: (o.exp_avg[k] ** 2) * 2 for k in KEYS}
            o.t = 2
        sd = lobe.zero_grads(batch)
        if fused:
            lobe.project_bwd_adam(ctx, batch, proj, g2d, opts, sd=sd, sparse=sparse)
        else:
            grads = lobe.project_bwd(ctx, batch, proj, g2d, sd)
            for i, (o, s) in enumerate(zip(opts, sets)):
                seen = torch.zeros(s.n, dtype=torch.bool, device="cuda")
                for e in [batch.entry_off[j] for j, it in enumerate(items) if it[0] == i]:
                    seen |= proj.radius[e:e + s.n] > 0
                o.step(ctx, grads[i], seen.to(torch.uint8) if sparse else None)
        torch.cuda.synchronize()
        return [{k: getattr(s, k).clone() for k in KEYS} for s in sets], \
               [({k: o.exp_avg[k].clone() for k in KEYS}, {k: o.exp_avg_sq[k].clone() for k in KEYS}) for o in opts], \
               [(d["sd_acc"].clone(), d["sd_cnt"].clone()) for d in sd]

    pf, mf, sf = run(True)
    pu, mu, su = run(False)
    worst = 0.0
    for s in range(2):
        for k in KEYS:
            for a, b in ((pf[s][k], pu[s][k]), (mf[s][0][k], mu[s][0][k]), (mf[s][1][k], mu[s][1][k])):
                if k != "means":  # the same float32 operations, bit for bit
                    assert torch.equal(a, b), (s, k)
                    continue
                # the two kernel instantiations may contract the position gradient's sums into
                # FMAs differently: float32 rounding, amplified where the sums cancel
                d = (a.double() - b.double()).abs()
                tol = 1e-5 * torch.maximum(b.double().abs(), 1e-3 * b.double().abs().max()) + 1e-30
                worst = max(worst, float((d / tol).max()))
                assert torch.all(d <= tol), (s, k, float(d.max()))
        assert torch.equal(sf[s][1], su[s][1])
        torch.testing.assert_close(sf[s][0], su[s][0], rtol=1e-6, atol=0)
    record("fused vs unfused adam, means (/1e-5 rel)", worst)


@pytest.mark.parametrize("sparse", [True, False])
def test_fused_adam_with_crop_mask_and_empty_set(sparse):
    """A cropped set next to an empty one: cropped Gaussians are culled, so sparse Adam leaves
    them (and everything unseen) bit for bit while standard Adam decays them; the empty set is a
    no-op; the seen Gaussians move as the adjoint followed by lobe_adam moves them."""
    rng = np.random.default_rng(3)
    g_np = scenes.uniform_gaussians(rng, 5_003, 1.0, 2.0, 6.0)
    crop = (rng.uniform(size=g_np.n) < 0.5).astype(np.uint8)
    empty = scenes.uniform_gaussians(rng, 0, 1.0, 2.0, 6.0)
    cams = [scenes.pinhole(96, 64, 80.0), scenes.pinhole(64, 64, 60.0)]
    items = [(0, 0, -1), (0, 1, -1), (1, 1, -1)]

    def make_sets():
        sets = [lobe.GaussianSet.from_numpy(g_np), lobe.GaussianSet.from_numpy(empty)]
        sets[0].crop_mask = torch.as_tensor(crop).cuda()
        return sets

    # one forward and render adjoint for both paths (its atomics sum in no fixed order)
    ctx = lobe.Context(tile=(16, 16))
    batch0 = lobe.Batch(make_sets(), cams, items)
    proj, bins, img = lobe.forward(ctx, batch0)
    dL = torch.as_tensor(np.random.default_rng(8).standard_normal(3 * batch0.n_pixels), dtype=torch.float32).cuda()
    g2d = lobe.render_bwd(ctx, batch0, proj, bins, img, dL)

    def run(fused):
        sets = make_sets()
        batch = lobe.Batch(sets, cams, items)
        opts = [lobe.Adam(s, lr=LR, betas=(B1, B2), eps=EPS) for s in sets]
        m0 = {k: torch.as_tensor(np.random.default_rng(2).standard_normal(shapes(g_np.n)[k]) * 1e-3,
                                 dtype=torch.float32).cuda() for k in KEYS}
        opts[0].exp_avg = {k: v.clone() for k, v in m0.items()}
        opts[0].exp_avg_sq = {k: (v * v * 3).contiguous() for k, v in m0.items()}
        opts[0].t = 4
        seen = ((proj.radius[0:g_np.n] > 0) | (proj.radius[g_np.n:2 * g_np.n] > 0))
        if fused:
            lobe.project_bwd_adam(ctx, batch, proj, g2d, opts, sparse=sparse)
        else:
            grads = lobe.project_bwd(ctx, batch, proj, g2d)
            opts[0].step(ctx, grads[0], seen.to(torch.uint8) if sparse else None)
        torch.cuda.synchronize()
        return {k: getattr(sets[0], k).clone() for k in KEYS}, seen

    pf, seen = run(True)
    pu, _ = run(False)
    seen = seen.cpu().numpy()
    cropped = crop == 0
    assert not np.any(seen & cropped)  # the crop mask culls
    assert seen.sum() > 100 and (~seen).sum() > 100
    p0 = {k: np.asarray(getattr(g_np, k)) for k in KEYS}
    for k in KEYS:
        a, b = pf[k].cpu().numpy(), pu[k].cpu().numpy()
        if k == "means":
            np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-7)
        else:
            np.testing.assert_array_equal(a, b)
        moved = np.any((a != p0[k]).reshape(g_np.n, -1), axis=1)
        if sparse:
            assert not np.any(moved[~seen]), k  # unseen rows keep their bits
        else:
            assert np.all(moved[~seen]), k  # standard Adam moves them by their momentum


def test_fused_adam_rejects_foreign_parameters():
    """The fused step updates the batch's own arrays: an Adam state over other tensors is an
    argument error (nothing launched), as is a missing optimizer."""
    rng = np.random.default_rng(4)
    g_np = scenes.uniform_gaussians(rng, 1_000, 1.0, 2.0, 6.0)
    gs = lobe.GaussianSet.from_numpy(g_np)
    other = lobe.GaussianSet.from_numpy(g_np)
    batch = lobe.Batch([gs], [scenes.pinhole(64, 64, 60.0)], [(0, 0, -1)])
    ctx = lobe.Context(tile=(16, 16))
    proj, bins, img = lobe.forward(ctx, batch)
    g2d = lobe.render_bwd(ctx, batch, proj, bins, img, torch.ones(3 * 64 * 64, device="cuda"))
    with pytest.raises(ValueError):
        lobe.project_bwd_adam(ctx, batch, proj, g2d, [lobe.Adam(other)])
    with pytest.raises(ValueError):
        lobe.project_bwd_adam(ctx, batch, proj, g2d, [])
    # the C ABI checks the same (the binding's check bypassed)
    opt = lobe.Adam(other)
    states = (lobe.raster.A.AdamState * 1)(opt._state())
    prms = (lobe.raster.A.AdamParams * 1)(opt._params(1))
    before_means, before_sh = gs.means.clone(), gs.sh.clone()
    code = ctx.lib.lobe_project_bwd_adam(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()),
                                         ctypes.c_void_p(g2d.data_ptr()), None, states, prms, 0)
    assert code == lobe.raster.A.ERR_ARG
    torch.cuda.synchronize()
    assert torch.equal(gs.means, before_means) and torch.equal(gs.sh, before_sh)
    ctx.status()
