"""Parity at full size, in the launch configurations bench.py times.

The oracle cannot composite whole 1600x1066 / 1920x1080 views in seconds, so it checks
sampled 32x32 pixel windows (every Gaussian projected, only the windows' tiles binned and
composited), 16 per view, chosen deterministically: the tiles with the longest lists, the
pixels with the deepest composites (largest n_contrib), and seeded random places. In each:
- end to end (GPU projection -> GPU bins -> GPU image): every pixel matches one of the
  oracle's admissible results (decisions float32 may take either way enumerated), and every
  window tile's list is the oracle's, each uncertain member in or out;
- the composite adjoint, a stage test on the oracle's float32 splats (both sides composite
  and differentiate the same inputs): with dL/dC nonzero on the windows, each per-splat 2D
  gradient (a float32 sum over up to thousands of pixels) lies within relative 1e-3 of the
  envelope of the adjoints of the results the GPU's forward matched, floored at 3e-3 of the
  sum of its terms' magnitudes;
- the projection adjoint fed the oracle's 2D gradients: every parameter gradient of every
  Gaussian within relative 1e-3 of its envelope (either outcome of a marginal culling or
  colour-clamp decision).
The batched multi-block step is checked item by item the same way (images and lists), and
its parameter gradients -- summed over the views of each set inside one CUDA graph --
against the sum of the oracle's per-view adjoint envelopes.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import (E2E_TERM_REL, assert_envelope, assert_params_in_envelope, match_image, oracle_grad2d_array,
                           param_envelope, rect_tiles, resolve_membership, splat_array, windows_tiles)

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe

WIN = 32


def pick_windows(cam, tile, tile_len, n_contrib, n_long=6, n_deep=5, n_rand=5, seed=0):
    """16 disjoint 32x32 windows (aligned to 16 px): around the tiles with the longest lists
    (tile_len per tile of this view), around the pixels with the deepest composites
    (n_contrib [H, W]), and at seeded random places."""
    W, H = cam["width"], cam["height"]
    gx = -(-W // tile[0])
    out = []

    def add(cx, cy):
        x0 = int(np.clip((cx - WIN // 2) // 16 * 16, 0, (W - WIN) // 16 * 16))
        y0 = int(np.clip((cy - WIN // 2) // 16 * 16, 0, (H - WIN) // 16 * 16))
        if any(x0 < b[2] and b[0] < x0 + WIN and y0 < b[3] and b[1] < y0 + WIN for b in out):
            return False
        out.append((x0, y0, x0 + WIN, y0 + WIN))
        return True

    k = 0
    for t in np.argsort(-tile_len, kind="stable"):
        if k == n_long:
            break
        k += add((t % gx) * tile[0] + tile[0] // 2, (t // gx) * tile[1] + tile[1] // 2)
    k = 0
    for p in np.argsort(-n_contrib.ravel(), kind="stable")[:200000]:
        if k == n_deep:
            break
        k += add(p % W, p // W)
    rng = np.random.default_rng(seed)
    while len(out) < n_long + n_deep + n_rand:
        add(int(rng.integers(0, W)), int(rng.integers(0, H)))
    return out


def check_image_windows(cam, tile, p, rgb, T, gpu_ids, gpu_ts, tile_off, entry_off, gpu_mean2d, gpu_radius, wins,
                        name):
    """End-to-end image and tile lists of one view's windows. The lists must be admissible
    (uncertain members in or out as the GPU's own radius and rectangle say); the oracle then
    composites its lists with those memberships, and every pixel must match one of its
    admissible results. Returns (resolved lists, admissible-leaf masks per window)."""
    with oracle.windows(wins):
        eb = oracle.bin_ext(p, cam, tile)
    tiles = sorted({t for w in wins for t in windows_tiles(w, cam, tile)})
    rb = resolve_membership(eb, gpu_ids, gpu_ts, tiles, tile_off, entry_off, gpu_mean2d, gpu_radius, p, cam, tile,
                            f"tile lists {name} (end to end)")
    adms = []
    for w in wins:
        lv = oracle.render_leaves(p, rb, cam, tile, margins=oracle.MARGINS_E2E, win=w)
        x0, y0, x1, y1 = w
        adms.append(match_image(lv, rgb[:, y0:y1, x0:x1], T[y0:y1, x0:x1], None, f"image {name} (end to end)"))
    return rb, adms


def windows_dL(cam, wins, seed=3):
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(seed)
    dL = np.zeros((3, H, W), np.float32)
    for (x0, y0, x1, y1) in wins:
        dL[:, y0:y1, x0:x1] = rng.standard_normal((3, y1 - y0, x1 - x0))
    return dL


def run_single(wl, crop=None, tile=None, px=(0, 0)):
    g = wl.sets[0]
    cam = wl.cameras[0].as_dict()
    W, H = cam["width"], cam["height"]
    tile = tuple(tile or wl.tile)
    name = f"{W}x{H} {tile[0]}x{tile[1]}"
    sets = [lobe.GaussianSet.from_numpy(g)]
    if crop is not None:
        sets[0].crop_mask = torch.as_tensor(crop).cuda()
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=tile, px_fwd=px[0], px_bwd=px[1])
    proj, bins, img = lobe.forward(ctx, batch)
    rgb = img.rgb.view(3, H, W).cpu().numpy()
    T = img.T_final.view(H, W).cpu().numpy()
    nc = img.n_contrib.view(H, W).cpu().numpy()
    gts = bins.tile_start.cpu().numpy()
    wins = pick_windows(cam, tile, np.diff(gts), nc)
    g64 = oracle.set_dict(g)
    p = oracle.project(g64, cam, tile, crop=crop, margins=oracle.MARGINS_E2E)
    sp = proj.splat.cpu().numpy()
    check_image_windows(cam, tile, p, rgb, T, bins.ids().cpu().numpy(), gts, 0, 0, sp[:, 0:2],
                        proj.radius.cpu().numpy(), wins, name)

    # composite adjoint, stage: the oracle's float32 splats on both sides
    ps = p.rounded()
    ps.flags[:] = 0
    gp = lobe.Projection(torch.as_tensor(splat_array(ps)).cuda(), torch.as_tensor(ps.radius).cuda(),
                         torch.as_tensor(rect_tiles(ps.mean2d, ps.radius, cam, tile)).cuda())
    sbins = lobe.bin_sort(ctx, batch, gp)
    sout = lobe.render_fwd(ctx, batch, gp, sbins)
    srgb = sout.rgb.view(3, H, W).cpu().numpy()
    sT = sout.T_final.view(H, W).cpu().numpy()
    snc = sout.n_contrib.view(H, W).cpu().numpy()
    sids, sts = sbins.ids().cpu().numpy(), sbins.tile_start.cpu().numpy()
    dL = windows_dL(cam, wins)
    with oracle.windows(wins):
        ids, ts = oracle.bin_sort(ps, cam, tile)
        g2_plain = oracle.render_bwd(ps, ids, ts, cam, dL.astype(np.float64), tile)
    eb = oracle.ExtBins(ids, np.zeros(len(ids), np.uint8), ts)
    lo = np.zeros((ps.n, 12))
    hi = np.zeros((ps.n, 12))
    ab = np.zeros((ps.n, 12))
    for w in wins:
        for t in windows_tiles(w, cam, tile):  # the stage lists are bit-exact
            np.testing.assert_array_equal(sids[sts[t]:sts[t + 1]], ids[ts[t]:ts[t + 1]])
        lv = oracle.render_leaves(ps, eb, cam, tile, margins=oracle.MARGINS_STAGE, win=w, certain=True)
        x0, y0, x1, y1 = w
        adm = match_image(lv, srgb[:, y0:y1, x0:x1], sT[y0:y1, x0:x1], snc[y0:y1, x0:x1], f"image {name} (stage)")
        l, h, a = oracle.render_bwd_envelope(ps, eb, cam, dL.astype(np.float64), adm, tile, margins=oracle.MARGINS_STAGE,
                                             win=w, certain=True)
        lo += l
        hi += h
        ab += a
    g2d = lobe.render_bwd(ctx, batch, gp, sbins, sout, torch.as_tensor(dL).cuda().reshape(-1)).cpu().numpy()
    vis = ps.radius > 0
    assert (np.abs(hi[vis, :9]).sum(1) > 0).sum() > 50
    for nm, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)), ("color", slice(6, 9))]:
        assert_envelope(g2d[vis, cols], lo[vis, cols], hi[vis, cols], f"grad2d {nm} {name} (stage)", abs_sum=ab[vis, cols])

    # projection adjoint on the GPU's own projection, fed the oracle's (float32) 2D gradients
    g2r = oracle_grad2d_array(oracle.Grad2D(*(a.astype(np.float32).astype(np.float64) for a in
                                              (g2_plain.mean2d, g2_plain.conic, g2_plain.color, g2_plain.opacity))))
    aabb = wl.blocks[0] if wl.blocks else None
    env = param_envelope(g64, cam, p, g2r, g2r, tile, crop=crop, aabb=aabb)
    grads = lobe.zero_grads(batch, sd=aabb is not None)
    lobe.project_bwd(ctx, batch, proj, torch.as_tensor(g2r, dtype=torch.float32).cuda(), grads, accumulate=True)
    gr = {k: v.cpu().numpy() for k, v in grads[0].items()}
    assert_params_in_envelope(gr, env, f"{name} (stage)")


# tile shape and pixels per lane: the defaults, and the configurations bench.py's autotuner picks
# for the workload (32x16 tiles with 4 / 8 pixels per lane for the medium view; 16x16 with 2 / 4
# for the city block, with 8x8 and 1 / 2 within a percent of it)
@pytest.mark.parametrize("tile, px", [((16, 16), (0, 0)), ((32, 16), (4, 8))])
def test_fullsize_medium_200k_1600x1066(tile, px):
    run_single(scenes.medium_scene(), tile=tile, px=px)


@pytest.mark.parametrize("tile, px", [((16, 16), (0, 0)), ((16, 16), (2, 4)), ((8, 8), (1, 2))])
def test_fullsize_city_block_with_visibility_crop(tile, px):
    wl = scenes.city_block_scene(n=4_000_000)
    # the block's visibility crop (Sec. 3.3) from the GPU, checked against the oracle's
    sets = [lobe.GaussianSet.from_numpy(wl.sets[0])]
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    crop = lobe.visibility_crop(lobe.Context(tile=wl.tile), batch)[0].cpu().numpy()
    g64 = oracle.set_dict(wl.sets[0])
    p = oracle.project(g64, wl.cameras[0].as_dict(), wl.tile, margins=oracle.MARGINS_E2E)
    marg = oracle.marginal_visibility(p)
    sure = (p.radius > 0) & ~marg
    np.testing.assert_array_equal(crop[sure], 1)
    np.testing.assert_array_equal(crop[~sure & ~marg], 0)
    assert 0.05 < sure.mean() < 0.95
    run_single(wl, crop=crop, tile=tile, px=px)


def test_fullsize_multi_block_batched_graph():
    """The batched multi-block step (graph-captured, autotuned tile shape and pixels per lane):
    images and tile lists item by item on 16 windows of one view per block, and the parameter
    gradients of every set -- each the sum over its views inside the graph -- against the sum
    of the oracle's per-view envelopes, with dL/dC nonzero on those windows only."""
    from paper_2510_01767_b300.batched import autotune
    wl = scenes.multi_block_scene(seed=0)
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    st, _ = autotune(sets, cams, wl.items, wl.blocks, reps=2, use_cache=False)
    tile = st.tile
    # one view per block: its first item
    chosen = {}
    for i, (s, c, b) in enumerate(wl.items):
        chosen.setdefault(s, i)
    st.dL.zero_()
    st.replay()  # forward with the graph, to place the windows
    torch.cuda.synchronize()
    ts = st.bins.tile_start.cpu().numpy()
    n_tiles, toffs = st.batch.tiles(tile)
    ncs = st.batch.image_views(st.image.n_contrib, channels=1)
    wins = {}
    dls = st.dL_views()
    for s, i in chosen.items():
        c = cams[wl.items[i][1]]
        nt = -(-c["width"] // tile[0]) * -(-c["height"] // tile[1])
        wins[i] = pick_windows(c, tile, np.diff(ts[toffs[i]:toffs[i] + nt + 1]), ncs[i].cpu().numpy(), seed=i)
        dls[i].copy_(torch.as_tensor(windows_dL(c, wins[i], seed=10 + i)).reshape(dls[i].shape))
    st.replay()
    torch.cuda.synchronize()
    ids = st.bins.gauss_ids[:int(st.bins.n_isect.item())].cpu().numpy()
    ts = st.bins.tile_start.cpu().numpy()
    views = st.images()
    Ts = st.batch.image_views(st.image.T_final, channels=1)
    splat = st.proj.splat.cpu().numpy()
    radius = st.proj.radius.cpu().numpy()
    for s, i in chosen.items():
        _, c, b = wl.items[i]
        cam = cams[c]
        g64 = oracle.set_dict(wl.sets[s])
        p = oracle.project(g64, cam, tile, margins=oracle.MARGINS_E2E)
        W, H = cam["width"], cam["height"]
        rgb = views[i].cpu().numpy().reshape(3, H, W)
        T = Ts[i].cpu().numpy().reshape(H, W)
        name = f"batched item {i} {W}x{H}"
        e0 = st.batch.entry_off[i]
        rb, adms = check_image_windows(cam, tile, p, rgb, T, ids, ts, toffs[i], e0, splat[:, 0:2], radius, wins[i],
                                       name)
        dL = dls[i].cpu().numpy().reshape(3, H, W).astype(np.float64)
        lo = np.zeros((p.n, 12))
        hi = np.zeros((p.n, 12))
        ab = np.zeros((p.n, 12))
        for w, adm in zip(wins[i], adms):
            l, h, a = oracle.render_bwd_envelope(p, rb, cam, dL, adm, tile, margins=oracle.MARGINS_E2E, win=w)
            lo += l
            hi += h
            ab += a
        # end to end the GPU's own float32 splats: the envelope widened by E2E_TERM_REL of the
        # terms' magnitudes
        lo -= E2E_TERM_REL * ab
        hi += E2E_TERM_REL * ab
        # the per-splat 2D gradients of this item's entries
        g2 = st.grad2d[e0:e0 + p.n].cpu().numpy()
        seen = np.abs(ab[:, :9]).sum(1) > 0
        for nm, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                         ("color", slice(6, 9))]:
            assert_envelope(g2[seen, cols], lo[seen, cols], hi[seen, cols], f"grad2d {nm} {name} (end to end)",
                            abs_sum=ab[seen, cols])
        env = param_envelope(g64, cam, p, lo, hi, tile, aabb=wl.blocks[b] if b >= 0 else None)
        # parameters only: the graph's SD statistic accumulates over every replay and view
        gr = {k: st.grads[s][k].cpu().numpy() for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        assert_params_in_envelope(gr, env, f"batched set {s} ({wl.sets[s].n} Gaussians, end to end)")
