"""GPU path vs the FP64 oracle, stage by stage and end to end, through the C ABI.

Stage tests feed every GPU stage the oracle's own upstream result rounded to float32, so
the comparison isolates one kernel's arithmetic; end-to-end tests chain the GPU stages.
Where float32 may take a decision either way (alpha at 1/255, T at 1e-4, the 0.99 clamp,
sigma < 0, a radius, rectangle edge or fov guard at its boundary, the colour clamp) the
oracle enumerates every outcome: each GPU pixel must match one of its pixel's admissible
results, and the gradients must lie in the envelope of the adjoints of the outcomes the
GPU's own forward matched (tests/helpers.py). No pixel or Gaussian is left out.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import (IMG_ATOL, STAGE_TERM_REL, add_envelopes, assert_envelope, assert_grad_close,
                           assert_params_in_envelope, check_lists_admissible, grad_rel_err, match_image,
                           oracle_grad2d_array, param_envelope, rect_of, rect_tiles, splat_array)

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def make_batch(wl, crop=None):
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    if crop is not None:
        sets[0].crop_mask = dev(crop, torch.uint8)
    return lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)


def gpu_projection_from_oracle(p, cam, tile):
    return lobe.Projection(dev(splat_array(p)), dev(p.radius, torch.int32),
                           dev(rect_tiles(p.mean2d, p.radius, cam, tile), torch.int32))


@pytest.fixture(scope="module")
def small():
    wl = scenes.small_scene()
    g64 = oracle.set_dict(wl.sets[0])
    return wl, g64


def ctx_for(wl, **kw):
    return lobe.Context(tile=wl.tile, **kw)


@pytest.mark.parametrize("posed", [False, True])
def test_project_matches_oracle(small, posed):
    wl, g = small
    cam = wl.cameras[0].as_dict()
    if posed:
        cam = dict(cam, viewmat=scenes.look_at((0.8, -0.6, -0.5), (0.0, 0.0, 4.0), up=(0, -1, 0)))
        wl = scenes.Workload(wl.name, wl.sets, [scenes.Camera(**{**cam})], wl.blocks, wl.items, wl.tile)
    ctx = ctx_for(wl)
    batch = make_batch(wl)
    proj = lobe.project(ctx, batch)
    torch.cuda.synchronize()
    p = oracle.project(g, cam, wl.tile, margins=oracle.MARGINS_E2E)
    rad = proj.radius.cpu().numpy()
    s = proj.splat.cpu().numpy().astype(np.float64)
    check_projection_admissible(p, rad, s, proj.tiles.cpu().numpy(), cam, wl.tile)


def check_projection_admissible(p, rad, s, tiles, cam, tile, min_visible=500):
    """Radius, culling and tile count of every Gaussian: the oracle's, or (where its radius,
    rectangle or guard decision is marginal) a radius within one of it or culled; the splat
    values of every Gaussian the GPU keeps; the tile count of the GPU's own exact rectangle."""
    marg = oracle.marginal_rect(p) | oracle.marginal_visibility(p)
    np.testing.assert_array_equal(rad[~marg], p.radius[~marg])
    alt_ok = (rad == p.radius) | (rad == 0) | (np.abs(rad - p.radius_all) <= 1)
    assert np.all(alt_ok[marg]), "a marginal Gaussian's radius is outside the admissible set"
    vis = rad > 0
    assert vis.sum() > min_visible
    np.testing.assert_allclose(s[vis, 0:2], p.mean2d[vis], rtol=1e-5, atol=2e-4)
    np.testing.assert_allclose(s[vis, 2:5], p.conic[vis], rtol=2e-4, atol=1e-7)
    np.testing.assert_allclose(s[vis, 5], p.opacity[vis], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(np.abs(s[vis, 6:9]), p.color[vis], atol=2e-5)
    # depth key: float32 rounding of the double-precision z, bit for bit
    np.testing.assert_array_equal(s[vis, 9].astype(np.float32), p.depth[vis].astype(np.float32))
    np.testing.assert_array_equal(tiles, rect_tiles(s[:, 0:2], rad, cam, tile))
    ok = ~marg
    np.testing.assert_array_equal(tiles[ok], np.where(p.radius[ok] > 0, (p.rect[ok, 2] - p.rect[ok, 0]) *
                                                      (p.rect[ok, 3] - p.rect[ok, 1]), 0))


def test_project_multi_set_matches_oracle():
    """A batch of three sets whose sizes are not multiples of 32 (so warps span two sets and
    take the per-thread copies of their SH rows), one of them visibility-cropped, each seen by
    one or two views: every item's projection matches the oracle's as in the single-set case."""
    rng = np.random.default_rng(17)
    sets = [scenes.uniform_gaussians(rng, n, 1.0, 2.0, 6.0) for n in (1001, 777, 1500)]
    cams = [scenes.pinhole(128, 128, 128.0, cx=64.0, cy=64.0),
            scenes.pinhole(128, 128, 128.0, cx=64.0, cy=64.0,
                           viewmat=scenes.look_at((0.6, -0.4, -0.3), (0.0, 0.0, 4.0), up=(0, -1, 0)))]
    items = [(0, 0, -1), (0, 1, -1), (1, 0, -1), (2, 1, -1), (2, 0, -1)]
    crop = (rng.random(1500) < 0.6).astype(np.uint8)  # set 2: 40% cropped away
    wl = scenes.Workload("multi_set", sets, cams, [], items, (16, 16))
    gsets = [lobe.GaussianSet.from_numpy(x) for x in sets]
    gsets[2].crop_mask = dev(crop, torch.uint8)
    batch = lobe.Batch(gsets, wl.cameras, items, [])
    ctx = ctx_for(wl)
    proj = lobe.project(ctx, batch)
    torch.cuda.synchronize()
    rad_all = proj.radius.cpu().numpy()
    s_all = proj.splat.cpu().numpy().astype(np.float64)
    t_all = proj.tiles.cpu().numpy()
    for i, (si, ci, _) in enumerate(items):
        cam = cams[ci].as_dict()
        p = oracle.project(oracle.set_dict(sets[si]), cam, wl.tile, crop=crop if si == 2 else None,
                           margins=oracle.MARGINS_E2E)
        e0, n = batch.entry_off[i], sets[si].n
        rad, s, t = rad_all[e0:e0 + n], s_all[e0:e0 + n], t_all[e0:e0 + n]
        if si == 2:
            assert np.all(rad[crop == 0] == 0) and np.all(t[crop == 0] == 0)
        check_projection_admissible(p, rad, s, t, cam, wl.tile, min_visible=400)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_lower_sh_degrees_match_oracle(small, deg):
    """Active SH degree below 3: the colour uses the first (deg + 1)^2 bands only, and the
    adjoint writes zero gradients for the others."""
    wl, g = small
    cam = wl.cameras[0].as_dict()
    ctx = ctx_for(wl, sh_degree=deg)
    batch = make_batch(wl)
    proj = lobe.project(ctx, batch)
    p = oracle.project(g, cam, wl.tile, sh_degree=deg, margins=oracle.MARGINS_E2E)
    s = proj.splat.cpu().numpy().astype(np.float64)
    rad = proj.radius.cpu().numpy()
    ok = rad > 0
    assert ok.sum() > 500
    np.testing.assert_allclose(np.abs(s[ok, 6:9]), p.color[ok], atol=2e-5)
    f = oracle.forward(g, cam, wl.tile, sh_degree=deg)
    dL = np.random.default_rng(6).standard_normal((3, 128, 128))
    g2d = oracle.render_bwd(f.proj, f.ids, f.tile_start, cam, dL, wl.tile)
    g2d_r = oracle_grad2d_array(oracle.Grad2D(*(a.astype(np.float32).astype(np.float64) for a in
                                                (g2d.mean2d, g2d.conic, g2d.color, g2d.opacity))))
    env = param_envelope(g, cam, p, g2d_r, g2d_r, wl.tile, sh_degree=deg)
    grads = lobe.project_bwd(ctx, batch, proj, dev(g2d_r))
    nb = (deg + 1) ** 2
    gsh = grads[0]["sh"].cpu().numpy()
    assert_envelope(gsh[:, :nb], env["sh"][0][:, :nb], env["sh"][1][:, :nb], f"sh degree {deg}")
    assert np.all(gsh[:, nb:] == 0)
    assert_envelope(grads[0]["means"].cpu().numpy(), env["means"][0], env["means"][1], f"means sh degree {deg}")


# ----------------------------------------------------------------------------- bin + sort

@pytest.mark.parametrize("general", [False, True])  # the one-CTA path for small batches, and the general one
@pytest.mark.parametrize("tile", [(16, 16), (16, 8)])
def test_bin_sort_bit_exact_on_oracle_projection(small, tile, general):
    wl, g = small
    wl = scenes.Workload(wl.name, wl.sets, wl.cameras, wl.blocks, wl.items, tile)
    cam = wl.cameras[0].as_dict()
    p = oracle.project(g, cam, wl.tile).rounded()
    ids, ts = oracle.bin_sort(p, cam, wl.tile)
    ctx = ctx_for(wl, bin_general=general)
    batch = make_batch(wl)
    gp = gpu_projection_from_oracle(p, cam, wl.tile)
    bins = lobe.bin_sort(ctx, batch, gp)
    assert bins.count == len(ids)
    np.testing.assert_array_equal(bins.ids().cpu().numpy(), ids)
    np.testing.assert_array_equal(bins.tile_start.cpu().numpy(), ts)


def test_bin_sort_bit_exact_multi_item_large_tile_count():
    """Several items (global tile ids across items), 8x8 tiles (>65536 tiles => 3 radix passes),
    ragged image sizes; each item's pairs must equal the oracle's for that item."""
    rng = np.random.default_rng(11)
    g = scenes.uniform_gaussians(rng, 3000, 1.0, 2.0, 6.0)
    cams = [scenes.pinhole(1920, 1080, 1500.0), scenes.pinhole(1000, 750, 800.0), scenes.pinhole(333, 201, 260.0),
            scenes.pinhole(2048, 1536, 1600.0)]
    tile = (8, 8)
    wl = scenes.Workload("t", [g], cams, [scenes.AABB()], [(0, i, 0) for i in range(4)], tile)
    ctx = ctx_for(wl)
    batch = make_batch(wl)
    gd = oracle.set_dict(g)
    parts, want_ids, want_ts = [], [], []
    n_tiles, toffs = batch.tiles(tile)
    assert n_tiles > 65536
    off_e = 0
    total = 0
    for i, cam in enumerate(cams):
        p = oracle.project(gd, cam.as_dict(), tile).rounded()
        ids, ts = oracle.bin_sort(p, cam.as_dict(), tile)
        parts.append(p)
        want_ids.append(ids + off_e)
        want_ts.append(ts[:-1] + total)
        off_e += g.n
        total += len(ids)
    want_ts.append(np.array([total]))
    splat = np.concatenate([splat_array(p) for p in parts])
    rad = np.concatenate([p.radius for p in parts])
    tl = np.concatenate([rect_tiles(p.mean2d, p.radius, c, tile) for p, c in zip(parts, cams)])
    gp = lobe.Projection(dev(splat), dev(rad, torch.int32), dev(tl, torch.int32))
    bins = lobe.bin_sort(ctx, batch, gp)
    assert bins.count == total
    np.testing.assert_array_equal(bins.ids().cpu().numpy(), np.concatenate(want_ids))
    np.testing.assert_array_equal(bins.tile_start.cpu().numpy(), np.concatenate(want_ts))


def test_bin_sort_and_composite_at_the_batch_limits():
    """The largest batch one call takes: 16 views of 4096x4096 with 8x8 tiles, i.e. 2^22 tiles
    (the length of the tile scan) in 2^16 blocks of 64x64 pixels (the 16 bits of a super-tile
    id). Stage inputs (the oracle's float32 splats of 800 Gaussians a view): every item's lists
    bit-exact against the oracle's; on four 32x32 windows of every view (one around its
    longest list) every pixel of the composite matches an admissible result; the adjoint of a
    loss on the windows of the first and the last view in the oracle's envelope. One more block
    is an argument error, with nothing enqueued: the context then bins the limit batch again."""
    rng = np.random.default_rng(21)
    g = scenes.uniform_gaussians(rng, 800, 1.0, 2.0, 6.0)
    cams = [scenes.pinhole(4096, 4096, 2600.0 + 120.0 * i) for i in range(16)]
    tile = (8, 8)
    wl = scenes.Workload("limits", [g], cams, [scenes.AABB()], [(0, i, 0) for i in range(16)], tile)
    ctx = ctx_for(wl)
    batch = make_batch(wl)
    n_tiles, toffs = batch.tiles(tile)
    assert n_tiles == 1 << 22
    gd = oracle.set_dict(g)
    parts, ids_view, ts_view, want_ids, want_ts = [], [], [], [], []
    total = 0
    for i, cam in enumerate(cams):
        p = oracle.project(gd, cam.as_dict(), tile).rounded()
        ids, ts = oracle.bin_sort(p, cam.as_dict(), tile)
        parts.append(p)
        ids_view.append(ids)
        ts_view.append(ts)
        want_ids.append(ids + i * g.n)
        want_ts.append(ts[:-1] + total)
        total += len(ids)
    want_ts.append(np.array([total]))
    splat = np.concatenate([splat_array(p) for p in parts])
    rad = np.concatenate([p.radius for p in parts])
    tl = np.concatenate([rect_tiles(p.mean2d, p.radius, c, tile) for p, c in zip(parts, cams)])
    gp = lobe.Projection(dev(splat), dev(rad, torch.int32), dev(tl, torch.int32))
    bins = lobe.bin_sort(ctx, batch, gp)
    assert bins.count == total
    np.testing.assert_array_equal(bins.ids().cpu().numpy(), np.concatenate(want_ids))
    np.testing.assert_array_equal(bins.tile_start.cpu().numpy(), np.concatenate(want_ts))
    out = lobe.render_fwd(ctx, batch, gp, bins)
    rgbs = batch.image_views(out.rgb)
    Ts = batch.image_views(out.T_final, channels=1)
    ncs = batch.image_views(out.n_contrib, channels=1)
    win_rng = np.random.default_rng(22)
    ebs, wins, adms = [], [], []
    for i, cam in enumerate(cams):
        c = cam.as_dict()
        gx = -(-c["width"] // tile[0])
        t = int(np.argmax(np.diff(ts_view[i])))
        starts = [((t % gx) * tile[0] // 32 * 32, (t // gx) * tile[1] // 32 * 32)]
        while len(starts) < 4:  # disjoint 32x32 windows on a 32-pixel grid
            x, y = (int(v) * 32 for v in win_rng.integers(0, 4096 // 32, 2))
            if (x, y) not in starts:
                starts.append((x, y))
        eb = oracle.ExtBins(ids_view[i], np.zeros(len(ids_view[i]), np.uint8), ts_view[i])
        rgb = rgbs[i].view(3, 4096, 4096)
        T = Ts[i].view(4096, 4096)
        nc = ncs[i].view(4096, 4096)
        ebs.append(eb)
        wins.append([(x0, y0, x0 + 32, y0 + 32) for x0, y0 in starts])
        adms.append([])
        for w in wins[i]:
            x0, y0, x1, y1 = w
            lv = oracle.render_leaves(parts[i], eb, c, tile, margins=oracle.MARGINS_STAGE, win=w, certain=True)
            adms[i].append(match_image(lv, rgb[:, y0:y1, x0:x1].cpu().numpy(), T[y0:y1, x0:x1].cpu().numpy(),
                                       nc[y0:y1, x0:x1].cpu().numpy(), f"image view {i} at the batch limits (stage)"))
    # the adjoint with dL/dC nonzero on the windows of the first and the last view only: their
    # splats' 2D gradients in the oracle's envelope, every other entry's exactly zero
    dL = torch.zeros(3 * batch.n_pixels, dtype=torch.float32, device="cuda")
    dls = batch.image_views(dL)
    dl_rng = np.random.default_rng(23)
    dl64 = {}
    for i in (0, 15):
        d = np.zeros((3, 4096, 4096), np.float32)
        for x0, y0, x1, y1 in wins[i]:
            d[:, y0:y1, x0:x1] = dl_rng.standard_normal((3, y1 - y0, x1 - x0))
        dls[i].copy_(torch.as_tensor(d).reshape(dls[i].shape))
        dl64[i] = d.astype(np.float64)
    g2d = lobe.render_bwd(ctx, batch, gp, bins, out, dL).cpu().numpy()
    for i in (0, 15):
        lo = np.zeros((g.n, 12))
        hi = np.zeros((g.n, 12))
        for w, adm in zip(wins[i], adms[i]):
            l, h, _ = oracle.render_bwd_envelope(parts[i], ebs[i], cams[i].as_dict(), dl64[i], adm, tile,
                                                 margins=oracle.MARGINS_STAGE, win=w, certain=True)
            lo += l
            hi += h
        rows = g2d[i * g.n:(i + 1) * g.n]
        vis = parts[i].radius > 0
        for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                           ("color", slice(6, 9))]:
            assert_envelope(rows[vis, cols], lo[vis, cols], hi[vis, cols], f"grad2d {name} view {i} at the batch limits")
    assert np.all(g2d[g.n:15 * g.n] == 0)
    # one more 64x64-pixel block: rejected before anything is enqueued
    cams2 = cams + [scenes.pinhole(64, 64, 64.0)]
    wl2 = scenes.Workload("limits+1", [g], cams2, [scenes.AABB()], [(0, i, 0) for i in range(17)], tile)
    batch2 = make_batch(wl2)
    p17 = oracle.project(gd, cams2[16].as_dict(), tile).rounded()
    gp2 = lobe.Projection(dev(np.concatenate([splat, splat_array(p17)])),
                          dev(np.concatenate([rad, p17.radius]), torch.int32),
                          dev(np.concatenate([tl, rect_tiles(p17.mean2d, p17.radius, cams2[16], tile)]), torch.int32))
    with pytest.raises(lobe._abi.LobeError) as e:
        lobe.bin_sort(ctx, batch2, gp2)
    assert e.value.code == lobe._abi.ERR_ARG
    again = lobe.bin_sort(ctx, batch, gp)
    assert again.count == total
    np.testing.assert_array_equal(again.tile_start.cpu().numpy(), np.concatenate(want_ts))


# ----------------------------------------------------------------------------- render

def stage_inputs(wl, g, cam):
    p = oracle.project(g, cam, wl.tile).rounded()
    ids, ts = oracle.bin_sort(p, cam, wl.tile)
    return p, ids, ts


def test_small_batch_binning_equals_general_and_oracle():
    """Two sets, four items of ragged sizes, 16x8 tiles (a small batch): the one-CTA binning and
    the general multi-kernel binning give identical pairs, tile starts and counts, and every
    item's lists equal the oracle's for that item."""
    rng = np.random.default_rng(17)
    sets = [scenes.uniform_gaussians(rng, 900, 1.0, 2.0, 6.0), scenes.uniform_gaussians(rng, 700, 1.0, 2.0, 6.0)]
    cams = [scenes.pinhole(150, 97, 120.0), scenes.pinhole(64, 64, 60.0, cx=20.0),
            scenes.pinhole(101, 130, 100.0, viewmat=scenes.look_at((0.3, 0.2, -0.2), (0, 0, 4.0), up=(0, -1, 0)))]
    items = [(0, 0, -1), (1, 1, -1), (0, 2, -1), (1, 0, -1)]
    tile = (16, 8)
    wl = scenes.Workload("sb", sets, cams, [], items, tile)
    batch = make_batch(wl)
    assert batch.n_entries <= 4096 and batch.tiles(tile)[0] <= 4096
    got = []
    for general in (False, True):
        ctx = ctx_for(wl, bin_general=general)
        proj = lobe.project(ctx, batch)
        bins = lobe.bin_sort(ctx, batch, proj)
        got.append((bins.count, bins.ids().cpu().numpy(), bins.tile_start.cpu().numpy(), proj))
    assert got[0][0] == got[1][0]
    np.testing.assert_array_equal(got[0][1], got[1][1])
    np.testing.assert_array_equal(got[0][2], got[1][2])
    # per item against the oracle, on the GPU's own projection (exact integer rectangles)
    proj = got[0][3]
    sp, rad = proj.splat.cpu().numpy(), proj.radius.cpu().numpy()
    _, toffs = batch.tiles(tile)
    ids, ts = got[0][1], got[0][2]
    for i, (si, ci, _) in enumerate(items):
        e0 = batch.entry_off[i]
        n = sets[si].n
        cam = cams[ci].as_dict()
        pg = oracle.Projection(sp[e0:e0 + n, 0:2].astype(np.float64), sp[e0:e0 + n, 2:5].astype(np.float64),
                               sp[e0:e0 + n, 6:9].astype(np.float64), sp[e0:e0 + n, 5].astype(np.float64),
                               sp[e0:e0 + n, 9].astype(np.float64), rad[e0:e0 + n].copy(),
                               rect_of(sp[e0:e0 + n, 0:2], rad[e0:e0 + n], cam, tile), np.zeros(n, np.int32),
                               rad[e0:e0 + n].copy())
        want_ids, want_ts = oracle.bin_sort(pg, cam, tile)
        t0 = toffs[i]
        nt = len(want_ts) - 1
        for t in range(nt):
            a = ids[ts[t0 + t]:ts[t0 + t + 1]] - e0
            np.testing.assert_array_equal(a, want_ids[want_ts[t]:want_ts[t + 1]])


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8), (32, 16)])
def test_render_fwd_matches_oracle(small, tile, persistent):
    wl, g = small
    wl = scenes.Workload(wl.name, wl.sets, wl.cameras, wl.blocks, wl.items, tile)
    cam = wl.cameras[0].as_dict()
    p, ids, ts = stage_inputs(wl, g, cam)
    bg = (0.1, 0.2, 0.3)
    eb = oracle.ExtBins(ids, np.zeros(len(ids), np.uint8), ts)
    lv = oracle.render_leaves(p, eb, cam, tile, bg, oracle.MARGINS_STAGE, certain=True)
    ctx = ctx_for(wl, bg=bg, persistent=persistent)
    batch = make_batch(wl)
    gp = gpu_projection_from_oracle(p, cam, tile)
    bins = lobe.bin_sort(ctx, batch, gp)
    out = lobe.render_fwd(ctx, batch, gp, bins)
    rgb = out.rgb.view(3, 128, 128).cpu().numpy()
    T = out.T_final.view(128, 128).cpu().numpy()
    nc = out.n_contrib.view(128, 128).cpu().numpy()
    match_image(lv, rgb, T, nc, "image small (stage)")


@pytest.mark.parametrize("recompute, tile, px, persistent, nb", [
    (False, (16, 16), 0, False, 32), (True, (16, 16), 0, False, 32), (False, (16, 8), 1, False, 32),
    (False, (16, 8), 4, False, 32), (True, (16, 8), 4, False, 32), (False, (16, 8), 4, True, 32),
    (True, (8, 8), 1, True, 32), (False, (32, 16), 8, True, 32),
    # 64-splat staging rounds (two splats a lane)
    (False, (16, 8), 4, True, 64), (True, (16, 16), 2, False, 64), (False, (32, 16), 8, False, 64)])
def test_render_bwd_matches_oracle(small, recompute, tile, px, persistent, nb):
    wl, g = small
    wl = scenes.Workload(wl.name, wl.sets, wl.cameras, wl.blocks, wl.items, tile)
    cam = wl.cameras[0].as_dict()
    p, ids, ts = stage_inputs(wl, g, cam)
    bg = (0.1, 0.2, 0.3)
    eb = oracle.ExtBins(ids, np.zeros(len(ids), np.uint8), ts)
    lv = oracle.render_leaves(p, eb, cam, wl.tile, bg, oracle.MARGINS_STAGE, certain=True)
    dL = np.random.default_rng(3).standard_normal((3, 128, 128)).astype(np.float32).astype(np.float64)
    ctx = ctx_for(wl, bg=bg, recompute_T=recompute, px_fwd=px, px_bwd=px, persistent=persistent, batch=(nb, nb))
    batch = make_batch(wl)
    gp = gpu_projection_from_oracle(p, cam, wl.tile)
    bins = lobe.bin_sort(ctx, batch, gp)
    out = lobe.render_fwd(ctx, batch, gp, bins)
    adm = match_image(lv, out.rgb.view(3, 128, 128).cpu().numpy(), out.T_final.view(128, 128).cpu().numpy(),
                      out.n_contrib.view(128, 128).cpu().numpy(), "image small (stage, before the adjoint)")
    lo, hi, _ = oracle.render_bwd_envelope(p, eb, cam, dL, adm, wl.tile, bg, oracle.MARGINS_STAGE, certain=True)
    g2d = lobe.render_bwd(ctx, batch, gp, bins, out, dev(dL).reshape(-1)).cpu().numpy()
    vis = p.radius > 0
    for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                       ("color", slice(6, 9))]:
        assert_envelope(g2d[vis, cols], lo[vis, cols], hi[vis, cols], name)
    assert np.all(g2d[:, 9:] == 0)


def test_project_bwd_matches_oracle(small):
    wl, g = small
    cam = wl.cameras[0].as_dict()
    f = oracle.forward(g, cam, wl.tile)
    dL = np.random.default_rng(4).standard_normal((3, 128, 128))
    box = scenes.AABB((-0.5, -0.5, -math.inf), (0.5, 0.5, math.inf))
    g2d = oracle.render_bwd(f.proj, f.ids, f.tile_start, cam, dL, wl.tile)
    g2d_r = oracle_grad2d_array(oracle.Grad2D(*(a.astype(np.float32).astype(np.float64) for a in
                                                (g2d.mean2d, g2d.conic, g2d.color, g2d.opacity))))
    p = oracle.project(g, cam, wl.tile, margins=oracle.MARGINS_E2E)
    env = param_envelope(g, cam, p, g2d_r, g2d_r, wl.tile, aabb=box)
    ctx = ctx_for(wl)
    wl2 = scenes.Workload(wl.name, wl.sets, wl.cameras, [box], wl.items, wl.tile)
    batch = make_batch(wl2)
    proj = lobe.project(ctx, batch)
    grads = lobe.zero_grads(batch)
    lobe.project_bwd(ctx, batch, proj, dev(g2d_r), grads, accumulate=True)
    gr = {k: v.cpu().numpy() for k, v in grads[0].items()}
    assert (env["sd_cnt"][0] > 0).sum() > 50
    assert_params_in_envelope(gr, env, "project_bwd small (stage)")


@pytest.mark.parametrize("recompute", [False, True])
def test_end_to_end_small(small, recompute):
    wl, g = small
    cam = wl.cameras[0].as_dict()
    p = oracle.project(g, cam, wl.tile, margins=oracle.MARGINS_E2E)
    eb = oracle.bin_ext(p, cam, wl.tile)
    lv = oracle.render_leaves(p, eb, cam, wl.tile, margins=oracle.MARGINS_E2E)
    ctx = ctx_for(wl, recompute_T=recompute)
    batch = make_batch(wl)
    proj, bins, img = lobe.forward(ctx, batch)
    rgb = img.rgb.view(3, 128, 128).cpu().numpy()
    adm = match_image(lv, rgb, img.T_final.view(128, 128).cpu().numpy(), None, "image small (end to end)")
    # sort order: per tile the GPU's list is the oracle's, each uncertain member in or out
    gx, gy = oracle.grid(cam, wl.tile)
    check_lists_admissible(bins.ids().cpu().numpy(), bins.tile_start.cpu().numpy(), eb, range(gx * gy),
                           name="tile lists small (end to end)")
    dL = np.random.default_rng(5).standard_normal((3, 128, 128)).astype(np.float32).astype(np.float64)
    lo, hi, _ = oracle.render_bwd_envelope(p, eb, cam, dL, adm, wl.tile, margins=oracle.MARGINS_E2E)
    g2d = lobe.render_bwd(ctx, batch, proj, bins, img, dev(dL).reshape(-1))
    got2 = g2d.cpu().numpy()
    for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                       ("color", slice(6, 9))]:
        assert_envelope(got2[:, cols], lo[:, cols], hi[:, cols], name + " small (end to end)")
    env = param_envelope(g, cam, p, lo, hi, wl.tile)
    grads = lobe.project_bwd(ctx, batch, proj, g2d)
    gr = {k: v.cpu().numpy() for k, v in grads[0].items()}
    assert_params_in_envelope(gr, env, "small (end to end)")


def test_project_bwd_sums_views_like_oracle(small):
    """One set seen by two cameras: the GPU adjoint sums its per-view contributions in registers
    and counts the SD statistic per view; the oracle runs each view's adjoint and adds them."""
    wl, g = small
    cam0 = wl.cameras[0].as_dict()
    cam1 = dict(cam0, viewmat=scenes.look_at((0.7, -0.5, -0.6), (0.0, 0.0, 4.0), up=(0, -1, 0)))
    cams = [cam0, cam1]
    box = scenes.AABB((-0.6, -0.4, -math.inf), (0.5, 0.7, math.inf))
    wl2 = scenes.Workload(wl.name, wl.sets, [scenes.Camera(**c) for c in cams], [box], [(0, 0, 0), (0, 1, 0)],
                          wl.tile)
    env, g2ds = None, []
    for v, cam in enumerate(cams):
        f = oracle.forward(g, cam, wl.tile)
        dL = np.random.default_rng(10 + v).standard_normal((3, 128, 128))
        g2d = oracle.render_bwd(f.proj, f.ids, f.tile_start, cam, dL, wl.tile)
        g2d_r = oracle_grad2d_array(oracle.Grad2D(*(a.astype(np.float32).astype(np.float64) for a in
                                                    (g2d.mean2d, g2d.conic, g2d.color, g2d.opacity))))
        p = oracle.project(g, cam, wl.tile, margins=oracle.MARGINS_E2E)
        env = add_envelopes(env, param_envelope(g, cam, p, g2d_r, g2d_r, wl.tile, aabb=box))
        g2ds.append(g2d_r)
    ctx = ctx_for(wl2)
    batch = make_batch(wl2)
    proj = lobe.project(ctx, batch)
    grads = lobe.zero_grads(batch)
    lobe.project_bwd(ctx, batch, proj, dev(np.concatenate(g2ds)), grads, accumulate=True)
    gr = {k: v.cpu().numpy() for k, v in grads[0].items()}
    rad = proj.radius.cpu().numpy().reshape(2, -1)
    assert (rad > 0).any(axis=0).sum() > 500 and (rad > 0).all(axis=0).sum() > 100  # many seen by both views
    assert env["sd_cnt"][1].max() == 2
    assert_params_in_envelope(gr, env, "(two views)")


def test_persistent_compositing_equals_one_block_per_tile():
    """The persistent kernels (warps taking tiles longest list first from a device counter)
    render every item of a ragged multi-item batch bit for bit like one block per tile, and
    their adjoint sums the same per-splat gradients (float32 atomic order aside)."""
    rng = np.random.default_rng(41)
    sets = [scenes.uniform_gaussians(rng, 2500, 1.0, 2.0, 6.0), scenes.uniform_gaussians(rng, 1500, 1.0, 2.0, 6.0)]
    cams = [scenes.pinhole(300, 170, 240.0), scenes.pinhole(97, 131, 100.0),
            scenes.pinhole(256, 256, 220.0, viewmat=scenes.look_at((0.3, 0.2, -0.2), (0, 0, 4.0), up=(0, -1, 0)))]
    items = [(0, 0, -1), (1, 1, -1), (0, 2, -1), (1, 0, -1)]
    for tile, px in (((16, 8), (2, 4)), ((32, 16), (4, 8)), ((8, 8), (1, 1))):
        wl = scenes.Workload("p", sets, cams, [], items, tile)
        batch = make_batch(wl)
        dL = torch.as_tensor(np.random.default_rng(3).standard_normal(3 * batch.n_pixels), dtype=torch.float32).cuda()
        out = []
        for persistent in (False, True):
            ctx = ctx_for(wl, px_fwd=px[0], px_bwd=px[1], persistent=persistent)
            proj, bins, img = lobe.forward(ctx, batch)
            g2d = lobe.render_bwd(ctx, batch, proj, bins, img, dL)
            ctx.status()
            out.append((img, g2d))
        (a, ga), (b, gb) = out
        assert torch.equal(a.rgb, b.rgb) and torch.equal(a.T_final, b.T_final) and torch.equal(a.n_contrib, b.n_contrib)
        scale = float(ga.abs().max())
        assert float((ga - gb).abs().max()) <= 1e-5 * scale, tile


def test_staging_batch_does_not_change_results():
    """Staging 64 splats a round (two a lane) instead of 32 renders every item of a ragged
    multi-item batch bit for bit alike (the walk visits the same splats in the same order) and
    sums the same adjoint (float32 atomic order aside), for the forward of every pixels-per-lane
    count that allows it and both adjoint modes."""
    rng = np.random.default_rng(43)
    sets = [scenes.uniform_gaussians(rng, 3000, 1.0, 2.0, 6.0), scenes.uniform_gaussians(rng, 1200, 1.0, 2.0, 6.0)]
    cams = [scenes.pinhole(300, 170, 240.0), scenes.pinhole(97, 131, 100.0),
            scenes.pinhole(256, 256, 220.0, viewmat=scenes.look_at((0.3, 0.2, -0.2), (0, 0, 4.0), up=(0, -1, 0)))]
    items = [(0, 0, -1), (1, 1, -1), (0, 2, -1), (1, 0, -1)]
    for tile, px, persistent, recompute in (((16, 8), (2, 4), True, False), ((16, 16), (4, 2), False, True),
                                            ((32, 16), (8, 8), True, True), ((8, 8), (2, 2), False, False)):
        wl = scenes.Workload("nb", sets, cams, [], items, tile)
        batch = make_batch(wl)
        dL = torch.as_tensor(np.random.default_rng(5).standard_normal(3 * batch.n_pixels), dtype=torch.float32).cuda()
        out = []
        for nb in (32, 64):
            ctx = ctx_for(wl, px_fwd=px[0], px_bwd=px[1], persistent=persistent, recompute_T=recompute,
                          batch=(nb, nb))
            proj, bins, img = lobe.forward(ctx, batch)
            g2d = lobe.render_bwd(ctx, batch, proj, bins, img, dL)
            ctx.status()
            out.append((img, g2d))
        (a, ga), (b, gb) = out
        assert bins.count > 20000
        assert torch.equal(a.rgb, b.rgb) and torch.equal(a.T_final, b.T_final) and torch.equal(a.n_contrib, b.n_contrib)
        scale = float(ga.abs().max())
        assert float((ga - gb).abs().max()) <= 1e-5 * scale, tile


def test_batched_equals_plain():
    rng = np.random.default_rng(21)
    sets = [scenes.uniform_gaussians(rng, 800, 1.0, 2.0, 6.0), scenes.uniform_gaussians(rng, 500, 1.0, 2.0, 6.0)]
    cams = [scenes.pinhole(160, 120, 140.0), scenes.pinhole(100, 75, 90.0),
            scenes.pinhole(128, 128, 128.0, viewmat=scenes.look_at((0.3, 0.2, -0.2), (0, 0, 4.0), up=(0, -1, 0)))]
    items = [(0, 0, -1), (1, 1, -1), (0, 2, -1), (1, 0, -1)]
    wl = scenes.Workload("b", sets, cams, [], items, (16, 16))
    ctx = ctx_for(wl)
    batch = make_batch(wl)
    proj, bins, img = lobe.forward(ctx, batch)
    rgbs = batch.image_views(img.rgb)
    for i, it in enumerate(items):
        one = scenes.Workload("o", [sets[it[0]]], [cams[it[1]]], [], [(0, 0, -1)], (16, 16))
        b1 = make_batch(one)
        _, _, im1 = lobe.forward(ctx, b1)
        torch.testing.assert_close(rgbs[i], b1.image_views(im1.rgb)[0], rtol=0, atol=0)


def test_largest_batch_matches_single_item_runs():
    """The largest batch (16 sets, 64 items of uneven size): every item's image equals that
    item rendered alone, bit for bit, and the summed adjoint of each set equals the sum of its
    items' single-item adjoints within float32 summation order."""
    rng = np.random.default_rng(33)
    sets = [scenes.uniform_gaussians(rng, int(rng.integers(50, 400)), 1.0, 2.0, 6.0) for _ in range(16)]
    cams = [scenes.pinhole(72, 40, 60.0), scenes.pinhole(33, 65, 50.0), scenes.pinhole(48, 48, 45.0, cx=20.0),
            scenes.pinhole(64, 32, 70.0, viewmat=scenes.look_at((0.2, 0.1, -0.3), (0, 0, 4.0), up=(0, -1, 0)))]
    items = [(i % 16, (i // 16 + i) % 4, -1) for i in range(64)]
    wl = scenes.Workload("max", sets, cams, [], items, (16, 16))
    ctx = ctx_for(wl)
    batch = make_batch(wl)
    proj, bins, img = lobe.forward(ctx, batch)
    dL = torch.as_tensor(np.random.default_rng(2).standard_normal(3 * batch.n_pixels), dtype=torch.float32).cuda()
    g2d = lobe.render_bwd(ctx, batch, proj, bins, img, dL)
    grads = lobe.project_bwd(ctx, batch, proj, g2d)
    rgbs = batch.image_views(img.rgb)
    dls = batch.image_views(dL)
    summed = [{k: torch.zeros_like(v) for k, v in g.items()} for g in grads]
    for i, (si, ci, _) in enumerate(items):
        one = scenes.Workload("o", [sets[si]], [cams[ci]], [], [(0, 0, -1)], (16, 16))
        b1 = make_batch(one)
        p1, bn1, im1 = lobe.forward(ctx, b1)
        torch.testing.assert_close(rgbs[i], b1.image_views(im1.rgb)[0], rtol=0, atol=0)
        g1 = lobe.project_bwd(ctx, b1, p1, lobe.render_bwd(ctx, b1, p1, bn1, im1, dls[i].reshape(-1).contiguous()))
        for k in summed[si]:
            summed[si][k] += g1[0][k]
    for g, s in zip(grads, summed):
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            a, b = g[k].double(), s[k].double()
            assert float((a - b).abs().max()) <= 1e-4 * max(float(b.abs().max()), 1e-12), k


def test_visibility_crop_matches_oracle():
    wl = scenes.small_scene()
    # two oblique views that each see only part of the scene
    cams = [dict(wl.cameras[0].as_dict(), viewmat=scenes.look_at((-0.5, 0.0, 4.0), (5.0, 0.0, 4.0))),
            dict(wl.cameras[0].as_dict(), viewmat=scenes.look_at((0.0, -0.5, 4.0), (0.0, 5.0, 4.0)))]
    g = oracle.set_dict(wl.sets[0])
    want = oracle.visibility_crop(g, cams, wl.tile)
    w2 = scenes.Workload("v", wl.sets, [scenes.Camera(**c) for c in cams], [], [(0, 0, -1), (0, 1, -1)], wl.tile)
    ctx = ctx_for(w2)
    batch = make_batch(w2)
    m = lobe.visibility_crop(ctx, batch)[0].cpu().numpy()
    # per view: visible for sure, or a marginal culling decision (either outcome admissible)
    sure, maybe = np.zeros(len(want), bool), np.zeros(len(want), bool)
    for c in cams:
        p = oracle.project(g, c, wl.tile, margins=oracle.MARGINS_E2E)
        marg = oracle.marginal_visibility(p)
        sure |= (p.radius > 0) & ~marg
        maybe |= marg
    np.testing.assert_array_equal(want[sure], 1)
    np.testing.assert_array_equal(want[~sure & ~maybe], 0)
    np.testing.assert_array_equal(m[sure], 1)
    np.testing.assert_array_equal(m[~sure & ~maybe], 0)
    assert 0 < want.sum() < len(want)


def test_crop_mask_culls():
    wl = scenes.small_scene(n=300)
    crop = (np.arange(300) % 3 != 0).astype(np.uint8)
    ctx = ctx_for(wl)
    batch = make_batch(wl, crop=crop)
    proj = lobe.project(ctx, batch)
    r = proj.radius.cpu().numpy()
    assert np.all(r[crop == 0] == 0)
    g = oracle.set_dict(wl.sets[0])
    p = oracle.project(g, wl.cameras[0].as_dict(), wl.tile, crop=crop)
    np.testing.assert_array_equal(r > 0, p.radius > 0)


# ----------------------------------------------------------------------------- edge cases

@pytest.mark.parametrize("tile, px, persistent", [((16, 16), 0, False), ((16, 8), 4, True), ((32, 16), 8, False),
                                                  ((8, 8), 1, True)])
def test_views_smaller_than_a_tile(tile, px, persistent):
    """One batch of views smaller than a tile, or one pixel wide or high (1x1, 3x2, 15x9, 17x1,
    1x33, 40x7), every one with deep lists (300 Gaussians of about two pixels): lists bit-exact,
    every pixel of every view's composite, and the adjoint's 2D gradients against the oracle
    (stage inputs)."""
    rng = np.random.default_rng(31)
    g = scenes.uniform_gaussians(rng, 300, 1.0, 2.0, 6.0)
    sizes = [(1, 1), (3, 2), (15, 9), (17, 1), (1, 33), (40, 7)]
    cams = [scenes.pinhole(w, h, float(w), float(h)) for w, h in sizes]  # a field of view of about 53 degrees
    bg = (0.1, 0.2, 0.3)
    wl = scenes.Workload("tiny", [g], cams, [scenes.AABB()], [(0, i, 0) for i in range(len(cams))], tile)
    ctx = ctx_for(wl, bg=bg, px_fwd=px, px_bwd=px, persistent=persistent)
    batch = make_batch(wl)
    gd = oracle.set_dict(g)
    parts, ebs, want_ids, want_ts = [], [], [], []
    total = 0
    for i, cam in enumerate(cams):
        p = oracle.project(gd, cam.as_dict(), tile).rounded()
        ids, ts = oracle.bin_sort(p, cam.as_dict(), tile)
        parts.append(p)
        ebs.append(oracle.ExtBins(ids, np.zeros(len(ids), np.uint8), ts))
        want_ids.append(ids + i * g.n)
        want_ts.append(ts[:-1] + total)
        total += len(ids)
    want_ts.append(np.array([total]))
    assert min(np.diff(eb.tile_start).max() for eb in ebs) >= 20  # every view has a deep list
    gp = lobe.Projection(dev(np.concatenate([splat_array(p) for p in parts])),
                         dev(np.concatenate([p.radius for p in parts]), torch.int32),
                         dev(np.concatenate([rect_tiles(p.mean2d, p.radius, c, tile) for p, c in zip(parts, cams)]),
                             torch.int32))
    bins = lobe.bin_sort(ctx, batch, gp)
    assert bins.count == total
    np.testing.assert_array_equal(bins.ids().cpu().numpy(), np.concatenate(want_ids))
    np.testing.assert_array_equal(bins.tile_start.cpu().numpy(), np.concatenate(want_ts))
    out = lobe.render_fwd(ctx, batch, gp, bins)
    rgbs, Ts = batch.image_views(out.rgb), batch.image_views(out.T_final, channels=1)
    ncs = batch.image_views(out.n_contrib, channels=1)
    dl_rng = np.random.default_rng(32)
    dL = torch.zeros(3 * batch.n_pixels, dtype=torch.float32, device="cuda")
    dls, dl64, adms = batch.image_views(dL), [], []
    for i, cam in enumerate(cams):
        c = cam.as_dict()
        lv = oracle.render_leaves(parts[i], ebs[i], c, tile, bg, oracle.MARGINS_STAGE, certain=True)
        adms.append(match_image(lv, rgbs[i].cpu().numpy(), Ts[i].cpu().numpy(), ncs[i].cpu().numpy(),
                                f"image {c['width']}x{c['height']} (stage, tile {tile[0]}x{tile[1]})"))
        d = dl_rng.standard_normal((3, c["height"], c["width"])).astype(np.float32)
        dls[i].copy_(torch.as_tensor(d))
        dl64.append(d.astype(np.float64))
    g2d = lobe.render_bwd(ctx, batch, gp, bins, out, dL).cpu().numpy()
    for i, cam in enumerate(cams):
        c = cam.as_dict()
        lo, hi, _ = oracle.render_bwd_envelope(parts[i], ebs[i], c, dl64[i], adms[i], tile, bg, oracle.MARGINS_STAGE,
                                               certain=True)
        rows = g2d[i * g.n:(i + 1) * g.n]
        vis = parts[i].radius > 0
        for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                           ("color", slice(6, 9))]:
            assert_envelope(rows[vis, cols], lo[vis, cols], hi[vis, cols],
                            f"grad2d {name} {c['width']}x{c['height']} (stage, tile {tile[0]}x{tile[1]})")
        assert np.all(rows[:, 9:] == 0)


@pytest.mark.parametrize("tile, px", [((16, 16), 0), ((16, 8), 4), ((32, 16), 8), ((8, 8), 1), ((16, 16), 2)])
def test_needle_gaussians_match_oracle(tile, px):
    """Needle-like Gaussians (two log-scales at -6.5, one in [-2, -1], random orientations:
    thin splats at every angle, a median axis ratio of 11.5, radii up to 77 px) whose 3-sigma
    squares hold many pixels far from the ellipse: the slab test that lets a warp skip a splat
    must never skip one that reaches a pixel. Every pixel of the composite and the adjoint's
    2D gradients against the oracle (stage inputs). A needle's conic gradient sums per-pixel
    terms that cancel (their magnitudes add up to 3000 times the result), so the envelope is
    widened by the stage margin of the float32 terms (STAGE_TERM_REL of that sum)."""
    rng = np.random.default_rng(41)
    n = 400
    g = scenes.uniform_gaussians(rng, n, 1.2, 2.0, 6.0)
    ls = np.full((n, 3), -6.5, np.float32)
    ls[np.arange(n), rng.integers(0, 3, n)] = rng.uniform(-2.0, -1.0, n)
    g = scenes.GaussianSet(g.means, ls, g.quats, (g.opacity_logits + 1.5).astype(np.float32), g.sh)
    cam = scenes.pinhole(160, 120, 140.0)
    wl = scenes.Workload("needles", [g], [cam], [scenes.AABB()], [(0, 0, 0)], tile)
    c = cam.as_dict()
    p, ids, ts = stage_inputs(wl, oracle.set_dict(g), c)
    bg = (0.1, 0.2, 0.3)
    eb = oracle.ExtBins(ids, np.zeros(len(ids), np.uint8), ts)
    lv = oracle.render_leaves(p, eb, c, tile, bg, oracle.MARGINS_STAGE, certain=True)
    ctx = ctx_for(wl, bg=bg, px_fwd=px, px_bwd=px)
    batch = make_batch(wl)
    gp = gpu_projection_from_oracle(p, c, tile)
    bins = lobe.bin_sort(ctx, batch, gp)
    np.testing.assert_array_equal(bins.ids().cpu().numpy(), ids)
    out = lobe.render_fwd(ctx, batch, gp, bins)
    adm = match_image(lv, out.rgb.view(3, 120, 160).cpu().numpy(), out.T_final.view(120, 160).cpu().numpy(),
                      out.n_contrib.view(120, 160).cpu().numpy(), f"image needles (stage, tile {tile[0]}x{tile[1]})")
    dL = np.random.default_rng(42).standard_normal((3, 120, 160)).astype(np.float32).astype(np.float64)
    lo, hi, ab = oracle.render_bwd_envelope(p, eb, c, dL, adm, tile, bg, oracle.MARGINS_STAGE, certain=True)
    lo -= STAGE_TERM_REL * ab
    hi += STAGE_TERM_REL * ab
    g2d = lobe.render_bwd(ctx, batch, gp, bins, out, dev(dL).reshape(-1)).cpu().numpy()
    vis = p.radius > 0
    for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                       ("color", slice(6, 9))]:
        assert_envelope(g2d[vis, cols], lo[vis, cols], hi[vis, cols],
                        f"grad2d {name} needles (stage, tile {tile[0]}x{tile[1]})")


def test_contexts_on_concurrent_threads_and_streams():
    """Three host threads, each with its own context on its own stream, run projection,
    binning (two of them the general path: look-back scans and the onesweep depth sort; one
    the one-CTA path of small batches), the composite and its adjoint on different batches ten
    times at the same time. Contexts share nothing (look-back counters, status words,
    scratch), so every image equals a lone run's bit for bit (the composite is deterministic)
    and the 2D gradients agree within the float32 atomic-order bound."""
    import threading

    def workload(seed, n, w, h):
        wl = scenes.small_scene(seed=seed, n=n)
        cam = scenes.pinhole(w, h, 0.9 * w)
        return scenes.Workload(wl.name, wl.sets, [cam], wl.blocks, wl.items, (16, 16))

    wls = [workload(0, 20000, 512, 384), workload(1, 30000, 320, 240), workload(2, 1000, 128, 96)]
    general = [True, True, False]

    def run(i, stream, reps, out):
        wl = wls[i]
        with torch.cuda.stream(stream):
            ctx = lobe.Context(tile=wl.tile, stream=stream, bin_general=general[i])
            batch = make_batch(wl)
            g = torch.Generator(device="cuda").manual_seed(5)
            dL = torch.randn(3 * batch.n_pixels, generator=g, device="cuda")
            res = []
            for _ in range(reps):
                proj, bins, img = lobe.forward(ctx, batch)
                g2d = lobe.render_bwd(ctx, batch, proj, bins, img, dL)
                res.append((img.rgb.clone(), img.T_final.clone(), img.n_contrib.clone(), g2d.clone()))
            stream.synchronize()
            ctx.status()
            out.extend(res)

    alone = []
    for i in range(len(wls)):
        r = []
        run(i, torch.cuda.Stream(), 1, r)
        alone.append(r[0])
    outs = [[] for _ in wls]
    errs = []

    def worker(i):
        try:
            run(i, torch.cuda.Stream(), 10, outs[i])
        except Exception as ex:  # reported below, in the main thread
            errs.append(ex)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(wls))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads) and not errs, errs
    for i in range(len(wls)):
        rgb0, T0, nc0, g0 = alone[i]
        assert len(outs[i]) == 10
        for rgb, T, nc, g2d in outs[i]:
            assert torch.equal(rgb, rgb0) and torch.equal(T, T0) and torch.equal(nc, nc0)
            assert grad_rel_err(g2d.cpu().numpy(), g0.cpu().numpy()) <= 1e-4


def test_empty_set_and_all_culled():
    empty = scenes.uniform_gaussians(np.random.default_rng(0), 0, 1.0, 2.0, 6.0)
    behind = scenes.uniform_gaussians(np.random.default_rng(1), 200, 1.0, -6.0, -2.0)
    cam = scenes.pinhole(64, 48, 60.0)
    for gs in (empty, behind):
        wl = scenes.Workload("e", [gs], [cam], [], [(0, 0, -1)], (16, 16))
        ctx = ctx_for(wl, bg=(0.25, 0.5, 0.75))
        batch = make_batch(wl)
        proj, bins, img = lobe.forward(ctx, batch)
        assert bins.count == 0
        rgb = img.rgb.view(3, 48, 64).cpu()
        for c, v in enumerate((0.25, 0.5, 0.75)):
            assert torch.all(rgb[c] == v)
        assert torch.all(img.T_final == 1.0) and torch.all(img.n_contrib == 0)
        dL = torch.ones(3 * 48 * 64, device="cuda")
        g2d = lobe.render_bwd(ctx, batch, proj, bins, img, dL)
        grads = lobe.project_bwd(ctx, batch, proj, g2d)
        for v in grads[0].values():
            assert torch.all(v == 0)


def test_ragged_image_matches_oracle():
    rng = np.random.default_rng(7)
    g = scenes.uniform_gaussians(rng, 600, 1.0, 2.0, 6.0)
    cam = scenes.pinhole(100, 75, 90.0, cx=50.0, cy=37.5)
    wl = scenes.Workload("r", [g], [cam], [], [(0, 0, -1)], (16, 16))
    gd = oracle.set_dict(g)
    c = cam.as_dict()
    p = oracle.project(gd, c, wl.tile, margins=oracle.MARGINS_E2E)
    eb = oracle.bin_ext(p, c, wl.tile)
    lv = oracle.render_leaves(p, eb, c, wl.tile, margins=oracle.MARGINS_E2E)
    ctx = ctx_for(wl)
    batch = make_batch(wl)
    _, _, img = lobe.forward(ctx, batch)
    match_image(lv, img.rgb.view(3, 75, 100).cpu().numpy(), img.T_final.view(75, 100).cpu().numpy(), None,
                "image ragged (end to end)")


@pytest.mark.parametrize("general", [False, True])
def test_capacity_overflow_is_reported_without_sync(general):
    wl = scenes.small_scene()
    ctx = ctx_for(wl, bin_general=general)
    batch = make_batch(wl)
    proj = lobe.project(ctx, batch)
    ctx.reserve(batch.n_entries, 1 << 16, batch.tiles(wl.tile)[0])
    n_tiles, _ = batch.tiles(wl.tile)
    small_bins = lobe.raster.empty_bins(100, n_tiles)
    lobe.bin_sort(ctx, batch, proj, small_bins, sync=False)
    with pytest.raises(lobe._abi.LobeError) as e:
        ctx.status()
    assert e.value.code == lobe._abi.ERR_CAPACITY
    # the bins then describe empty tiles, and the context stays usable
    assert int(small_bins.tile_start.max().item()) == 0
    ctx.status()
