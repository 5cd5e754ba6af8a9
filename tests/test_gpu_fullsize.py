"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot composite whole 1600x1066 / 1920x1080 views in seconds, so it renders
sampled windows of pixels (every Gaussian projected, only the windows' tiles binned and
composited) and the comparison runs on those:
- end to end (GPU projection -> GPU bins -> GPU image vs the FP64 oracle): per-tile lists of
  the windows' tiles, bit-exact once the few Gaussians whose tile rectangles came out
  differently in float32 are removed, and pixel values, max-abs 1e-4;
- the composite adjoint, with dL/dC nonzero only inside the windows (its adjoint is exactly
  the oracle's windowed backward), on the GPU's own float32 splats: per-splat 2D gradients,
  relative 1e-3 of each float32 sum, floored at 1e-3 of the sum of its terms' magnitudes;
- the projection adjoint fed the oracle's 2D gradients: every parameter gradient, relative 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import IMG_ATOL, differing_rects, grad_rel_err, oracle_grad2d_array, rect_of, record, sum_rel_err

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe


def windows_of(cam, n=3, size=32, seed=0):
    rng = np.random.default_rng(seed)
    W, H = cam["width"], cam["height"]
    out = []
    for _ in range(n):
        x0 = int(rng.integers(0, (W - size) // 16)) * 16
        y0 = int(rng.integers(0, (H - size) // 16)) * 16
        out.append((x0, y0, x0 + size, y0 + size))
    return out


def only_differing(p, diff):
    """The projection with the rectangle flag kept only on Gaussians whose rectangles differ."""
    q = oracle.Projection(p.mean2d, p.conic, p.color, p.opacity, p.depth, p.radius, p.rect,
                          np.where(diff, oracle.F_RECT, 0).astype(np.int32), p.radius_all)
    return q


def check_item(g64, cam, tile, gpu_rgb, gpu_ids, gpu_ts, tile_off, entry_off, wins, gpu_splat, gpu_radius, crop=None):
    """Compare one item's windows against the oracle. Returns (oracle projection, pixel
    flags of the windows, pixels compared)."""
    W, H = cam["width"], cam["height"]
    p = oracle.project(g64, cam, tile, crop=crop, margins=oracle.MARGINS_E2E)
    marg = differing_rects(p, gpu_splat[:, 0:2], gpu_radius, cam, tile)
    assert marg.mean() < 1e-3
    pm = only_differing(p, marg)
    gx = (W + tile[0] - 1) // tile[0]
    compared = 0
    pxf_all = np.zeros((H, W), np.int32)
    for (x0, y0, x1, y1) in wins:
        with oracle.window(x0, y0, x1, y1):
            ids, ts = oracle.bin_sort(p, cam, tile)
            pxf = oracle.flag_pixels(pm, cam, tile)
            img = oracle.render_fwd(p, ids, ts, cam, tile, (0, 0, 0), oracle.MARGINS_E2E, pxf)
        pxf_all |= img.flags
        for ty in range(y0 // tile[1], (y1 + tile[1] - 1) // tile[1]):
            for tx in range(x0 // tile[0], (x1 + tile[0] - 1) // tile[0]):
                t = ty * gx + tx
                a = gpu_ids[gpu_ts[tile_off + t]:gpu_ts[tile_off + t + 1]] - entry_off
                b = ids[ts[t]:ts[t + 1]]
                np.testing.assert_array_equal(a[~marg[a]], b[~marg[b]])
        ok = img.flags[y0:y1, x0:x1] == 0
        assert ok.mean() > 0.9
        d = np.abs(gpu_rgb[:, y0:y1, x0:x1] - img.rgb[:, y0:y1, x0:x1])[:, ok]
        record(f"image full size {cam['width']}x{cam['height']}", d.max())
        assert d.max() <= IMG_ATOL, d.max()
        compared += int(ok.sum())
    return p, marg, pxf_all, compared


def windowed_backward(g64, cam, tile, p, dL, wins, crop=None, aabb=None):
    total = None
    for (x0, y0, x1, y1) in wins:
        with oracle.window(x0, y0, x1, y1):
            ids, ts = oracle.bin_sort(p, cam, tile)
            g2d = oracle.render_bwd(p, ids, ts, cam, dL, tile)
        if total is None:
            total = g2d
        else:
            for k in ("mean2d", "conic", "color", "opacity"):
                getattr(total, k)[...] += getattr(g2d, k)
    return oracle.project_bwd(g64, cam, total, tile, crop=crop, aabb=aabb)


def sparse_dL(cam, wins, pixel_ok, seed=3):
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(seed)
    dL = np.zeros((3, H, W), np.float32)
    for (x0, y0, x1, y1) in wins:
        dL[:, y0:y1, x0:x1] = rng.standard_normal((3, y1 - y0, x1 - x0))
    return dL * pixel_ok[None]


def run_single(wl, crop=None, n_win=3, tile=None, px=(0, 0)):
    g = wl.sets[0]
    cam = wl.cameras[0].as_dict()
    tile = tuple(tile or wl.tile)
    sets = [lobe.GaussianSet.from_numpy(g)]
    if crop is not None:
        sets[0].crop_mask = torch.as_tensor(crop).cuda()
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=tile, px_fwd=px[0], px_bwd=px[1])
    proj, bins, img = lobe.forward(ctx, batch)
    rgb = img.rgb.view(3, cam["height"], cam["width"]).cpu().numpy()
    g64 = oracle.set_dict(g)
    wins = windows_of(cam, n_win)
    p, marg, pxf, n = check_item(g64, cam, tile, rgb, bins.ids().cpu().numpy(), bins.tile_start.cpu().numpy(), 0, 0,
                                 wins, proj.splat.cpu().numpy(), proj.radius.cpu().numpy(), crop=crop)
    assert n > 0.9 * n_win * 32 * 32
    # gradients from a dL/dC that is nonzero only on the windows' unflagged pixels
    aabb = wl.blocks[0] if wl.blocks else None
    # composite adjoint at full size, on the GPU's own float32 splats (the oracle composites and
    # differentiates the same splats in FP64): per-splat 2D gradients, each a float32 sum over
    # up to thousands of pixels
    sp = proj.splat.cpu().numpy().astype(np.float64)
    rad = proj.radius.cpu().numpy()
    pg = oracle.Projection(sp[:, 0:2].copy(), sp[:, 2:5].copy(), sp[:, 6:9].copy(), sp[:, 5].copy(),
                           sp[:, 9].copy(), rad.copy(), rect_of(sp[:, 0:2], rad, cam, tile), np.zeros_like(rad),
                           rad.copy())
    pxf_s = np.zeros_like(pxf)
    for (x0, y0, x1, y1) in wins:
        with oracle.window(x0, y0, x1, y1):
            ids, ts = oracle.bin_sort(pg, cam, tile)
            pxf_s |= oracle.render_fwd(pg, ids, ts, cam, tile, (0, 0, 0), oracle.MARGINS_STAGE).flags
    dL = sparse_dL(cam, wins, (pxf == 0) & (pxf_s == 0))
    with oracle.abs_sums(g.n) as A:
        tot = None
        for (x0, y0, x1, y1) in wins:
            with oracle.window(x0, y0, x1, y1):
                ids, ts = oracle.bin_sort(pg, cam, tile)
                g2 = oracle.render_bwd(pg, ids, ts, cam, dL.astype(np.float64), tile)
            tot = g2 if tot is None else oracle.Grad2D(tot.mean2d + g2.mean2d, tot.conic + g2.conic,
                                                       tot.color + g2.color, tot.opacity + g2.opacity)
    want2 = oracle_grad2d_array(tot)
    g2d = lobe.render_bwd(ctx, batch, proj, bins, img, torch.as_tensor(dL).cuda().reshape(-1))
    ok = ~marg & ((p.flags & oracle.F_COLOR) == 0) & (p.radius > 0)
    got2 = g2d.cpu().numpy()
    assert (np.abs(want2[ok, :9]).sum(1) > 0).sum() > 50
    for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                       ("color", slice(6, 9))]:
        err = sum_rel_err(got2[ok, cols], want2[ok, cols], A.a[ok, cols])
        record(f"grad2d sum rel {name} full size {cam['width']}x{cam['height']}", err)
        assert err <= 1e-3, (name, err)
    # projection adjoint at full size, fed the oracle's 2D gradients
    want = oracle.project_bwd(g64, cam, tot, tile, crop=crop, aabb=aabb)
    grads = lobe.project_bwd(ctx, batch, proj, torch.as_tensor(want2, dtype=torch.float32).cuda())
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        err = grad_rel_err(grads[0][k].cpu().numpy()[ok], getattr(want, k)[ok])
        record(f"grad rel {k} full size {cam['width']}x{cam['height']}", err)
        assert err <= 1e-3, (k, err)


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
    want = oracle.visibility_crop(g64, [wl.cameras[0].as_dict()], wl.tile)
    flags = oracle.project(g64, wl.cameras[0].as_dict(), wl.tile, margins=oracle.MARGINS_E2E).flags
    ok = (flags & (oracle.F_GUARD | oracle.F_RECT | oracle.F_RADIUS)) == 0
    np.testing.assert_array_equal(crop[ok], want[ok])
    assert 0.05 < want.mean() < 0.95
    run_single(wl, crop=crop, tile=tile, px=px)


def test_fullsize_multi_block_batched_graph_items():
    """The batched multi-block step (graph-captured, autotuned tile) checked item by item on
    sampled windows of two of its views (the smallest and the largest block)."""
    from paper_2510_01767_b300.batched import autotune
    wl = scenes.multi_block_scene(seed=0)
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    st, _ = autotune(sets, cams, wl.items, wl.blocks, reps=2, use_cache=False)
    st.replay()
    torch.cuda.synchronize()
    tile = st.tile
    ids = st.bins.ids().cpu().numpy() if st.bins.count is not None else \
        st.bins.gauss_ids[:int(st.bins.n_isect.item())].cpu().numpy()
    ts = st.bins.tile_start.cpu().numpy()
    _, toffs = st.batch.tiles(tile)
    views = st.images()
    splat = st.proj.splat.cpu().numpy()
    radius = st.proj.radius.cpu().numpy()
    for i in (0, len(wl.items) - 1):
        s, c, b = wl.items[i]
        cam = cams[c]
        g64 = oracle.set_dict(wl.sets[s])
        wins = windows_of(cam, 2, seed=i)
        e0, n = st.batch.entry_off[i], wl.sets[s].n
        check_item(g64, cam, tile, views[i].cpu().numpy(), ids, ts, toffs[i], e0, wins, splat[e0:e0 + n],
                   radius[e0:e0 + n])
