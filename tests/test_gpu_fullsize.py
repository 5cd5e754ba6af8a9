"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot composite whole 1600x1066 / 1920x1080 views in seconds, so it renders
sampled windows of pixels (every Gaussian projected, only the windows' tiles binned and
composited) and the comparison runs on those: per-tile lists of the windows' tiles
(bit-exact once marginal Gaussians are removed), pixel values (max-abs 1e-4), and -- with
dL/dC nonzero only inside the windows -- every parameter gradient (relative 1e-3), since the
adjoint of a sparse dL/dC is exactly the oracle's windowed backward.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import IMG_ATOL, grad_rel_err

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


def check_item(g64, cam, tile, gpu_rgb, gpu_ids, gpu_ts, tile_off, entry_off, wins, grads_gpu=None, crop=None,
               aabb=None, dL_full=None):
    """Compare one item's windows against the oracle. Returns pixels compared."""
    W, H = cam["width"], cam["height"]
    p = oracle.project(g64, cam, tile, crop=crop, margins=oracle.MARGINS_E2E)
    marg = (p.flags & (oracle.F_GUARD | oracle.F_RADIUS | oracle.F_RECT)) != 0
    gx = (W + tile[0] - 1) // tile[0]
    compared = 0
    for (x0, y0, x1, y1) in wins:
        with oracle.window(x0, y0, x1, y1):
            ids, ts = oracle.bin_sort(p, cam, tile)
            pxf = oracle.flag_pixels(p, cam, tile)
            img = oracle.render_fwd(p, ids, ts, cam, tile, (0, 0, 0), oracle.MARGINS_E2E, pxf)
        for ty in range(y0 // tile[1], (y1 + tile[1] - 1) // tile[1]):
            for tx in range(x0 // tile[0], (x1 + tile[0] - 1) // tile[0]):
                t = ty * gx + tx
                a = gpu_ids[gpu_ts[tile_off + t]:gpu_ts[tile_off + t + 1]] - entry_off
                b = ids[ts[t]:ts[t + 1]]
                np.testing.assert_array_equal(a[~marg[a]], b[~marg[b]])
        ok = img.flags[y0:y1, x0:x1] == 0
        assert ok.mean() > 0.9
        d = np.abs(gpu_rgb[:, y0:y1, x0:x1] - img.rgb[:, y0:y1, x0:x1])[:, ok]
        assert d.max() <= IMG_ATOL, d.max()
        compared += int(ok.sum())
    return p, compared


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


def run_single(wl, crop=None, n_win=3):
    g = wl.sets[0]
    cam = wl.cameras[0].as_dict()
    tile = wl.tile
    sets = [lobe.GaussianSet.from_numpy(g)]
    if crop is not None:
        sets[0].crop_mask = torch.as_tensor(crop).cuda()
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=tile)  # default pixels per lane, as in bench.py
    proj, bins, img = lobe.forward(ctx, batch)
    rgb = img.rgb.view(3, cam["height"], cam["width"]).cpu().numpy()
    g64 = oracle.set_dict(g)
    wins = windows_of(cam, n_win)
    p, n = check_item(g64, cam, tile, rgb, bins.ids().cpu().numpy(), bins.tile_start.cpu().numpy(), 0, 0, wins,
                      crop=crop)
    assert n > 0.9 * n_win * 32 * 32
    # gradients from a dL/dC that is nonzero only on the windows' unflagged pixels
    pxf = np.zeros((cam["height"], cam["width"]), np.int32)
    for (x0, y0, x1, y1) in wins:
        with oracle.window(x0, y0, x1, y1):
            ids, ts = oracle.bin_sort(p, cam, tile)
            pxf |= oracle.render_fwd(p, ids, ts, cam, tile, (0, 0, 0), oracle.MARGINS_E2E,
                                     oracle.flag_pixels(p, cam, tile)).flags
    dL = sparse_dL(cam, wins, pxf == 0)
    aabb = wl.blocks[0] if wl.blocks else None
    want = windowed_backward(g64, cam, tile, p, dL.astype(np.float64), wins, crop=crop, aabb=aabb)
    g2d = lobe.render_bwd(ctx, batch, proj, bins, img, torch.as_tensor(dL).cuda().reshape(-1))
    grads = lobe.project_bwd(ctx, batch, proj, g2d)
    ok = (p.flags == 0) & (p.radius > 0)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        err = grad_rel_err(grads[0][k].cpu().numpy()[ok], getattr(want, k)[ok])
        assert err <= 1e-3, (k, err)


def test_fullsize_medium_200k_1600x1066():
    run_single(scenes.medium_scene())


def test_fullsize_city_block_with_visibility_crop():
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
    run_single(wl, crop=crop)


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
    for i in (0, len(wl.items) - 1):
        s, c, b = wl.items[i]
        cam = cams[c]
        g64 = oracle.set_dict(wl.sets[s])
        wins = windows_of(cam, 2, seed=i)
        check_item(g64, cam, tile, views[i].cpu().numpy(), ids, ts, toffs[i], st.batch.entry_off[i], wins)
