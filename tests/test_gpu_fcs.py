"""Fast camera selection (Sec. 3.2) on the GPU against the FP64 oracle: the composite depth
channel, the back-projection and block counts, and the camera-to-block assignment.

The depth map is compared stage-wise (the oracle's float32-rounded splats on both sides) and
end to end, with a tolerance of 1e-4 relative to the scene's largest depth (the image bar
scaled to depth units): every pixel must match one of the oracle's admissible composites
(every outcome of a decision float32 may take either way). The counts are compared on the
GPU's own depth map, exactly, except for points the oracle flags as lying within float32
reach of a box face, whose count may go either way.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import scenes
from tests.helpers import match_image, rect_tiles, resolve_membership, splat_array

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe

DEPTH_RTOL = 1e-4
FACE_MARGIN = 1e-5


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def depth_projection(p):
    """The projection with each splat's depth as its three colour channels: the depth channel
    of Sec. 3.2 composites exactly like a colour."""
    return oracle.Projection(p.mean2d, p.conic, np.repeat(p.depth[:, None], 3, axis=1), p.opacity, p.depth,
                             p.radius, p.rect, p.flags, p.radius_all, p.color_raw)


def test_depth_channel_stage_matches_oracle():
    wl = scenes.small_scene()
    cam = wl.cameras[0].as_dict()
    g = oracle.set_dict(wl.sets[0])
    p = oracle.project(g, cam, wl.tile).rounded()
    ids, ts = oracle.bin_sort(p, cam, wl.tile)
    eb = oracle.ExtBins(ids, np.zeros(len(ids), np.uint8), ts)
    lv = oracle.render_leaves(depth_projection(p), eb, cam, wl.tile, margins=oracle.MARGINS_STAGE, certain=True)
    ctx = lobe.Context(tile=wl.tile)
    batch = lobe.Batch([lobe.GaussianSet.from_numpy(s) for s in wl.sets], wl.cameras, wl.items, wl.blocks)
    gp = lobe.Projection(dev(splat_array(p)), dev(p.radius, torch.int32),
                         dev(rect_tiles(p.mean2d, p.radius, cam, wl.tile), torch.int32))
    bins = lobe.bin_sort(ctx, batch, gp)
    img, depth = lobe.render_depth(ctx, batch, gp, bins)
    D = depth.view(128, 128).cpu().numpy()
    zmax = float(p.depth[p.radius > 0].max())
    match_image(lv, np.repeat(D[None], 3, axis=0), img.T_final.view(128, 128).cpu().numpy(),
                img.n_contrib.view(128, 128).cpu().numpy(), "depth small (stage)", atol=DEPTH_RTOL * zmax)
    # the colour channels are the plain forward's, bit for bit
    plain = lobe.render_fwd(ctx, batch, gp, bins)
    assert torch.equal(plain.rgb, img.rgb) and torch.equal(plain.T_final, img.T_final)


def fcs_setup(n=60_000, n_cams=6, W=160, H=120, seed=0):
    """A small city, its median-KD blocks and aerial cameras around it."""
    g = scenes.city_layout(seed, n, extent=200.0, n_boxes=20)
    leaves = scenes.kd_median_leaves(g.means, 2)
    blocks = [box for _, box in leaves]
    rng = np.random.default_rng(seed + 5)
    cams = [scenes.aerial_camera((rng.uniform(-60, 60), rng.uniform(-60, 60), 0.0), rng.uniform(80, 120),
                                 rng.uniform(35, 60), rng.uniform(0, 360), W, H, 1.1 * W) for _ in range(n_cams)]
    return g, blocks, cams


def test_depth_end_to_end_and_coverage_match_oracle():
    g, blocks, cams = fcs_setup()
    tile = (16, 16)
    sets = [lobe.GaussianSet.from_numpy(g)]
    items = [(0, c, -1) for c in range(len(cams))]
    batch = lobe.Batch(sets, cams, items)
    ctx = lobe.Context(tile=tile)
    proj, bins, _ = lobe.forward(ctx, batch)
    img, depth = lobe.render_depth(ctx, batch, proj, bins)
    counts, npts = lobe.fcs_coverage(ctx, batch, img, depth, blocks)
    countsn, nptsn = lobe.fcs_coverage(ctx, batch, img, depth, blocks, normalize=True)
    counts, npts = counts.cpu().numpy(), npts.cpu().numpy()
    countsn = countsn.cpu().numpy()
    Ds = batch.image_views(depth, channels=1)
    Ts = batch.image_views(img.T_final, channels=1)
    g64 = oracle.set_dict(g)
    splat, radius = proj.splat.cpu().numpy(), proj.radius.cpu().numpy()
    gids, gts = bins.ids().cpu().numpy(), bins.tile_start.cpu().numpy()
    _, toffs = batch.tiles(tile)
    zmax = 0.0
    for i, cam in enumerate(cams):
        c = cam.as_dict()
        D, T = Ds[i].cpu().numpy().astype(np.float64), Ts[i].cpu().numpy().astype(np.float64)
        # counting on the GPU's own depth map: exact but for points at a box face
        for norm, got in ((False, counts[i]), (True, countsn[i])):
            want, n, near = oracle.fcs_coverage(D, T, c, blocks, normalize=norm, rel_margin=FACE_MARGIN)
            assert npts[i] == n
            assert np.all(np.abs(got.astype(np.int64) - want) <= int(near.sum())), (i, norm, got, want, near.sum())
        # the depth map itself, end to end
        p = oracle.project(g64, c, tile, margins=oracle.MARGINS_E2E)
        zmax = max(zmax, float(p.depth[p.radius > 0].max()))
        eb = oracle.bin_ext(p, c, tile)
        gx, gy = oracle.grid(c, tile)
        rb = resolve_membership(eb, gids, gts, range(gx * gy), toffs[i], batch.entry_off[i], splat[:, 0:2], radius,
                                p, c, tile, "tile lists city cameras (end to end)")
        lv = oracle.render_leaves(depth_projection(p), rb, c, tile, margins=oracle.MARGINS_E2E)
        match_image(lv, np.repeat(D[None], 3, axis=0), T, None, "depth city cameras (end to end)",
                    atol=DEPTH_RTOL * zmax)
    # the assignment of the paper (tau = 0.1) from these counts
    V, assign = lobe.fcs_select(torch.as_tensor(counts), torch.as_tensor(npts), tau=0.1)
    assert V.shape == (len(cams), len(blocks))
    assert all(sorted(a) == [c for c in range(len(cams)) if V[c, b] >= 0.1] for b, a in enumerate(assign))


def test_coverage_of_a_wall_split_by_a_block_face():
    """The closed form the oracle is pinned by, through the GPU kernels: a dense wall of
    Gaussians at depth z facing an identity-pose camera; the points left of the principal
    point fall in the block x < 0 (normalised depth puts them on the wall)."""
    rng = np.random.default_rng(0)
    n, z = 40_000, 7.0
    W, H = 64, 48
    gs = scenes.GaussianSet(
        means=np.stack([rng.uniform(-8, 8, n), rng.uniform(-6, 6, n), np.full(n, z)], 1).astype(np.float32),
        log_scales=np.full((n, 3), math.log(0.08), np.float32), quats=scenes.random_quats(rng, n),
        opacity_logits=np.full(n, 4.0, np.float32), sh=scenes.random_sh(rng, n))
    cam = scenes.pinhole(W, H, 60.0, cx=27.0, cy=24.0)
    batch = lobe.Batch([lobe.GaussianSet.from_numpy(gs)], [cam], [(0, 0, -1)])
    ctx = lobe.Context(tile=(16, 16))
    proj, bins, _ = lobe.forward(ctx, batch)
    img, depth = lobe.render_depth(ctx, batch, proj, bins)
    left = scenes.AABB((-math.inf,) * 3, (0.0, math.inf, math.inf))
    right = scenes.AABB((0.0, -math.inf, -math.inf), (math.inf,) * 3)
    counts, npts = lobe.fcs_coverage(ctx, batch, img, depth, [left, right], normalize=True)
    assert int(npts[0]) == W * H  # the wall covers the view
    cols_left = int(np.sum(np.arange(W) + 0.5 < 27.0))
    assert counts[0].tolist() == [H * cols_left, H * (W - cols_left)]
    Dn = (depth / (1 - img.T_final)).cpu().numpy()
    assert np.abs(Dn - z).max() < 0.05 * z  # the wall's depth, up to the Gaussians' extent
