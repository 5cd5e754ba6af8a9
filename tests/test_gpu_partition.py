"""Load-balanced KD partition with cutline refinement (Alg. 1) driven by fast camera selection
on the GPU, against the oracle's loops over the same cameras' back-projected points.

The depth maps are synthetic and exact: aerial cameras over the ground plane z = 0, each
pixel's depth the camera-space z of its ray's hit point (no hit: T = 1). Both sides partition
the same coarse centres; the cuts (percentiles of the same coordinates) and the camera sets
must agree exactly."""
import math

import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300.partition import CameraDepths, kd_partition, workloads


def ground_depth(cam, W, H):
    """Camera-space depth of the plane z = 0 at every pixel centre (T = 1 where the ray misses)."""
    V = np.asarray(cam["viewmat"], np.float64)
    R, t = V[:3, :3], V[:3, 3]
    eye = -R.T @ t
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    dc = np.stack([(px + 0.5 - cam["cx"]) / cam["fx"], (py + 0.5 - cam["cy"]) / cam["fy"], np.ones_like(px)], -1)
    dw = dc @ R  # world direction of each ray (camera z = 1)
    s = -eye[2] / dw[..., 2]  # ray parameter of the hit; camera-space depth = s (dc has z = 1)
    hit = s > 0
    return np.where(hit, s, 0.0), np.where(hit, 0.0, 1.0)


def cameras(rng, n, W, H):
    return [scenes.aerial_camera((rng.uniform(-80, 80), rng.uniform(-40, 40), 0.0), rng.uniform(60, 120),
                                 rng.uniform(30, 70), rng.uniform(0, 360), W, H, 1.1 * W).as_dict() for _ in range(n)]


@pytest.mark.parametrize("n_blocks", [2, 6])
def test_partition_matches_oracle(n_blocks):
    rng = np.random.default_rng(n_blocks)
    W, H = 96, 64
    cams = cameras(rng, 24, W, H)
    maps = [ground_depth(c, W, H) for c in cams]
    centers = np.stack([rng.uniform(-100, 100, 50_000), rng.uniform(-50, 50, 50_000), np.zeros(50_000)], 1)
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    # oracle: the cameras' back-projected points from the same depth maps
    pts = []
    for c, (D, T) in zip(cams, maps):
        p, m = oracle.backproject(D, T, c)
        pts.append(p[m])
    want = oracle.kd_partition(centers, root, n_blocks, pts)
    ctx = lobe.Context()
    depth = torch.as_tensor(np.concatenate([D.reshape(-1) for D, _ in maps]), dtype=torch.float32).cuda()
    T = torch.as_tensor(np.concatenate([t.reshape(-1) for _, t in maps]), dtype=torch.float32).cuda()
    got = kd_partition(centers, root, n_blocks, CameraDepths.from_maps(ctx, cams, depth, T))
    assert len(got) == len(want) == n_blocks
    for (glo, ghi, gc), (wlo, whi, wc) in zip(got, want):
        np.testing.assert_array_equal(glo, wlo)
        np.testing.assert_array_equal(ghi, whi)
        assert gc == wc
    assert max(workloads(got)) < len(cams)


def test_partition_of_a_rendered_city():
    """End to end on a coarse model: depth maps rendered from the Gaussians, 4 blocks; every
    leaf gets cameras and the worst leaf carries at most the parent's set."""
    g = scenes.city_layout(3, 200_000, extent=200.0, n_boxes=20)
    rng = np.random.default_rng(9)
    cams = cameras(rng, 16, 160, 120)
    ctx = lobe.Context()
    depths = CameraDepths(ctx, lobe.GaussianSet.from_numpy(g), cams)
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    leaves = kd_partition(g.means, root, 4, depths)
    assert len(leaves) == 4 and all(len(c) > 0 for _, _, c in leaves)
    owner = np.zeros(g.n, int)
    for lo, hi, _ in leaves:
        owner += np.all((g.means >= lo) & (g.means < hi), axis=1)
    assert np.all(owner == 1)
