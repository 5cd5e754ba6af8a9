"""Host logic of the load-balanced KD partition (Alg. 1, Sec. 3.1) without a GPU: the library's
tree bookkeeping (best-first growth on |C(B)|, axis choice, percentile cuts, bisection toward
the lighter child) driven by camera ratios counted on the CPU from explicit point sets (in
place of the GPU's coverage counts of back-projected depth maps) reproduces the oracle's loops
exactly."""
import math

import numpy as np
import pytest

import oracle
import scenes
from paper_2510_01767_b300.partition import kd_partition, workloads


class PointDepths:
    """The interface kd_partition uses (``cameras``, ``ratios(boxes)``), from per-camera points:
    V[c, b] = points of camera c inside box b (half-open) / all its points."""

    def __init__(self, pts):
        self.cameras = list(range(len(pts)))
        self.pts = [np.asarray(p, np.float64) for p in pts]

    def ratios(self, boxes):
        V = np.zeros((len(self.pts), len(boxes)))
        for c, p in enumerate(self.pts):
            if len(p) == 0:
                continue
            for b, box in enumerate(boxes):
                inside = np.all((p >= np.asarray(box.lo)) & (p < np.asarray(box.hi)), axis=1)
                V[c, b] = inside.sum() / len(p)
        return V


def camera_points(rng, n_cams, spread):
    return [np.stack([rng.normal(cx, spread[0], 400), rng.normal(cy, spread[1], 400), np.zeros(400)], 1)
            for cx, cy in zip(rng.uniform(-60, 60, n_cams), rng.uniform(-25, 25, n_cams))]


@pytest.mark.parametrize("n_blocks, seed", [(2, 0), (5, 1), (8, 2), (12, 3)])
def test_kd_partition_host_logic_matches_oracle(n_blocks, seed):
    rng = np.random.default_rng(seed)
    centers = np.stack([rng.uniform(-60, 60, 30_000) * rng.uniform(0.3, 1.0, 30_000),
                        rng.uniform(-25, 25, 30_000), np.zeros(30_000)], 1)
    cams = camera_points(rng, 40, (10.0, 5.0))
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    want = oracle.kd_partition(centers, root, n_blocks, cams)
    got = kd_partition(centers, root, n_blocks, PointDepths(cams))
    assert len(got) == len(want) == n_blocks
    for (glo, ghi, gc), (wlo, whi, wc) in zip(got, want):
        np.testing.assert_array_equal(glo, wlo)
        np.testing.assert_array_equal(ghi, whi)
        assert list(gc) == list(wc)
    assert max(workloads(got)) <= len(cams)


def test_kd_partition_camera_sets_shrink_down_the_tree():
    """A child's camera set is a subset of its parent's (Alg. 1 filters the parent's cameras),
    so the workload never exceeds the root's and every leaf keeps only cameras seeing >= tau."""
    rng = np.random.default_rng(7)
    centers = np.stack([rng.uniform(-60, 60, 20_000), rng.uniform(-25, 25, 20_000), np.zeros(20_000)], 1)
    cams = camera_points(rng, 30, (8.0, 4.0))
    depths = PointDepths(cams)
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    leaves = kd_partition(centers, root, 6, depths)
    V = depths.ratios([type("B", (), {"lo": lo, "hi": hi})() for lo, hi, _ in leaves])
    for b, (_, _, cs) in enumerate(leaves):
        assert all(V[c, b] >= 0.1 for c in cs)
        assert set(cs) <= set(range(30))
