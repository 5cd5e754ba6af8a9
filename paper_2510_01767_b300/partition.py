"""Load-balanced KD-tree scene partition with cutline refinement (Alg. 1, Sec. 3.1), driven by
fast camera selection on the GPU (Sec. 3.2).

The camera sets of candidate boxes come from ``lobe_fcs_coverage`` over the depth maps of all
cameras, rendered once from the coarse model (``CameraDepths``); every cut the refinement
tries costs one pass over those maps. The tree logic itself (best-first growth on the
workload L(B) = |C(B)|, axis choice, percentile cuts, bisection toward the lighter child) is
host code in the library, ``lobe_kd_partition``; this module marshals its arguments.

Readings (the paper leaves them open): boxes are half-open (lo <= p < hi) as for selective
densification; the split axis is the longer of the x / y extents of the coarse centres inside
the node; the cut at percentile q interpolates linearly between the order statistics of those
centres' coordinates at (n - 1) q; after the bisection the children of the last evaluated cut are kept; among
leaves of equal workload the earliest created is split first.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi as A
from . import raster as R


class CameraDepths:
    """Depth maps (composite depth + T_final) of every camera over one Gaussian set, and the
    per-box coverage counts of their back-projected points."""

    def __init__(self, ctx: R.Context, gaussians: R.GaussianSet, cameras, normalize=False):
        self.ctx = ctx
        self.cameras = [c if isinstance(c, dict) else c.as_dict() for c in cameras]
        self.batch = R.Batch([gaussians], self.cameras, [(0, c, -1) for c in range(len(self.cameras))])
        proj, bins, _ = R.forward(ctx, self.batch)
        self.image, self.depth = R.render_depth(ctx, self.batch, proj, bins)
        self.normalize = normalize

    @classmethod
    def from_maps(cls, ctx: R.Context, cameras, depth: torch.Tensor, T_final: torch.Tensor, normalize=False):
        """Coverage over given depth / T_final maps (flat, items in camera order)."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.cameras = [c if isinstance(c, dict) else c.as_dict() for c in cameras]
        dummy = R.GaussianSet(*(torch.zeros((0,) + s, device="cuda") for s in ((3,), (3,), (4,), (), (16, 3))))
        self.batch = R.Batch([dummy], self.cameras, [(0, c, -1) for c in range(len(self.cameras))])
        n = self.batch.n_pixels
        self.image = R.Image(torch.zeros(3 * n, device="cuda"), T_final.contiguous(),
                             torch.zeros(n, dtype=torch.int32, device="cuda"))
        self.depth = depth.contiguous()
        self.normalize = normalize
        return self

    def ratios(self, boxes):
        """V[camera, box] = points inside the box / the camera's points (0 without points)."""
        counts, npts = R.fcs_coverage(self.ctx, self.batch, self.image, self.depth, boxes, self.normalize)
        V, _ = R.fcs_select(counts, npts, tau=0.0)
        return V.numpy()


class Box:
    def __init__(self, lo, hi):
        self.lo, self.hi = tuple(float(x) for x in lo), tuple(float(x) for x in hi)


def kd_partition(centers, root, n_blocks: int, depths, tau=0.1, q_lo=0.1, q_hi=0.9, steps=3):
    """Returns the leaves [(lo, hi, camera indices)] in creation order (see the module); the
    tree runs in the library (``lobe_kd_partition``), calling back here only for the ratios
    (``depths.ratios(boxes)``, a [cameras, boxes] array)."""
    c = np.ascontiguousarray(np.asarray(centers, np.float64).reshape(-1, 3))
    n_cams = len(depths.cameras)
    root_box = A.BoxD()
    root_box.lo[:] = [float(x) for x in root.lo]
    root_box.hi[:] = [float(x) for x in root.hi]
    failure = []

    def ratios(_user, boxes, nb, out):
        try:
            bx = [Box(tuple(boxes[b].lo), tuple(boxes[b].hi)) for b in range(nb)]
            V = np.ascontiguousarray(depths.ratios(bx), np.float64).reshape(n_cams, nb)
            ctypes.memmove(out, V.ctypes.data, V.nbytes)
            return 0
        except Exception as e:  # reported after the call returns
            failure.append(e)
            return 1

    cb = A.RATIO_FN(ratios)
    prm = A.KdParams(int(n_blocks), float(tau), float(q_lo), float(q_hi), int(steps))
    leaves = (A.BoxD * int(n_blocks))()
    cams = np.zeros((int(n_blocks), max(n_cams, 1)), np.uint8)
    code = A.lib().lobe_kd_partition(c.ctypes.data, c.shape[0], ctypes.byref(root_box), n_cams, cb, None,
                                     ctypes.byref(prm), leaves, cams.ctypes.data)
    if failure:
        raise failure[0]
    A.check(code)
    return [(np.array(leaves[b].lo), np.array(leaves[b].hi), [int(k) for k in np.nonzero(cams[b, :n_cams])[0]])
            for b in range(int(n_blocks))]


def workloads(leaves):
    """L(B) = |C(B)| of each leaf (the paper's proxy of fine-training time)."""
    return [len(c) for _, _, c in leaves]
