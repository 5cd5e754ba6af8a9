"""Load-balanced KD-tree scene partition with cutline refinement (Alg. 1, Sec. 3.1), driven by
fast camera selection on the GPU (Sec. 3.2).

The camera sets of candidate boxes come from ``lobe_fcs_coverage`` over the depth maps of all
cameras, rendered once from the coarse model (``camera_depths``); every cut the refinement
tries costs one pass over those maps. The tree logic itself (best-first growth on the
workload L(B) = |C(B)|, axis choice, percentile cuts, bisection toward the lighter child) is
host-side bookkeeping.

Readings (the paper leaves them open): boxes are half-open (lo <= p < hi) as for selective
densification; the split axis is the longer of the x / y extents of the coarse centres inside
the node; the cut at percentile q is numpy's linear-interpolated quantile of those centres'
coordinates; after the bisection the children of the last evaluated cut are kept; among
leaves of equal workload the earliest created is split first.
"""
from __future__ import annotations

import heapq
import math

import numpy as np
import torch

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
        c, n = counts.cpu().numpy().astype(np.float64), npts.cpu().numpy().astype(np.float64)
        return np.where(n[:, None] > 0, c / np.maximum(n, 1)[:, None], 0.0)


class Box:
    def __init__(self, lo, hi):
        self.lo, self.hi = tuple(float(x) for x in lo), tuple(float(x) for x in hi)


def kd_partition(centers, root, n_blocks: int, depths: CameraDepths, tau=0.1, q_lo=0.1, q_hi=0.9, steps=3):
    """Returns the leaves [(lo, hi, camera indices)] in creation order (see the module)."""
    centers = np.asarray(centers, np.float64)
    lo0 = np.array(root.lo, np.float64)
    hi0 = np.array(root.hi, np.float64)

    def cams_of(boxes, parent):
        V = depths.ratios([Box(lo, hi) for lo, hi in boxes])
        return [[c for c in parent if V[c, b] >= tau] for b in range(len(boxes))]

    root_cams = cams_of([(lo0, hi0)], list(range(len(depths.cameras))))[0]
    heap = [(-len(root_cams), 0, lo0, hi0, root_cams)]
    serial = 1
    while len(heap) < n_blocks:
        _, _, lo, hi, cams = heapq.heappop(heap)
        m = np.all((centers >= lo) & (centers < hi), axis=1)
        pts = centers[m]
        ext = [float(pts[:, d].max() - pts[:, d].min()) if len(pts) else 0.0 for d in (0, 1)]
        a = 0 if ext[0] >= ext[1] else 1
        coords = np.sort(pts[:, a])
        qlo, qhi, q = q_lo, q_hi, 0.5
        for _ in range(steps):
            cut = float(np.quantile(coords, q)) if len(coords) else 0.5 * (lo[a] + hi[a])
            hl, lr = hi.copy(), lo.copy()
            hl[a] = cut
            lr[a] = cut
            cl, cr = cams_of([(lo, hl), (lr, hi)], cams)
            if len(cl) > len(cr):
                qhi, q = q, 0.5 * (qlo + q)
            elif len(cr) > len(cl):
                qlo, q = q, 0.5 * (qhi + q)
            else:
                break
        heapq.heappush(heap, (-len(cl), serial, lo, hl, cl))
        heapq.heappush(heap, (-len(cr), serial + 1, lr, hi, cr))
        serial += 2
    leaves = sorted(heap, key=lambda e: e[1])
    return [(lo, hi, cams) for _, _, lo, hi, cams in leaves]


def workloads(leaves):
    """L(B) = |C(B)| of each leaf (the paper's proxy of fine-training time)."""
    return [len(c) for _, _, c in leaves]
