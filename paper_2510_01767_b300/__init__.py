"""B300-native differentiable tile rasterizer for the per-block training step of LoBE-GS
(arXiv 2510.01767): EWA projection with SH colour, visibility cropping, tile binning by
(tile, depth) sort, front-to-back compositing and its adjoint, all in hand-written CUDA
for sm_103a behind the C ABI of include/lobe.h.

There is no CPU fallback: every stage needs liblobe.so (``python -m
paper_2510_01767_b300.build``) and a CUDA device.
"""
from .raster import (ADAM_LR_3DGS, Adam, Batch, Bins, Context, GaussianSet, Image, Projection, PARAM_KEYS, bin_sort,
                     densify, fcs_coverage, project_bwd_adam,
                     fcs_select, forward, project, project_bwd, render_bwd, render_depth, render_fwd, visibility_crop,
                     zero_grads)

from .autograd import LobeRasterize, Rasterizer, crop_compact, rasterize

__all__ = ["LobeRasterize", "Rasterizer", "crop_compact", "rasterize","Batch", "Bins", "Context", "GaussianSet", "Image", "Projection", "PARAM_KEYS", "bin_sort", "forward",
           "project", "project_bwd", "render_bwd", "render_fwd", "visibility_crop", "zero_grads", "render_depth",
           "fcs_coverage", "fcs_select", "densify", "ADAM_LR_3DGS", "Adam", "project_bwd_adam"]
