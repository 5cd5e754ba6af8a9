"""torch.autograd binding of the rasterizer for the per-block training loop.

``rasterize(means, log_scales, quats, opacity_logits, sh, cameras, raster)`` renders one or
more views of one Gaussian set through the CUDA stages (project -> bin/sort -> composite);
its backward is the library's hand-written adjoint (render_bwd -> project_bwd), which also
accumulates the selective-densification statistic of Sec. 3.3 into ``raster.sd_acc`` /
``raster.sd_cnt`` (for Gaussians visible in a view whose mean lies in the block box).

``Rasterizer(recompute_T=True)`` makes the backward re-derive each pixel's stop position and
colour with a forward sweep instead of keeping the forward's per-pixel state alive until
backward (a memory/compute trade; both give the same gradients).
"""
from __future__ import annotations

import torch

from . import raster as R


class Rasterizer:
    """Per-block rasterizer state: CUDA context, block box, crop mask, SD statistics."""

    def __init__(self, n_gaussians: int, tile=(16, 16), sh_degree=3, bg=(0.0, 0.0, 0.0), recompute_T=False,
                 block=None, crop_mask: torch.Tensor | None = None):
        self.ctx = R.Context(tile=tile, sh_degree=sh_degree, bg=bg, recompute_T=recompute_T)
        self.block = block
        self.crop_mask = crop_mask
        self.sd_acc = torch.zeros(n_gaussians, dtype=torch.float32, device="cuda")
        self.sd_cnt = torch.zeros(n_gaussians, dtype=torch.int32, device="cuda")
        self.last_bins = None

    def reset_stats(self):
        self.sd_acc.zero_()
        self.sd_cnt.zero_()

    def grow_stats(self, n):
        """Resize the SD statistics after densification (new Gaussians start at zero)."""
        acc = torch.zeros(n, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        k = min(n, self.sd_acc.shape[0])
        acc[:k] = self.sd_acc[:k]
        cnt[:k] = self.sd_cnt[:k]
        self.sd_acc, self.sd_cnt = acc, cnt

    def batch(self, params, cameras):
        g = R.GaussianSet(*[p.detach().contiguous() for p in params], crop_mask=self.crop_mask)
        return self.batch_of(g, cameras)

    def batch_of(self, g: R.GaussianSet, cameras):
        blocks = [self.block] if self.block is not None else []
        items = [(0, i, 0 if blocks else -1) for i in range(len(cameras))]
        return R.Batch([g], cameras, items, blocks)

    def train_step(self, opt: R.Adam, cameras, loss_fn, sparse: bool = False):
        """One training step with the Adam update fused into the projection adjoint: render
        the views of ``cameras`` from opt.set, loss_fn(list of [3,H,W] views) -> scalar tensor
        (differentiated by torch on the images only), render adjoint, then the fused projection
        adjoint + Adam (standard, or sparse: only the Gaussians some view sees change). The SD
        statistics accumulate as in ``rasterize``. Returns the loss (detached)."""
        if isinstance(cameras, dict) or hasattr(cameras, "as_dict"):
            cameras = [cameras]
        if opt.set.crop_mask is not self.crop_mask:
            opt.set.crop_mask = self.crop_mask
        batch = self.batch_of(opt.set, list(cameras))
        proj, bins, img = R.forward(self.ctx, batch, sync=True)
        self.last_bins = bins
        rgb = img.rgb.detach().requires_grad_(True)
        loss = loss_fn(batch.image_views(rgb))
        (d_rgb,) = torch.autograd.grad(loss, rgb)
        g2d = R.render_bwd(self.ctx, batch, proj, bins, None if self.ctx.recompute_T else img, d_rgb.contiguous())
        sd = [{"sd_acc": self.sd_acc, "sd_cnt": self.sd_cnt}] if self.sd_acc.shape[0] == opt.set.n else None
        R.project_bwd_adam(self.ctx, batch, proj, g2d, [opt], sd=sd, sparse=sparse)
        return loss.detach()


class LobeRasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, cameras, raster: Rasterizer):
        batch = raster.batch((means, log_scales, quats, opacity_logits, sh), cameras)
        proj, bins, img = R.forward(raster.ctx, batch, sync=True)
        raster.last_bins = bins
        ctx.raster = raster
        ctx.batch = batch
        ctx.proj = proj
        ctx.bins = bins
        ctx.img = None if raster.ctx.recompute_T else img
        ctx.shapes = [p.shape for p in (means, log_scales, quats, opacity_logits, sh)]
        views = batch.image_views(img.rgb)
        if len(views) == 1:
            return views[0]
        if all(v.shape == views[0].shape for v in views):
            return img.rgb.view(len(views), *views[0].shape)
        return img.rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        raster = ctx.raster
        dL = grad_rgb.contiguous().reshape(-1)
        g2d = R.render_bwd(raster.ctx, ctx.batch, ctx.proj, ctx.bins, ctx.img, dL)
        n = ctx.batch.sets[0].n
        grads = {k: torch.empty(s, dtype=torch.float32, device="cuda") for k, s in zip(R.PARAM_KEYS, ctx.shapes)}
        if raster.sd_acc.shape[0] == n:
            grads["sd_acc"], grads["sd_cnt"] = raster.sd_acc, raster.sd_cnt
        R.project_bwd(raster.ctx, ctx.batch, ctx.proj, g2d, [grads], accumulate=False)
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"], grads["sh"], None, None)


def rasterize(means, log_scales, quats, opacity_logits, sh, cameras, raster: Rasterizer):
    """Differentiable render of one Gaussian set in ``cameras`` (a camera dict or a list).
    Returns [3,H,W] for one view, [V,3,H,W] for views of equal size, else the flat planar
    buffer (see Batch.image_views)."""
    if isinstance(cameras, dict) or hasattr(cameras, "as_dict"):
        cameras = [cameras]
    return LobeRasterize.apply(means, log_scales, quats, opacity_logits, sh, list(cameras), raster)


def crop_compact(params: dict, mask: torch.Tensor) -> dict:
    """Visibility cropping (Sec. 3.3) applied once before fine training: keep only the
    Gaussians of ``mask`` (from raster.visibility_crop). Returns new contiguous tensors."""
    idx = mask.nonzero().squeeze(1)
    return {k: v.index_select(0, idx).contiguous() for k, v in params.items()}
