"""Photometric loss of the 3DGS training step: L1 + lambda (1 - SSIM), lambda = 0.2.

This is the loss the per-block fine training minimises (appendix "3DGS Training"; the paper
evaluates SSIM with a fused kernel). It is not part of the rasterizer: the rasterizer's
adjoint starts from dL/dC, which this module produces with ordinary PyTorch ops (11x11
Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, zero padding, mean over pixels).
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

_WINDOWS = {}


def _window(device, channels=3, size=11, sigma=1.5):
    key = (device, channels, size, sigma)
    w = _WINDOWS.get(key)
    if w is None:
        x = torch.arange(size, dtype=torch.float32, device=device) - (size - 1) / 2
        g = torch.exp(-x * x / (2 * sigma * sigma))
        g = g / g.sum()
        w = (g[:, None] * g[None, :]).expand(channels, 1, size, size).contiguous()
        _WINDOWS[key] = w
    return w


def ssim(img: torch.Tensor, ref: torch.Tensor) -> torch.Tensor:
    """Mean SSIM of two [C,H,W] images."""
    C = img.shape[0]
    w = _window(img.device, C)
    x, y = img[None], ref[None]
    pad = w.shape[-1] // 2
    mu_x = F.conv2d(x, w, padding=pad, groups=C)
    mu_y = F.conv2d(y, w, padding=pad, groups=C)
    sxx = F.conv2d(x * x, w, padding=pad, groups=C) - mu_x * mu_x
    syy = F.conv2d(y * y, w, padding=pad, groups=C) - mu_y * mu_y
    sxy = F.conv2d(x * y, w, padding=pad, groups=C) - mu_x * mu_y
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    s = ((2 * mu_x * mu_y + c1) * (2 * sxy + c2)) / ((mu_x * mu_x + mu_y * mu_y + c1) * (sxx + syy + c2))
    return s.mean()


def l1_ssim_loss(img: torch.Tensor, ref: torch.Tensor, lam: float = 0.2) -> torch.Tensor:
    return (1.0 - lam) * (img - ref).abs().mean() + lam * (1.0 - ssim(img, ref))


def loss_and_grad(img: torch.Tensor, ref: torch.Tensor, lam: float = 0.2):
    """(loss, dL/dimg) of l1_ssim_loss for a detached image."""
    x = img.detach().requires_grad_(True)
    loss = l1_ssim_loss(x, ref, lam)
    (g,) = torch.autograd.grad(loss, x)
    return loss.detach(), g
