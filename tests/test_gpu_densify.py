"""Selective densification (Sec. 3.3, with the 3DGS density control) on the GPU against the
oracle: which Gaussians are pruned, cloned, split or kept, and in which order (bit-exact: both
sides decide in float32), and the output parameters (copies exact; split children's means
within float32 rounding of mu + R (s * z), log-scales of log_s - log 1.6)."""
import math

import numpy as np
import pytest
import torch

import oracle
import scenes

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def random_stats(rng, n, block_frac=0.6):
    cnt = np.where(rng.uniform(size=n) < block_frac, rng.integers(1, 8, n), 0).astype(np.int32)
    acc = (rng.exponential(2e-4, n) * np.maximum(cnt, 1)).astype(np.float32)
    acc[cnt == 0] = rng.exponential(1.0, int((cnt == 0).sum()))  # outside the block: ignored
    return acc, cnt


@pytest.mark.parametrize("n_split", [2, 3])
def test_densify_matches_oracle(n_split):
    rng = np.random.default_rng(n_split)
    n = 200_000
    g = scenes.uniform_gaussians(rng, n, 10.0, 5.0, 50.0, logscale_shift=math.log(10.0))
    g.opacity_logits[:] = rng.normal(0.0, 3.0, n).astype(np.float32)  # some below logit(0.005)
    acc, cnt = random_stats(rng, n)
    normals = rng.standard_normal((n, n_split, 3)).astype(np.float32)
    extent = 20.0
    gs = lobe.GaussianSet.from_numpy(g)
    ctx = lobe.Context()
    out, src = lobe.densify(ctx, gs, torch.as_tensor(acc).cuda(), torch.as_tensor(cnt).cuda(),
                            torch.as_tensor(normals).cuda(), grad_threshold=2e-4, percent_dense=0.01,
                            scene_extent=extent, min_opacity=0.005, n_split=n_split)
    want, wsrc = oracle.densify(g.arrays(), acc, cnt, normals, 2e-4, math.log(0.01 * extent),
                                math.log(0.005 / 0.995), n_split, math.log(0.8 * n_split))
    src = src.cpu().numpy()
    np.testing.assert_array_equal(src, wsrc)
    # split children are the outputs whose log-scales shrank
    kids = np.any(want["log_scales"] != np.asarray(g.log_scales, np.float64)[wsrc], axis=1)
    assert 0 < kids.sum() < len(wsrc)
    assert len(wsrc) != n  # something was pruned, cloned or split
    for k in ("quats", "opacity_logits", "sh"):  # copied unchanged
        np.testing.assert_array_equal(getattr(out, k).cpu().numpy(), np.asarray(getattr(g, k))[wsrc])
    m = out.means.cpu().numpy().astype(np.float64)
    ls = out.log_scales.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(m[~kids], np.asarray(g.means, np.float64)[wsrc[~kids]])
    np.testing.assert_array_equal(ls[~kids], np.asarray(g.log_scales, np.float64)[wsrc[~kids]])
    # children: float32 arithmetic against FP64, relative to the mean and the parent's extent
    scale = np.abs(want["means"][kids]) + np.exp(want["log_scales"][kids]).max(1, keepdims=True) * 2
    assert float((np.abs(m[kids] - want["means"][kids]) / scale).max()) < 1e-5
    np.testing.assert_allclose(ls[kids], want["log_scales"][kids], rtol=0, atol=1e-5)


def test_densify_capacity_and_empty():
    ctx = lobe.Context()
    rng = np.random.default_rng(1)
    g = scenes.uniform_gaussians(rng, 0, 1.0, 2.0, 6.0)
    gs = lobe.GaussianSet.from_numpy(g)
    out, src = lobe.densify(ctx, gs, torch.zeros(0, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert out.n == 0 and src.numel() == 0
