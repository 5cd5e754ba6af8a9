"""The allocation-free binning entry point, lobe_bin_sort_noalloc.

Callers that may not allocate device memory (an embedding application that owns the GPU's
memory through its own pool or budget, or a real-time loop that cannot afford an
allocation's synchronisation) bin through this call, whose scratch is a fixed device array
inside the library. Here it is called through the C ABI twice in a row on different inputs
and must give exactly the ids, tile ranges and pair count of the context-based
lobe_bin_sort (binning is index work: the comparison is bit for bit). The second call
checks that nothing left in the shared array by the first one leaks into its result.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300 import _abi as A


def reference_and_noalloc(wl):
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=wl.tile)
    proj = lobe.project(ctx, batch)
    ref = lobe.bin_sort(ctx, batch, proj)  # context-owned scratch
    n_tiles, _ = batch.tiles(wl.tile)
    out = lobe.raster.empty_bins(ref.count + 1024, n_tiles)
    out.gauss_ids.fill_(-7)
    out.tile_start.fill_(-7)
    torch.cuda.synchronize()
    n = ctypes.c_int64(-1)
    code = A.lib().lobe_bin_sort_noalloc(ctypes.byref(ctx._config()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(batch.c), ctypes.byref(proj.c()), ctypes.byref(out.c()),
                                         ctypes.byref(n))
    assert code == A.OK, A.STATUS_NAMES.get(code, code)
    torch.cuda.synchronize()
    return ref, out, n.value


def check_equal(ref, out, n):
    assert n == ref.count
    assert int(out.n_isect.item()) == ref.count
    np.testing.assert_array_equal(out.gauss_ids[:n].cpu().numpy(), ref.ids().cpu().numpy())
    np.testing.assert_array_equal(out.tile_start.cpu().numpy(), ref.tile_start.cpu().numpy())


def test_noalloc_matches_bin_sort_on_two_calls():
    first = scenes.small_scene(seed=0)
    rng = np.random.default_rng(5)
    g = scenes.uniform_gaussians(rng, 5000, 1.5, 2.0, 8.0)
    cams = [scenes.pinhole(320, 200, 260.0), scenes.pinhole(100, 75, 90.0)]
    second = scenes.Workload("two_items", [g], cams, [], [(0, 0, -1), (0, 1, -1)], (8, 8))
    ref1, out1, n1 = reference_and_noalloc(first)
    ref2, out2, n2 = reference_and_noalloc(second)
    assert n1 > 0 and n2 > 0 and n1 != n2
    check_equal(ref1, out1, n1)
    check_equal(ref2, out2, n2)


def test_noalloc_rejects_batches_beyond_its_limits():
    rng = np.random.default_rng(2)
    g = scenes.uniform_gaussians(rng, 1000, 1.0, 2.0, 6.0)
    # 4096 x 4096 with 8x8 tiles: 262144 tiles > LOBE_NOALLOC_MAX_TILES
    wl = scenes.Workload("big", [g], [scenes.pinhole(4096, 4096, 3000.0)], [], [(0, 0, -1)], (8, 8))
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=wl.tile)
    proj = lobe.project(ctx, batch)
    n_tiles, _ = batch.tiles(wl.tile)
    out = lobe.raster.empty_bins(1 << 16, n_tiles)
    code = A.lib().lobe_bin_sort_noalloc(ctypes.byref(ctx._config()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(batch.c), ctypes.byref(proj.c()), ctypes.byref(out.c()), None)
    assert code == A.ERR_CAPACITY


def call_noalloc(ctx, batch, proj, out):
    n = ctypes.c_int64(-1)
    code = A.lib().lobe_bin_sort_noalloc(ctypes.byref(ctx._config()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(batch.c), ctypes.byref(proj.c()), ctypes.byref(out.c()),
                                         ctypes.byref(n))
    torch.cuda.synchronize()
    return code, n.value


def test_noalloc_lists_match_the_oracle():
    """One small view binned by the allocation-free call against the oracle's (tile, depth,
    index) sort of the same float32 splats: the lists and tile ranges bit for bit."""
    import oracle

    wl = scenes.small_scene(seed=3)
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=wl.tile)
    proj = lobe.project(ctx, batch)
    n_tiles, _ = batch.tiles(wl.tile)
    out = lobe.raster.empty_bins(1 << 16, n_tiles)
    code, n = call_noalloc(ctx, batch, proj, out)
    assert code == A.OK, A.STATUS_NAMES.get(code, code)
    sp = proj.splat.cpu().numpy().astype(np.float64)
    radius = proj.radius.cpu().numpy()
    p = oracle.Projection(sp[:, 0:2], sp[:, 2:5], sp[:, 6:9], sp[:, 5], sp[:, 9], radius,
                          np.zeros((len(radius), 4), np.int32), np.zeros(len(radius), np.int32), radius)
    ids, ts = oracle.bin_sort(p, wl.cameras[0].as_dict(), wl.tile)
    assert n == len(ids) > 0
    np.testing.assert_array_equal(out.gauss_ids[:n].cpu().numpy(), ids)
    np.testing.assert_array_equal(out.tile_start.cpu().numpy(), ts)


def test_noalloc_reports_overflow_then_recovers():
    """Bins one pair too small: LOBE_ERR_CAPACITY with the true pair count and every tile
    empty. The next call, on the same shared array (whose status word the overflow latched),
    must then bin bit-exactly like lobe_bin_sort again."""
    wl = scenes.small_scene(seed=4)
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    ctx = lobe.Context(tile=wl.tile)
    proj = lobe.project(ctx, batch)
    ref = lobe.bin_sort(ctx, batch, proj)
    n_tiles, _ = batch.tiles(wl.tile)
    small = lobe.raster.empty_bins(ref.count - 1, n_tiles)
    small.tile_start.fill_(-7)
    code, n = call_noalloc(ctx, batch, proj, small)
    assert code == A.ERR_CAPACITY
    assert n == ref.count
    assert int(small.tile_start.abs().max().item()) == 0
    out = lobe.raster.empty_bins(ref.count, n_tiles)
    code, n = call_noalloc(ctx, batch, proj, out)
    assert code == A.OK, A.STATUS_NAMES.get(code, code)
    check_equal(ref, out, n)
