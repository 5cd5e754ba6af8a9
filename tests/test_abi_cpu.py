"""CPU-side checks of the C ABI: the library loads, exports every entry point that
include/lobe.h declares, and its host-only calls (argument validation, batch sizing)
behave as documented. No GPU needed: nothing here launches a kernel."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lobe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lobe_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2510_01767_b300 import build, _abi
    build.build()
    return _abi.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("lobe_project", "lobe_bin_sort", "lobe_render_fwd", "lobe_render_bwd", "lobe_project_bwd"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    from paper_2510_01767_b300 import _abi
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in _abi.SIGNATURES, f"{name} has no ctypes signature"


def test_abi_version(L):
    assert L.lobe_abi_version() == 1


def test_struct_sizes_match_header_layout():
    from paper_2510_01767_b300 import _abi as A
    assert ctypes.sizeof(A.Camera) == 16 * 4 + 4 * 4 + 2 * 4 + 2 * 4
    assert ctypes.sizeof(A.AABB) == 24
    assert ctypes.sizeof(A.Item) == 12
    assert ctypes.sizeof(A.Gaussians) == 6 * 8 + 8
    assert ctypes.sizeof(A.Config) == 4 * 3 + 12 + 4 + 28


def _batch(A, cams, n_per_set, items):
    sets = (A.Gaussians * len(n_per_set))()
    for i, n in enumerate(n_per_set):
        # host-only sizing never dereferences these; 16-byte aligned fake addresses
        sets[i].means = sets[i].log_scales = sets[i].quats = sets[i].opacity_logits = sets[i].sh = 4096
        sets[i].n = n
    cs = (A.Camera * len(cams))()
    for i, (w, h) in enumerate(cams):
        cs[i].width, cs[i].height, cs[i].fx, cs[i].fy = w, h, 100.0, 100.0
        cs[i].viewmat[0] = cs[i].viewmat[5] = cs[i].viewmat[10] = cs[i].viewmat[15] = 1.0
    its = (A.Item * len(items))(*[A.Item(s, c, -1) for s, c in items])
    return A.Batch(sets, len(n_per_set), cs, len(cams), None, 0, its, len(items)), (sets, cs, its)


def test_batch_sizes(L):
    from paper_2510_01767_b300 import _abi as A
    cfg = A.Config(16, 16, 3)
    b, keep = _batch(A, [(1600, 1066), (100, 75)], [1000, 250], [(0, 0), (1, 1), (0, 1)])
    out = (ctypes.c_int64 * 3)()
    assert L.lobe_batch_sizes(ctypes.byref(cfg), ctypes.byref(b), out) == 0
    for n in (32, 64):  # either staging batch is a valid configuration
        cfg.batch_fwd = cfg.batch_bwd = n
        assert L.lobe_batch_sizes(ctypes.byref(cfg), ctypes.byref(b), out) == 0
    assert out[0] == 1000 + 250 + 1000
    assert out[1] == 100 * 67 + 7 * 5 + 7 * 5
    assert out[2] == 1600 * 1066 + 2 * 100 * 75


@pytest.mark.parametrize("bad", ["tile", "degree", "set_index", "camera_index", "intrinsics", "alignment", "items",
                                 "batch_size", "batch_one_px", "batch_odd_px"])
def test_argument_errors(L, bad):
    from paper_2510_01767_b300 import _abi as A
    cfg = A.Config(16, 16, 3)
    b, keep = _batch(A, [(64, 64)], [10], [(0, 0)])
    sets, cs, its = keep
    if bad == "tile":
        cfg.tile_w = 12
    elif bad == "degree":
        cfg.sh_degree = 4
    elif bad == "set_index":
        its[0].set = 3
    elif bad == "camera_index":
        its[0].camera = 2
    elif bad == "intrinsics":
        cs[0].fx = 0.0
    elif bad == "alignment":
        sets[0].sh = 4100
    elif bad == "items":
        b.n_items = 0
    elif bad == "batch_size":
        cfg.batch_fwd = 48  # staging rounds of 32 or 64 splats only
    elif bad == "batch_one_px":
        cfg.tile_w, cfg.tile_h, cfg.px_fwd, cfg.batch_fwd = 16, 8, 1, 64  # 64 needs two or more pixels a lane
    elif bad == "batch_odd_px":
        cfg.tile_w, cfg.tile_h, cfg.px_bwd, cfg.batch_bwd = 8, 8, 1, 64  # the paired adjoint only
    out = (ctypes.c_int64 * 3)()
    assert L.lobe_batch_sizes(ctypes.byref(cfg), ctypes.byref(b), out) == A.ERR_ARG


def test_product_path_fails_loudly_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2510_01767_b300 as lobe
    with pytest.raises(RuntimeError, match="CUDA"):
        lobe.Context()


def test_batch_limits(L):
    """LOBE_MAX_SETS sets and LOBE_MAX_ITEMS items pass; one more of either is an argument error."""
    from paper_2510_01767_b300 import _abi as A
    cfg = A.Config(16, 16, 3)
    out = (ctypes.c_int64 * 3)()
    n_sets, n_items = 16, 64
    b, keep = _batch(A, [(64, 48)] * 4, [10] * n_sets, [(i % n_sets, i % 4) for i in range(n_items)])
    assert L.lobe_batch_sizes(ctypes.byref(cfg), ctypes.byref(b), out) == 0
    assert out[0] == n_items * 10
    b, keep = _batch(A, [(64, 48)] * 4, [10] * n_sets, [(i % n_sets, i % 4) for i in range(n_items + 1)])
    assert L.lobe_batch_sizes(ctypes.byref(cfg), ctypes.byref(b), out) == A.ERR_ARG
    b, keep = _batch(A, [(64, 48)] * 4, [10] * (n_sets + 1), [(i % (n_sets + 1), 0) for i in range(n_sets + 1)])
    assert L.lobe_batch_sizes(ctypes.byref(cfg), ctypes.byref(b), out) == A.ERR_ARG
