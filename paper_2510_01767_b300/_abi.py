"""ctypes mirror of include/lobe.h and the loader of liblobe.so.

Argument marshalling only: every stage runs inside the CUDA library. Importing this module
does not touch the GPU; the first call to :func:`lib` loads liblobe.so and raises if it is
missing, so there is no silent fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblobe.so")

MAX_SETS = 16
MAX_ITEMS = 64

OK, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_OOM, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {OK: "OK", ERR_ARG: "ARG", ERR_CAPACITY: "CAPACITY", ERR_CUDA: "CUDA", ERR_TIMEOUT: "TIMEOUT",
                ERR_OOM: "OOM", ERR_STATE: "STATE"}

c_float_p = ctypes.POINTER(ctypes.c_float)
vp = ctypes.c_void_p


class Gaussians(ctypes.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp), ("sh", vp),
                ("crop_mask", vp), ("n", ctypes.c_int64)]


class Camera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_plane", ctypes.c_float), ("far_plane", ctypes.c_float)]


class AABB(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class Item(ctypes.Structure):
    _fields_ = [("set", ctypes.c_int32), ("camera", ctypes.c_int32), ("block", ctypes.c_int32)]


class Batch(ctypes.Structure):
    _fields_ = [("sets", ctypes.POINTER(Gaussians)), ("n_sets", ctypes.c_int32),
                ("cameras", ctypes.POINTER(Camera)), ("n_cameras", ctypes.c_int32),
                ("blocks", ctypes.POINTER(AABB)), ("n_blocks", ctypes.c_int32),
                ("items", ctypes.POINTER(Item)), ("n_items", ctypes.c_int32)]


class BoxD(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class KdParams(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("tau", ctypes.c_double), ("q_lo", ctypes.c_double),
                ("q_hi", ctypes.c_double), ("steps", ctypes.c_int32)]


RATIO_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(BoxD), ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_double))


class Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("bg", ctypes.c_float * 3), ("recompute_T", ctypes.c_int32), ("px_fwd", ctypes.c_int32),
                ("px_bwd", ctypes.c_int32), ("bin_general", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("batch_fwd", ctypes.c_int32), ("batch_bwd", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Projected(ctypes.Structure):
    _fields_ = [("splat", vp), ("radius", vp), ("tiles_touched", vp)]


class Bins(ctypes.Structure):
    _fields_ = [("gauss_ids", vp), ("tile_start", vp), ("n_isect", vp), ("capacity", ctypes.c_int64)]


class Image(ctypes.Structure):
    _fields_ = [("rgb", vp), ("T_final", vp), ("n_contrib", vp)]


class Grads(ctypes.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp), ("sh", vp),
                ("sd_acc", vp), ("sd_cnt", vp)]


class DensifyParams(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("max_clone_log_scale", ctypes.c_float),
                ("prune_logit", ctypes.c_float), ("n_split", ctypes.c_int32), ("split_log_shrink", ctypes.c_float)]


class ParamsOut(ctypes.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp), ("sh", vp),
                ("capacity", ctypes.c_int64)]


class ParamArrays(ctypes.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp), ("sh", vp)]


class AdamParams(ctypes.Structure):
    _fields_ = [("lr_means", ctypes.c_float), ("lr_log_scales", ctypes.c_float), ("lr_quats", ctypes.c_float),
                ("lr_opacity", ctypes.c_float), ("lr_sh_dc", ctypes.c_float), ("lr_sh_rest", ctypes.c_float),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_float),
                ("step", ctypes.c_int64)]


class AdamState(ctypes.Structure):
    _fields_ = [("param", ParamArrays), ("exp_avg", ParamArrays), ("exp_avg_sq", ParamArrays)]


# name -> (restype, argtypes); the exported symbols of liblobe.so (checked by the tests)
SIGNATURES = {
    "lobe_abi_version": (ctypes.c_int32, []),
    "lobe_peak_probe": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp]),
    "lobe_sync_status": (ctypes.c_int, [vp]),
    "lobe_kd_partition": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.POINTER(BoxD), ctypes.c_int32, RATIO_FN, vp,
                                         ctypes.POINTER(KdParams), ctypes.POINTER(BoxD), vp]),
    "lobe_fcs_select": (ctypes.c_int, [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp, vp]),
    "lobe_kernel_launches": (ctypes.c_int64, []),
    "lobe_batch_sizes": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Batch), ctypes.POINTER(ctypes.c_int64)]),
    "lobe_ctx_create": (ctypes.c_int, [ctypes.POINTER(vp), vp, ctypes.POINTER(Config)]),
    "lobe_ctx_destroy": (ctypes.c_int, [vp]),
    "lobe_ctx_set_stream": (ctypes.c_int, [vp, vp]),
    "lobe_ctx_set_config": (ctypes.c_int, [vp, ctypes.POINTER(Config)]),
    "lobe_last_error": (ctypes.c_char_p, [vp]),
    "lobe_ctx_reserve": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]),
    "lobe_get_status": (ctypes.c_int, [vp]),
    "lobe_project": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected)]),
    "lobe_bin_sort": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected), ctypes.POINTER(Bins),
                                     ctypes.POINTER(ctypes.c_int64)]),
    "lobe_bin_sort_noalloc": (ctypes.c_int, [ctypes.POINTER(Config), vp, ctypes.POINTER(Batch),
                                             ctypes.POINTER(Projected), ctypes.POINTER(Bins),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "lobe_render_fwd": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected), ctypes.POINTER(Bins),
                                       ctypes.POINTER(Image)]),
    "lobe_render_bwd": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected), ctypes.POINTER(Bins),
                                       ctypes.POINTER(Image), vp, vp]),
    "lobe_project_bwd": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected), vp,
                                        ctypes.POINTER(Grads), ctypes.c_int32]),
    "lobe_visibility_crop": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(vp)]),
    "lobe_densify": (ctypes.c_int, [vp, ctypes.POINTER(Gaussians), vp, vp, vp, ctypes.POINTER(DensifyParams),
                                    ctypes.POINTER(ParamsOut), vp, ctypes.POINTER(ctypes.c_int64)]),
    "lobe_render_depth": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected), ctypes.POINTER(Bins),
                                         ctypes.POINTER(Image), vp]),
    "lobe_fcs_coverage": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Image), vp, ctypes.POINTER(AABB),
                                         ctypes.c_int32, ctypes.c_int32, vp, vp]),
    "lobe_selftest_wait": (ctypes.c_int, [vp]),
    "lobe_adam": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.POINTER(AdamState), ctypes.POINTER(ParamArrays), vp,
                                 ctypes.POINTER(AdamParams)]),
    "lobe_project_bwd_adam": (ctypes.c_int, [vp, ctypes.POINTER(Batch), ctypes.POINTER(Projected), vp,
                                             ctypes.POINTER(Grads), ctypes.POINTER(AdamState),
                                             ctypes.POINTER(AdamParams), ctypes.c_int32]),
}

_lib = None


class LobeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lobe {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Loads liblobe.so (raising if it was not built) and declares its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2510_01767_b300.build` "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code, ctx=None):
    if code != OK:
        msg = lib().lobe_last_error(ctx).decode() if ctx else ""
        raise LobeError(code, msg)
