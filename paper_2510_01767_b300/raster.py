"""Python binding of the C ABI: the same stages as include/lobe.h, on torch CUDA tensors.

PyTorch supplies device memory and the stream; every stage runs in liblobe.so. The names
mirror the C entry points: :func:`project`, :func:`bin_sort`, :func:`render_fwd`,
:func:`render_bwd`, :func:`project_bwd`, :func:`visibility_crop`.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import torch

from . import _abi as A

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _require_cuda(t: torch.Tensor, name: str, dtype=torch.float32):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclass
class GaussianSet:
    """Device parameters of one Gaussian set (float32, contiguous)."""
    means: torch.Tensor           # [n,3]
    log_scales: torch.Tensor      # [n,3]
    quats: torch.Tensor           # [n,4] (w,x,y,z)
    opacity_logits: torch.Tensor  # [n]
    sh: torch.Tensor              # [n,16,3]
    crop_mask: torch.Tensor | None = None  # [n] uint8

    @property
    def n(self):
        return int(self.means.shape[0])

    @classmethod
    def from_numpy(cls, g, device="cuda"):
        a = g.arrays() if hasattr(g, "arrays") else g
        t = {k: torch.as_tensor(a[k], dtype=torch.float32).contiguous().to(device) for k in PARAM_KEYS}
        crop = getattr(g, "crop_mask", None)
        if crop is not None:
            crop = torch.as_tensor(crop, dtype=torch.uint8).to(device)
        return cls(**t, crop_mask=crop)

    def params(self):
        return [getattr(self, k) for k in PARAM_KEYS]


def camera_struct(cam) -> A.Camera:
    c = cam if isinstance(cam, dict) else cam.as_dict()
    s = A.Camera()
    vm = [float(x) for x in torch.as_tensor(c["viewmat"], dtype=torch.float32).reshape(16).tolist()]
    s.viewmat[:] = vm
    s.fx, s.fy, s.cx, s.cy = float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"])
    s.width, s.height = int(c["width"]), int(c["height"])
    s.near_plane, s.far_plane = float(c.get("near", 0.01)), float(c.get("far", 1e10))
    return s


def aabb_struct(box) -> A.AABB:
    s = A.AABB()
    lo = getattr(box, "lo", None) if box is not None else None
    hi = getattr(box, "hi", None) if box is not None else None
    s.lo[:] = [float(x) for x in (lo if lo is not None else (-math.inf,) * 3)]
    s.hi[:] = [float(x) for x in (hi if hi is not None else (math.inf,) * 3)]
    return s


class Batch:
    """Host description of a batch of (set, camera, block) items (a lobe_batch)."""

    def __init__(self, sets, cameras, items, blocks=()):
        if len(sets) > A.MAX_SETS or len(items) > A.MAX_ITEMS:
            raise ValueError("too many sets or items for one batch")
        self.sets = list(sets)
        self.cameras = [c if isinstance(c, dict) else c.as_dict() for c in cameras]
        self.blocks = list(blocks)
        self.items = [tuple(int(x) for x in it) for it in items]
        for g in self.sets:
            for k in PARAM_KEYS:
                _require_cuda(getattr(g, k), k)
            if g.crop_mask is not None:
                _require_cuda(g.crop_mask, "crop_mask", torch.uint8)
        self._c_sets = (A.Gaussians * len(self.sets))()
        for i, g in enumerate(self.sets):
            s = self._c_sets[i]
            s.means, s.log_scales, s.quats = g.means.data_ptr(), g.log_scales.data_ptr(), g.quats.data_ptr()
            s.opacity_logits, s.sh = g.opacity_logits.data_ptr(), g.sh.data_ptr()
            s.crop_mask = g.crop_mask.data_ptr() if g.crop_mask is not None else None
            s.n = g.n
        self._c_cams = (A.Camera * len(self.cameras))(*[camera_struct(c) for c in self.cameras])
        nb = max(1, len(self.blocks))
        self._c_blocks = (A.AABB * nb)(*([aabb_struct(b) for b in self.blocks] or [aabb_struct(None)]))
        self._c_items = (A.Item * len(self.items))(*[A.Item(s, c, b) for s, c, b in self.items])
        self.c = A.Batch(self._c_sets, len(self.sets), self._c_cams, len(self.cameras), self._c_blocks,
                         len(self.blocks), self._c_items, len(self.items))
        # host-side layout (mirrors the library's offsets)
        self.entry_off, self.pix_off = [], []
        e = p = 0
        for s, c, _ in self.items:
            self.entry_off.append(e)
            self.pix_off.append(p)
            e += self.sets[s].n
            p += self.cameras[c]["width"] * self.cameras[c]["height"]
        self.n_entries, self.n_pixels = e, p

    def tiles(self, tile):
        t = 0
        offs = []
        for _, c, _ in self.items:
            cam = self.cameras[c]
            offs.append(t)
            t += -(-cam["width"] // tile[0]) * -(-cam["height"] // tile[1])
        return t, offs

    def image_views(self, flat: torch.Tensor, channels=3):
        """Split a flat planar image buffer into per-item [C,H,W] views."""
        out = []
        for (s, c, _), p in zip(self.items, self.pix_off):
            cam = self.cameras[c]
            W, H = cam["width"], cam["height"]
            out.append(flat[channels * p: channels * (p + W * H)].view(channels, H, W) if channels > 1
                       else flat[p: p + W * H].view(H, W))
        return out


class Context:
    """A lobe_ctx bound to a CUDA stream (the current torch stream by default)."""

    def __init__(self, tile=(16, 16), sh_degree=3, bg=(0.0, 0.0, 0.0), recompute_T=False, stream=None, px_fwd=0,
                 px_bwd=0, bin_general=False, persistent=False, batch=(0, 0)):
        if not torch.cuda.is_available():
            raise RuntimeError("the lobe rasterizer needs a CUDA device (no CPU fallback)")
        self.lib = A.lib()
        self.tile = tuple(tile)
        self.sh_degree = sh_degree
        self.bg = tuple(float(b) for b in bg)
        self.recompute_T = bool(recompute_T)
        self.px = (int(px_fwd), int(px_bwd))
        self.bin_general = bool(bin_general)  # never the one-CTA binning of small batches
        self.persistent = bool(persistent)  # compositing as persistent kernels, tiles longest list first
        self.batch = (int(batch[0]), int(batch[1]))  # splats a warp stages per round (fwd, bwd): 0/32 or 64
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = ctypes.c_void_p()
        A.check(self.lib.lobe_ctx_create(ctypes.byref(self.handle), ctypes.c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(self._config())))
        self._bins = None

    def _config(self) -> A.Config:
        c = A.Config()
        c.tile_w, c.tile_h = self.tile
        c.sh_degree = self.sh_degree
        c.bg[:] = list(self.bg)
        c.recompute_T = int(self.recompute_T)
        c.px_fwd, c.px_bwd = self.px
        c.bin_general = int(self.bin_general)
        c.persistent = int(self.persistent)
        c.batch_fwd, c.batch_bwd = self.batch
        return c

    def configure(self, tile=None, recompute_T=None, sh_degree=None, bg=None, px=None, persistent=None, batch=None):
        """Change the configuration (tile changes need new bins; px = (fwd, bwd) pixels per lane;
        batch = (fwd, bwd) splats a warp stages per round)."""
        if persistent is not None:
            self.persistent = bool(persistent)
        if batch is not None:
            self.batch = (int(batch[0]), int(batch[1]))
        if px is not None:
            self.px = (int(px[0]), int(px[1]))
        if tile is not None:
            self.tile = tuple(tile)
        if recompute_T is not None:
            self.recompute_T = bool(recompute_T)
        if sh_degree is not None:
            self.sh_degree = sh_degree
        if bg is not None:
            self.bg = tuple(float(b) for b in bg)
        self._check(self.lib.lobe_ctx_set_config(self.handle, ctypes.byref(self._config())))

    def set_stream(self, stream):
        self.stream = stream
        self._check(self.lib.lobe_ctx_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))

    def reserve(self, max_entries, max_isect, max_tiles):
        self._check(self.lib.lobe_ctx_reserve(self.handle, int(max_entries), int(max_isect), int(max_tiles)))

    def status(self):
        self._check(self.lib.lobe_get_status(self.handle))

    def _check(self, code):
        A.check(code, self.handle)

    def close(self):
        if self.handle:
            self.lib.lobe_ctx_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- stage outputs

@dataclass
class Projection:
    splat: torch.Tensor   # [E,12] float32
    radius: torch.Tensor  # [E] int32
    tiles: torch.Tensor   # [E] int32

    def c(self):
        return A.Projected(self.splat.data_ptr(), self.radius.data_ptr(), self.tiles.data_ptr())


@dataclass
class Bins:
    gauss_ids: torch.Tensor   # [capacity] int32
    tile_start: torch.Tensor  # [n_tiles+1] int32
    n_isect: torch.Tensor     # [1] int64
    count: int | None = None  # host copy when known

    @property
    def capacity(self):
        return int(self.gauss_ids.shape[0])

    def c(self):
        return A.Bins(self.gauss_ids.data_ptr(), self.tile_start.data_ptr(), self.n_isect.data_ptr(), self.capacity)

    def ids(self):
        n = self.count if self.count is not None else int(self.n_isect.item())
        return self.gauss_ids[:n]


@dataclass
class Image:
    rgb: torch.Tensor        # [3*pixels] float32 (planar per item)
    T_final: torch.Tensor    # [pixels]
    n_contrib: torch.Tensor  # [pixels] int32

    def c(self):
        return A.Image(self.rgb.data_ptr(), self.T_final.data_ptr(), self.n_contrib.data_ptr())


def empty_projection(n_entries, device="cuda") -> Projection:
    return Projection(torch.empty((n_entries, 12), dtype=torch.float32, device=device),
                      torch.empty(n_entries, dtype=torch.int32, device=device),
                      torch.empty(n_entries, dtype=torch.int32, device=device))


def empty_bins(capacity, n_tiles, device="cuda") -> Bins:
    return Bins(torch.empty(max(1, int(capacity)), dtype=torch.int32, device=device),
                torch.empty(n_tiles + 1, dtype=torch.int32, device=device),
                torch.zeros(1, dtype=torch.int64, device=device))


def empty_image(n_pixels, device="cuda") -> Image:
    return Image(torch.empty(3 * n_pixels, dtype=torch.float32, device=device),
                 torch.empty(n_pixels, dtype=torch.float32, device=device),
                 torch.empty(n_pixels, dtype=torch.int32, device=device))


# --------------------------------------------------------------------------- stages

def project(ctx: Context, batch: Batch, out: Projection | None = None) -> Projection:
    out = out if out is not None else empty_projection(batch.n_entries)
    ctx._check(ctx.lib.lobe_project(ctx.handle, ctypes.byref(batch.c), ctypes.byref(out.c())))
    return out


def bin_sort(ctx: Context, batch: Batch, proj: Projection, bins: Bins | None = None, sync: bool = True) -> Bins:
    """Sorts all (splat, tile) pairs. With sync=True the pair count is read back and the bins
    grow as needed (not graph-capturable); with sync=False the given bins must be large enough
    (an overflow is latched on the device and read by Context.status())."""
    n_tiles, _ = batch.tiles(ctx.tile)
    if bins is None:
        bins = ctx._bins
        if bins is None or bins.tile_start.shape[0] != n_tiles + 1:
            cap = bins.capacity if bins is not None else max(1 << 16, 8 * batch.n_entries)
            bins = empty_bins(cap, n_tiles)
    if not sync:
        ctx._check(ctx.lib.lobe_bin_sort(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()),
                                         ctypes.byref(bins.c()), None))
        bins.count = None
        return bins
    n = ctypes.c_int64(0)
    code = ctx.lib.lobe_bin_sort(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()), ctypes.byref(bins.c()),
                                 ctypes.byref(n))
    if code == A.ERR_CAPACITY:
        bins = empty_bins(int(n.value * 1.25) + 1024, n_tiles)
        code = ctx.lib.lobe_bin_sort(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()),
                                     ctypes.byref(bins.c()), ctypes.byref(n))
    ctx._check(code)
    bins.count = int(n.value)
    ctx._bins = bins
    return bins


def render_fwd(ctx: Context, batch: Batch, proj: Projection, bins: Bins, out: Image | None = None) -> Image:
    out = out if out is not None else empty_image(batch.n_pixels)
    ctx._check(ctx.lib.lobe_render_fwd(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()),
                                       ctypes.byref(bins.c()), ctypes.byref(out.c())))
    return out


def render_depth(ctx: Context, batch: Batch, proj: Projection, bins: Bins, out: Image | None = None,
                 depth: torch.Tensor | None = None):
    """render_fwd plus the composite depth of fast camera selection (Sec. 3.2): returns
    (image, depth[pixels]) with depth = sum_i d_i alpha_i T_i per pixel."""
    out = out if out is not None else empty_image(batch.n_pixels)
    depth = depth if depth is not None else torch.empty(batch.n_pixels, dtype=torch.float32, device="cuda")
    ctx._check(ctx.lib.lobe_render_depth(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()),
                                         ctypes.byref(bins.c()), ctypes.byref(out.c()), _ptr(depth)))
    return out, depth


def fcs_coverage(ctx: Context, batch: Batch, image: Image, depth: torch.Tensor, blocks, normalize=False):
    """Fast camera selection (Sec. 3.2): counts[item, block] of back-projected depth points
    inside each block box and n_points[item] (pixels some splat reached). The visibility
    ratio is V = counts / n_points."""
    blocks = list(blocks)
    arr = (A.AABB * max(1, len(blocks)))()
    for i, b in enumerate(blocks):
        arr[i] = aabb_struct(b)
    n_items = len(batch.items)
    counts = torch.empty((n_items, max(1, len(blocks))), dtype=torch.int32, device="cuda")
    npts = torch.empty(n_items, dtype=torch.int32, device="cuda")
    ctx._check(ctx.lib.lobe_fcs_coverage(ctx.handle, ctypes.byref(batch.c), ctypes.byref(image.c()), _ptr(depth), arr,
                                         len(blocks), int(bool(normalize)), _ptr(counts), _ptr(npts)))
    return counts[:, :len(blocks)], npts


def densify(ctx: Context, g: GaussianSet, sd_acc: torch.Tensor, sd_cnt: torch.Tensor, normals: torch.Tensor | None = None,
            grad_threshold=2e-4, percent_dense=0.01, scene_extent=1.0, min_opacity=0.005, n_split=2,
            generator: torch.Generator | None = None):
    """Selective densification (Sec. 3.3) with the 3DGS density control: returns (the new
    GaussianSet, source index of every output Gaussian). Gaussians outside the block have
    sd_cnt = 0 and never clone or split. ``normals`` [n, n_split, 3] are the split children's
    standard normal draws (drawn here from ``generator`` when not given)."""
    n = g.n
    if normals is None:
        normals = torch.randn((n, n_split, 3), device="cuda", generator=generator)
    _require_cuda(normals, "normals")
    _require_cuda(sd_acc, "sd_acc")
    _require_cuda(sd_cnt, "sd_cnt", torch.int32)
    prm = A.DensifyParams(float(grad_threshold), float(math.log(percent_dense * scene_extent)),
                          float(math.log(min_opacity / (1 - min_opacity))), int(n_split), float(math.log(0.8 * n_split)))
    src = A.Gaussians(g.means.data_ptr(), g.log_scales.data_ptr(), g.quats.data_ptr(), g.opacity_logits.data_ptr(),
                      g.sh.data_ptr(), None, n)
    cap = n * max(2, n_split)
    out = {k: torch.empty((cap,) + tuple(getattr(g, k).shape[1:]), dtype=torch.float32, device="cuda")
           for k in PARAM_KEYS}
    source = torch.empty(cap, dtype=torch.int32, device="cuda")
    po = A.ParamsOut(out["means"].data_ptr(), out["log_scales"].data_ptr(), out["quats"].data_ptr(),
                     out["opacity_logits"].data_ptr(), out["sh"].data_ptr(), cap)
    n_out = ctypes.c_int64(0)
    ctx._check(ctx.lib.lobe_densify(ctx.handle, ctypes.byref(src), _ptr(sd_acc), _ptr(sd_cnt), _ptr(normals),
                                    ctypes.byref(prm), ctypes.byref(po), _ptr(source), ctypes.byref(n_out)))
    m = int(n_out.value)
    return GaussianSet(**{k: v[:m].contiguous() for k, v in out.items()}), source[:m]


# learning rates of the 3DGS procedure (means: times the scene extent, decayed by the caller)
ADAM_LR_3DGS = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20)


def _arrays(d) -> A.ParamArrays:
    get = (lambda k: getattr(d, k)) if isinstance(d, GaussianSet) else (lambda k: d[k])
    for k in PARAM_KEYS:
        _require_cuda(get(k), k)
    return A.ParamArrays(*(get(k).data_ptr() for k in PARAM_KEYS))


class Adam:
    """Adam state of one Gaussian set: the two moment buffers in the set's layout, the
    per-group learning rates (ADAM_LR_3DGS keys) and the step count. ``step`` applies an
    update from given gradients (lobe_adam); ``project_bwd_adam`` fuses it into the
    projection adjoint. The set's tensors are updated in place."""

    def __init__(self, g: GaussianSet, lr=None, betas=(0.9, 0.999), eps=1e-15):
        self.set = g
        self.lr = dict(ADAM_LR_3DGS if lr is None else lr)
        self.betas = (float(betas[0]), float(betas[1]))
        self.eps = float(eps)
        self.exp_avg = {k: torch.zeros_like(getattr(g, k)) for k in PARAM_KEYS}
        self.exp_avg_sq = {k: torch.zeros_like(getattr(g, k)) for k in PARAM_KEYS}
        self.t = 0

    def _state(self) -> A.AdamState:
        return A.AdamState(_arrays(self.set), _arrays(self.exp_avg), _arrays(self.exp_avg_sq))

    def _params(self, t) -> A.AdamParams:
        lr = self.lr
        return A.AdamParams(lr["means"], lr["log_scales"], lr["quats"], lr["opacity_logits"], lr["sh_dc"],
                            lr["sh_rest"], self.betas[0], self.betas[1], self.eps, int(t))

    def step(self, ctx: Context, grads: dict, rows: torch.Tensor | None = None):
        """One update from grads (dict of PARAM_KEYS tensors); with rows (uint8 [n]) only
        the rows marked nonzero change (sparse Adam)."""
        if rows is not None:
            _require_cuda(rows, "rows", torch.uint8)
        st, ga = self._state(), _arrays(grads)
        ctx._check(ctx.lib.lobe_adam(ctx.handle, self.set.n, ctypes.byref(st), ctypes.byref(ga), _ptr(rows),
                                     ctypes.byref(self._params(self.t + 1))))
        self.t += 1


def project_bwd_adam(ctx: Context, batch: Batch, proj: Projection, grad2d: torch.Tensor, optimizers, sd=None,
                     sparse: bool = False):
    """The projection adjoint fused with Adam: optimizers[s] (an Adam of batch.sets[s]) takes
    one step with the batch's gradients, which are never written out. sparse: only the
    Gaussians some item sees change; otherwise every Gaussian of every set does (standard
    Adam). sd: optional list of dicts with sd_acc / sd_cnt (accumulated)."""
    if len(optimizers) != len(batch.sets) or any(o.set is not g for o, g in zip(optimizers, batch.sets)):
        raise ValueError("one Adam per set of the batch, in order")
    _require_cuda(grad2d, "grad2d")
    states = (A.AdamState * len(optimizers))(*[o._state() for o in optimizers])
    prms = (A.AdamParams * len(optimizers))(*[o._params(o.t + 1) for o in optimizers])
    sdarr = None
    if sd is not None:
        sdarr = (A.Grads * len(batch.sets))()
        for i, d in enumerate(sd):
            sdarr[i].sd_acc = d["sd_acc"].data_ptr() if d.get("sd_acc") is not None else None
            sdarr[i].sd_cnt = d["sd_cnt"].data_ptr() if d.get("sd_cnt") is not None else None
    ctx._check(ctx.lib.lobe_project_bwd_adam(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()), _ptr(grad2d),
                                             sdarr, states, prms, int(bool(sparse))))
    for o in optimizers:
        o.t += 1


def fcs_select(counts: torch.Tensor, n_points: torch.Tensor, tau: float = 0.1):
    """The paper's assignment C(b) = {c : V(c, b) >= tau}: returns (V [items, blocks], list of
    item indices per block)."""
    import numpy as np
    c = np.ascontiguousarray(counts.detach().cpu().numpy(), dtype=np.uint32)
    n = np.ascontiguousarray(n_points.detach().cpu().numpy(), dtype=np.uint32)
    items, blocks = c.shape
    V = np.zeros((items, blocks), np.float64)
    assign = np.zeros((items, blocks), np.uint8)
    A.check(A.lib().lobe_fcs_select(c.ctypes.data, n.ctypes.data, items, blocks, float(tau), V.ctypes.data,
                                    assign.ctypes.data))
    return torch.as_tensor(V), [np.nonzero(assign[:, b])[0].tolist() for b in range(blocks)]


def render_bwd(ctx: Context, batch: Batch, proj: Projection, bins: Bins, image: Image | None,
               dL_drgb: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    _require_cuda(dL_drgb, "dL_drgb")
    out = out if out is not None else torch.empty((batch.n_entries, 12), dtype=torch.float32, device="cuda")
    img = ctypes.byref(image.c()) if image is not None else None
    ctx._check(ctx.lib.lobe_render_bwd(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()),
                                       ctypes.byref(bins.c()), img, _ptr(dL_drgb), _ptr(out)))
    return out


def zero_grads(batch: Batch, sd=True):
    out = []
    for g in batch.sets:
        d = {k: torch.zeros_like(getattr(g, k)) for k in PARAM_KEYS}
        if sd:
            d["sd_acc"] = torch.zeros(g.n, dtype=torch.float32, device="cuda")
            d["sd_cnt"] = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        out.append(d)
    return out


def project_bwd(ctx: Context, batch: Batch, proj: Projection, grad2d: torch.Tensor, grads=None,
                accumulate: bool = False):
    """Parameter gradients per set (list of dicts with the PARAM_KEYS, plus optional
    sd_acc / sd_cnt which always accumulate)."""
    if grads is None:
        grads = []
        for g in batch.sets:
            d = {k: torch.empty_like(getattr(g, k)) for k in PARAM_KEYS}
            grads.append(d)
        accumulate = False
    arr = (A.Grads * len(batch.sets))()
    for i, d in enumerate(grads):
        s = arr[i]
        s.means, s.log_scales, s.quats = d["means"].data_ptr(), d["log_scales"].data_ptr(), d["quats"].data_ptr()
        s.opacity_logits, s.sh = d["opacity_logits"].data_ptr(), d["sh"].data_ptr()
        s.sd_acc = d["sd_acc"].data_ptr() if d.get("sd_acc") is not None else None
        s.sd_cnt = d["sd_cnt"].data_ptr() if d.get("sd_cnt") is not None else None
    ctx._check(ctx.lib.lobe_project_bwd(ctx.handle, ctypes.byref(batch.c), ctypes.byref(proj.c()), _ptr(grad2d),
                                        arr, int(bool(accumulate))))
    return grads


def visibility_crop(ctx: Context, batch: Batch, masks=None):
    """Visibility cropping (Sec. 3.3): per set, uint8 mask of Gaussians visible from at
    least one item of that set (OR-ed into ``masks`` when given)."""
    if masks is None:
        masks = [torch.zeros(g.n, dtype=torch.uint8, device="cuda") for g in batch.sets]
    arr = (ctypes.c_void_p * len(masks))(*[m.data_ptr() for m in masks])
    ctx._check(ctx.lib.lobe_visibility_crop(ctx.handle, ctypes.byref(batch.c), arr))
    return masks


def forward(ctx: Context, batch: Batch, sync=True):
    """project -> bin_sort -> render_fwd. Returns (proj, bins, image)."""
    proj = project(ctx, batch)
    bins = bin_sort(ctx, batch, proj, sync=sync)
    img = render_fwd(ctx, batch, proj, bins)
    return proj, bins, img
