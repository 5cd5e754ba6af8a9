"""Batched multi-view, multi-block forward + backward in one CUDA graph, and its autotuner.

A ``BatchedStep`` owns every buffer of one training step over a batch of items (many views
of uneven resolution across several KD-tree blocks of uneven Gaussian counts): projection
(one thread per Gaussian of a set, looping over that set's views), binning of all items'
tiles in one global tile space, compositing of all tiles of all items in one launch,
the adjoint, and the per-set parameter gradients summed over views in registers. Because
the binning scratch is reserved up front and no stage synchronises with the host, the whole
step is captured once in a CUDA graph and replayed as a single launch.

``autotune`` picks the tile shape (8x8, 16x8, 16x16, 32x16), the pixels each lane composites (a
kernel knob: fewer means more warps per tile, more means fewer splat loads and reductions per
pixel), whether the composite and its adjoint run as persistent kernels that take tiles
longest list first, and the per-tile staging batch (32 or 64 splats of the tile's list fetched by
a warp per round), by timing graph replays on the actual batch; results are cached per (GPU,
batch signature) in ``~/.cache/lobe/autotune.json``.
``PlainSteps`` is the reference it is compared with: one view per call sequence, eager,
each view projecting its block's Gaussians itself.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import torch

from . import raster as R

TILES = ((8, 8), (16, 8), (16, 16), (32, 16))
PX_OPTIONS = {(8, 8): (1, 2), (16, 8): (1, 2, 4), (16, 16): (2, 4, 8), (32, 16): (2, 4, 8)}  # pixels per lane per tile shape
BATCH_OPTIONS = (32, 64)  # splats a warp stages from its tile's list per round


def config_name(tile, px=(0, 0), batch=(0, 0)):
    nb = tuple(n or 32 for n in batch) if batch else (32, 32)
    return (f"{tile[0]}x{tile[1]}" + (f"/f{px[0]}b{px[1]}" if px and px[0] else "") +
            (f"/s{nb[0]}.{nb[1]}" if nb != (32, 32) else ""))
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "lobe", "autotune.json")


class BatchedStep:
    def __init__(self, sets, cameras, items, blocks=(), tile=(16, 16), sh_degree=3, bg=(0.0, 0.0, 0.0),
                 recompute_T=False, slack=1.25, stream=None, px=(0, 0), persistent=False, batch=(0, 0)):
        self.stream = stream if stream is not None else torch.cuda.Stream()
        px = (px, px) if isinstance(px, int) else tuple(px)
        batch = (batch, batch) if isinstance(batch, int) else tuple(batch)
        self.ctx = R.Context(tile=tile, sh_degree=sh_degree, bg=bg, recompute_T=recompute_T, stream=self.stream,
                             px_fwd=px[0], px_bwd=px[1], persistent=persistent, batch=batch)
        self.px = px
        self.batch_size = batch
        self.batch_times = None
        self.persistent = bool(persistent)
        self.batch = R.Batch(sets, cameras, items, blocks)
        self.tile = tuple(tile)
        with torch.cuda.stream(self.stream):
            proj, bins, _ = R.forward(self.ctx, self.batch, sync=True)
            self.n_isect = bins.count
            n_tiles, _ = self.batch.tiles(self.tile)
            cap = int(self.n_isect * slack) + 4096
            self.ctx.reserve(self.batch.n_entries, cap, n_tiles)
            self.proj = proj
            self.bins = R.empty_bins(cap, n_tiles)
            self.image = R.empty_image(self.batch.n_pixels)
            self.grad2d = torch.empty((self.batch.n_entries, 12), dtype=torch.float32, device="cuda")
            self.grads = R.zero_grads(self.batch, sd=True)
            self.dL = torch.zeros(3 * self.batch.n_pixels, dtype=torch.float32, device="cuda")
        self.stream.synchronize()
        self.graph = None

    # one step, every stage enqueued on self.stream, no host synchronisation
    def run(self):
        c, b = self.ctx, self.batch
        R.project(c, b, self.proj)
        R.bin_sort(c, b, self.proj, self.bins, sync=False)
        R.render_fwd(c, b, self.proj, self.bins, self.image)
        R.render_bwd(c, b, self.proj, self.bins, self.image, self.dL, self.grad2d)
        R.project_bwd(c, b, self.proj, self.grad2d, self.grads, accumulate=False)

    def tune_px(self, options, reps=3):
        """Times the composite and its adjoint at each pixels-per-lane option and keeps the
        fastest for each (they are independent knobs). Returns (fwd, bwd)."""
        c, b = self.ctx, self.batch
        best = {}
        with torch.cuda.stream(self.stream):
            self.run()
            for px in options:
                c.configure(px=(px, px))
                fwd = _time(lambda: R.render_fwd(c, b, self.proj, self.bins, self.image), reps, self.stream)
                bwd = _time(lambda: R.render_bwd(c, b, self.proj, self.bins, self.image, self.dL, self.grad2d), reps,
                            self.stream)
                if fwd < best.get("f", (float("inf"), 0))[0]:
                    best["f"] = (fwd, px)
                if bwd < best.get("b", (float("inf"), 0))[0]:
                    best["b"] = (bwd, px)
        self.px = (best["f"][1], best["b"][1])
        c.configure(px=self.px)
        return self.px

    def tune_batch(self, options=BATCH_OPTIONS, reps=3):
        """Times the composite and its adjoint at each staging batch (splats a warp fetches from
        its tile's list per round) and keeps the fastest for each; a size the library rejects for
        this configuration (64 needs two or more pixels a lane, an even count in the adjoint) is
        skipped. Returns (fwd, bwd)."""
        c, b = self.ctx, self.batch
        best = {"f": (float("inf"), 32), "b": (float("inf"), 32)}
        self.batch_times = {"fwd": {}, "bwd": {}}  # ms of the composite / adjoint per staging batch

        def settable(batch):
            old = c.batch
            try:
                c.configure(batch=batch)
                return True
            except R.A.LobeError:
                c.batch = old
                return False

        with torch.cuda.stream(self.stream):
            self.run()
            for n in options:
                if settable((n, 32)):
                    fwd = _time(lambda: R.render_fwd(c, b, self.proj, self.bins, self.image), reps, self.stream)
                    self.batch_times["fwd"][n] = round(fwd, 4)
                    if fwd < best["f"][0]:
                        best["f"] = (fwd, n)
                if settable((32, n)):
                    bwd = _time(lambda: R.render_bwd(c, b, self.proj, self.bins, self.image, self.dL, self.grad2d),
                                reps, self.stream)
                    self.batch_times["bwd"][n] = round(bwd, 4)
                    if bwd < best["b"][0]:
                        best["b"] = (bwd, n)
        self.set_batch((best["f"][1], best["b"][1]))
        return self.batch_size

    def set_batch(self, batch):
        """Set the staging batch (fwd, bwd) of the composite and its adjoint (drops a captured graph)."""
        self.batch_size = tuple(batch)
        self.ctx.configure(batch=self.batch_size)
        self.graph = None

    def set_persistent(self, on):
        """Switch the composite and its adjoint between one block per tile and persistent
        kernels taking tiles longest list first (drops a captured graph)."""
        self.persistent = bool(on)
        self.ctx.configure(persistent=self.persistent)
        self.graph = None

    def capture(self, warmup=2):
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                self.run()
        self.stream.synchronize()
        self.ctx.status()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.run()
        self.graph = g
        return self

    def replay(self):
        if self.graph is None:
            raise RuntimeError("call capture() first")
        with torch.cuda.stream(self.stream):  # replay is enqueued on the current stream
            self.graph.replay()

    def images(self):
        return self.batch.image_views(self.image.rgb)

    def dL_views(self):
        return self.batch.image_views(self.dL)


class PlainSteps:
    """The one-view-per-call reference: each item is its own batch, run eagerly in turn."""

    def __init__(self, sets, cameras, items, blocks=(), tile=(16, 16), **kw):
        self.steps = []
        for s, c, b in items:
            bl = [blocks[b]] if b >= 0 and blocks else []
            self.steps.append(BatchedStep([sets[s]], [cameras[c]], [(0, 0, 0 if bl else -1)], bl, tile=tile,
                                          stream=torch.cuda.current_stream(), **kw))

    def run(self):
        for st in self.steps:
            st.run()


def _time(fn, reps, stream):
    fn()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def signature(sets, cameras, items):
    h = hashlib.sha1()
    h.update(repr([s.n for s in sets]).encode())
    h.update(repr([(c["width"], c["height"]) if isinstance(c, dict) else (c.width, c.height) for c in cameras]).encode())
    h.update(repr(items).encode())
    return h.hexdigest()[:16]


def autotune(sets, cameras, items, blocks=(), tiles=TILES, reps=5, use_cache=True, dL_init=None, tune_px=True,
             **kw):
    """Returns (best BatchedStep captured in a graph, {"<tile>/f<px>b<px>": ms per step}): per tile
    shape, the pixels per lane of the composite and of its adjoint are tuned separately, then
    the whole step is timed as a graph replay."""
    key = f"{torch.cuda.get_device_name()}|{signature(sets, cameras, items)}|{config_name_list(tiles)}|{int(tune_px)}"
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        tile, px = tuple(cache[key]["tile"]), tuple(cache[key].get("px", (0, 0)))
        st = BatchedStep(sets, cameras, items, blocks, tile=tile, px=px, persistent=cache[key].get("persistent", False),
                         batch=tuple(cache[key].get("batch", (0, 0))), **kw)
        if dL_init is not None:
            dL_init(st)
        return st.capture(), cache[key]["times"]
    times, best, best_ms = {}, None, float("inf")
    for tile in tiles:
        tile = tuple(tile)
        st = BatchedStep(sets, cameras, items, blocks, tile=tile, **kw)
        if dL_init is not None:
            dL_init(st)
        if tune_px:
            st.tune_px(PX_OPTIONS.get(tile, (0,)), reps=max(2, reps // 2))
        st.capture()
        ms = _time(st.replay, reps, st.stream)
        times[config_name(tile, st.px)] = ms
        if ms < best_ms:
            if best is not None:
                del best
            best, best_ms = st, ms
        else:
            del st
        torch.cuda.empty_cache()
    # the winner once more with persistent compositing (tiles longest list first)
    best.set_persistent(True)
    best.capture()
    ms = _time(best.replay, reps, best.stream)
    times[config_name(best.tile, best.px) + "/persistent"] = ms
    if ms >= best_ms:
        best.set_persistent(False)
        best.capture()
    else:
        best_ms = ms
    # then the staging batch of the composite and of its adjoint, kept if the whole step is faster
    if tune_px:
        nb = best.tune_batch(reps=max(2, reps // 2))
        if nb != (32, 32):
            best.capture()
            ms = _time(best.replay, reps, best.stream)
            times[config_name(best.tile, best.px, nb) + ("/persistent" if best.persistent else "")] = ms
            if ms >= best_ms:
                best.set_batch((32, 32))
                best.capture()
        else:
            best.set_batch((32, 32))
            best.capture()
    if use_cache:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        cache[key] = {"tile": list(best.tile), "px": list(best.px), "persistent": best.persistent,
                      "batch": list(best.batch_size), "times": times, "when": time.time()}
        with open(CACHE, "w") as f:
            json.dump(cache, f)
    return best, times


def config_name_list(tiles):
    return ",".join(f"{t[0]}x{t[1]}" for t in tiles)
