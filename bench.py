#!/usr/bin/env python3
"""Throughput of the differentiable tile rasterizer: one step = project -> bin/sort ->
render fwd -> render bwd -> project bwd over every view of one synthetic batch (the
per-block training step's rasterizer pass; the loss gradient dL/dC is computed once before
timing, from L1 + 0.2 (1 - SSIM) against a render of a perturbed copy).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lobe|reference] [--workload NAME]

Default workload (the largest single-GPU configuration): four KD-tree blocks of a synthetic
city (0.5 / 1 / 2 / 3 M Gaussians), 16 views of uneven resolution (640x480 ... 1920x1080,
17.9 Mpx), 4 per block, all rendered forward and backward in one CUDA graph (tile shape and
pixels per lane autotuned on the batch). Prints ONE JSON line (rank 0). Under torchrun every
rank renders its own independent replica (a different seeded city): weak scaling, no
collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "fwd+bwd rasterization Mpix/s"
UNIT = "Mpix/s"
L2_BYTES = 126 * 2 ** 20
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")

# Algorithmic work per unit, counted from the operations the method needs (not the SIMT
# lanes a kernel happens to burn).
FLOP_FWD_PAIR = 19    # per (pixel, splat) pair up to the last contributor, FMA = 2 FLOP
FLOP_BWD_PAIR = 55
PARAM_BYTES = 236     # a Gaussian's parameters (59 floats)
PROJ_OUT_VISIBLE = 56  # splat record 48 B + radius + tile count
PROJ_OUT_CULLED = 8    # radius + tile count
PROJ_IN_CULLED = 44    # mean, scale, quaternion, logit: enough to cull
GRAD2D_BYTES = 48      # a 2D gradient record
SD_BYTES = 8           # SD statistic (acc, count)
SORT_BYTES_PAIR = 12 + 12 + 12 + 8  # per intersection for duplication + pair sort + ranges (key/value written,
#                                     read, sorted and written, range read); this binning moves fewer (see traffic)
WORKLOADS = ("multi", "medium", "small", "city", "multi_quarter")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lobe", choices=["lobe", "reference"])
    ap.add_argument("--workload", default="multi", choices=WORKLOADS)
    ap.add_argument("--tile", default="auto", help="WxH, or auto: tile shape and pixels per lane by the autotuner")
    ap.add_argument("--px", default="0,0", help="with --tile WxH: pixels per lane of the composite and its adjoint")
    ap.add_argument("--persistent", action="store_true", help="with --tile WxH: persistent compositing kernels")
    ap.add_argument("--batch", default="32,32", help="with --tile WxH: splats a warp stages per round in the "
                                                      "composite and its adjoint (32 or 64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the medium view, batched-vs-plain, fast camera "
                                                              "selection, densification, Adam and training measurements")
    ap.add_argument("--recompute", action="store_true")
    return ap.parse_args()


def build_workload(name, seed):
    if name == "small":
        return scenes.small_scene(seed=seed)
    if name == "medium":
        return scenes.medium_scene(seed=seed)
    if name == "city":
        return scenes.city_block_scene(seed=seed)
    if name == "multi_quarter":  # the batched workload at a quarter of the Gaussians (profiling size)
        wl = scenes.multi_block_scene(seed=seed, block_sizes=(125_000, 250_000, 500_000, 750_000))
        wl.name = "multi_block_quarter_4x_16views"
        return wl
    return scenes.multi_block_scene(seed=seed)


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi every 200 ms while running (the timed region)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first_sample(self, timeout=5.0):
        """nvidia-smi takes a moment to start: wait for its first line, then keep only the
        samples taken from now on (the timed region)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)
        self.lines.clear()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU baseline (oracle)
#
# The FP64 oracle (plain C, one thread a process) on 128x128 pixel windows of the workload's
# views: every Gaussian of the view's set projected, the window's tiles binned, composited and
# differentiated, then the projection adjoint of the whole set. Windows run in a pool of
# processes (spawn: started before any CUDA call is inherited) over the host's cores. The
# Gaussian sets are shared with the workers through .npy files read with mmap.

CPU_WIN = 128
CPU_MAX_PROCS = 32  # each worker widens its set to float64 (~0.5 GB for 1M Gaussians)


def _oracle_window_task(args):
    """One window: (seconds, pixels, gaussians)."""
    import oracle
    set_dir, s, cam, tile, box, x0, y0, seed = args
    g = {k: np.load(os.path.join(set_dir, f"set{s}_{k}.npy"), mmap_mode="r") for k in
         ("means", "log_scales", "quats", "opacity_logits", "sh")}
    g = oracle.set_dict(g)
    W, H = cam["width"], cam["height"]
    w = min(CPU_WIN, W, H)
    dL = np.zeros((3, H, W))
    dL[:, y0:y0 + w, x0:x0 + w] = np.random.default_rng(seed).standard_normal((3, w, w))
    t0 = time.perf_counter()
    with oracle.window(x0, y0, x0 + w, y0 + w):
        f = oracle.forward(g, cam, tile)
        oracle.backward(g, cam, f, dL, tile, aabb=box)
    return time.perf_counter() - t0, w * w, g["means"].shape[0]


class OracleSampler:
    """Oracle windows of one workload, run serially or over a process pool."""

    def __init__(self, wl, max_set=1_100_000):
        self.dir = tempfile.mkdtemp(prefix="lobe_oracle_sets_")
        self.tasks = []
        # the sets a worker can hold in float64 comfortably; each item of those, windows spread
        # over the view
        for s, gs in enumerate(wl.sets):
            if gs.n > max_set and len(wl.sets) > 1:
                continue
            for k, v in gs.arrays().items():
                np.save(os.path.join(self.dir, f"set{s}_{k}.npy"), v)
        rng = np.random.default_rng(0)
        for i, (s, c, b) in enumerate(wl.items):
            if not os.path.exists(os.path.join(self.dir, f"set{s}_means.npy")):
                continue
            cam = wl.cameras[c].as_dict()
            W, H = cam["width"], cam["height"]
            w = min(CPU_WIN, W, H)
            box = wl.blocks[b] if b >= 0 and wl.blocks else None
            for _ in range(8):
                self.tasks.append((self.dir, s, cam, tuple(wl.tile), box, int(rng.integers(0, W - w + 1)),
                                   int(rng.integers(0, H - w + 1)), len(self.tasks)))
        self.sets_used = sorted({t[1] for t in self.tasks})
        self.gaussians = {s: wl.sets[s].n for s in self.sets_used}
        self.pool = None
        self.procs = 1

    def start_pool(self):
        import multiprocessing as mp
        self.procs = max(1, min(os.cpu_count() or 1, CPU_MAX_PROCS))
        self.pool = mp.get_context("spawn").Pool(self.procs)
        # warm the workers (oracle build/load, page-in of the sets)
        self.pool.map(_oracle_window_task, self.tasks[:self.procs])

    def run(self, n_tasks, offset=0, parallel=True):
        """Runs n_tasks windows; returns (wall seconds, pixels, gaussian-projections)."""
        sel = [self.tasks[(offset + k) % len(self.tasks)] for k in range(n_tasks)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_window_task, sel) if parallel and self.pool else [_oracle_window_task(a) for a in sel]
        wall = time.perf_counter() - t0
        return wall, sum(r[1] for r in res), sum(r[2] for r in res)

    def close(self):
        if self.pool is not None:
            self.pool.terminate()
            self.pool.join()
        import shutil
        shutil.rmtree(self.dir, ignore_errors=True)

    def describe(self, wl):
        return (f"{CPU_WIN}x{CPU_WIN} pixel windows of the views of set(s) {self.sets_used} "
                f"({', '.join(str(self.gaussians[s]) for s in self.sets_used)} Gaussians) of {wl.name}; per window "
                f"the FP64 C oracle projects every Gaussian of the set, bins, composites and differentiates the "
                f"window and runs the projection adjoint of the set")


def cpu_baseline(wl, sampler, budget_s=12.0):
    """The oracle over all host cores (a pool of single-thread processes) and on one core."""
    n1, wall1, px1, g1 = 0, 0.0, 0, 0
    while wall1 < budget_s / 3 and n1 < 8:
        w, p, g = sampler.run(1, n1, parallel=False)
        wall1, px1, g1, n1 = wall1 + w, px1 + p, g1 + g, n1 + 1
    walls, pxs, gs = 0.0, 0, 0
    k = 0
    while walls < budget_s * 2 / 3:
        w, p, g = sampler.run(sampler.procs, k)
        walls, pxs, gs, k = walls + w, pxs + p, gs + g, k + sampler.procs
    return {"value": pxs / walls / 1e6, "unit": UNIT, "cores": sampler.procs, "kind": "oracle",
            "sample": sampler.describe(wl) + f"; {k} windows over {sampler.procs} processes in {walls:.1f} s",
            "gaussians_per_s": gs / walls, "host_cpus": os.cpu_count(),
            "single_thread": {"value": px1 / wall1 / 1e6, "unit": UNIT, "cores": 1, "windows": n1,
                              "seconds": round(wall1, 2), "gaussians_per_s": g1 / wall1}}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle (the only reference implementation: the paper ships
    no code) over the host's cores on windows of the same workload, one pool round a step."""
    if rank != 0:
        return
    wl = build_workload(args.workload, 0)
    sampler = OracleSampler(wl)
    sampler.start_pool()
    try:
        for k in range(args.warmup):
            sampler.run(sampler.procs, k * sampler.procs)
        walls, pxs = [], 0
        for k in range(args.steps):
            w, p, _ = sampler.run(sampler.procs, (args.warmup + k) * sampler.procs)
            walls.append(w)
            pxs += p
    finally:
        sampler.close()
    tot = sum(walls)
    value = pxs / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name,
                                            "sample": f"{sampler.procs} {CPU_WIN}x{CPU_WIN} windows a step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": sampler.procs, "kind": "oracle",
                             "sample": sampler.describe(wl)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- device peaks

def probe_peaks(lobe_abi, torch, reps=3):
    """FP32 FMA (scalar and packed f32x2) and ex2 throughput of this GPU, measured by the
    library's probe kernel with CUDA events: one wave of 256-thread blocks (8 per SM), eight
    independent chains a thread. Returns a dict with the SM count read from the device."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    L = lobe_abi.lib()
    sink = torch.zeros(256, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    blocks = sms * 8
    out = {"sms": sms}
    for kind, name, per_step, iters in ((0, "fp32_fma_scalar_tflops", 2 * 8, 1 << 15),
                                        (1, "fp32_fma_packed_tflops", 4 * 8, 1 << 15),
                                        (2, "mufu_ex2_gops", 8, 1 << 13)):
        best = 0.0
        for _ in range(reps):
            L.lobe_peak_probe(stream.cuda_stream, kind, blocks, iters, sink.data_ptr())
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            L.lobe_peak_probe(stream.cuda_stream, kind, blocks, iters, sink.data_ptr())
            b.record(stream)
            b.synchronize()
            ops = blocks * 256.0 * iters * per_step
            best = max(best, ops / (a.elapsed_time(b) / 1e3))
        out[name] = round(best / (1e12 if "tflops" in name else 1e9), 2)
    out["fp32_tflops"] = max(out["fp32_fma_scalar_tflops"], out["fp32_fma_packed_tflops"])
    out["how"] = (f"lobe_peak_probe: {blocks} blocks x 256 threads x 8 independent chains, best of {reps} "
                  "(CUDA events); FMA = 2 FLOP")
    return out


# --------------------------------------------------------------------------- the step

def make_step(lobe, wl, args, rank, sets=None, tile=None, px=None):
    """A BatchedStep over the whole workload, captured in a CUDA graph, with dL/dC of the
    L1 + 0.2 (1 - SSIM) training loss against a render of a perturbed copy of each set.
    Tile shape and pixels per lane: autotuned on the batch unless given. Returns (step,
    tuning times, sets, number of input Gaussians)."""
    import torch
    from paper_2510_01767_b300.batched import BatchedStep, autotune
    from paper_2510_01767_b300.losses import loss_and_grad
    sets = sets or [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    n_input = sum(s.n for s in sets)
    cams = [c.as_dict() for c in wl.cameras]
    if wl.name.startswith("city"):
        # visibility cropping (Sec. 3.3): once per block, before its fine training, the Gaussians
        # no camera of the block sees are removed; every training step then renders the rest
        batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
        mask = lobe.visibility_crop(lobe.Context(), batch)[0]
        sets = [lobe.GaussianSet(**lobe.crop_compact({k: getattr(sets[0], k) for k in lobe.PARAM_KEYS}, mask))]
    gen = torch.Generator(device="cuda").manual_seed(7 + rank)

    def fill(st):
        st.dL.copy_(torch.randn(st.dL.shape, generator=gen, device="cuda"))

    tuning = None
    if tile is None:
        st, tuning = autotune(sets, cams, wl.items, wl.blocks, reps=3, use_cache=False, dL_init=fill,
                              recompute_T=args.recompute)
    else:
        st = BatchedStep(sets, cams, wl.items, wl.blocks, tile=tile, px=px, recompute_T=args.recompute,
                         persistent=args.persistent, batch=tuple(int(x) for x in args.batch.split(",")))
    # dL/dC of the training loss
    tsets = [lobe.GaussianSet.from_numpy(scenes.perturbed_copy(s, seed=2 + rank)) for s in wl.sets]
    if wl.name.startswith("city"):
        tsets = sets  # the cropped set is the target's layout; perturb it on the device
        tsets = [lobe.GaussianSet(**{k: getattr(s, k).clone() for k in lobe.PARAM_KEYS}) for s in sets]
        tsets[0].means.add_(torch.randn(tsets[0].means.shape, generator=gen, device="cuda") * 0.01)
    tctx = lobe.Context(tile=st.tile)
    tbatch = lobe.Batch(tsets, wl.cameras, wl.items, wl.blocks)
    _, _, timg = lobe.forward(tctx, tbatch, sync=True)
    with torch.cuda.stream(st.stream):
        st.run()
    st.stream.synchronize()
    for v, t, d in zip(st.images(), tbatch.image_views(timg.rgb), st.dL_views()):
        d.copy_(loss_and_grad(v, t)[1])
    del timg, tbatch, tctx, tsets
    if st.graph is None:
        st.capture()
    torch.cuda.synchronize()
    return st, tuning, sets, n_input


def reference_pairs(lobe, torch, st):
    """Sum over pixels of n_contrib (list positions up to each pixel's last contributor) at the
    3DGS tile shape, 16x16, whatever tile the step runs: the compositing work unit of the
    rooflines. A larger tile lists more splats per pixel, so counting the step's own tile
    would credit a larger tile with more work for the same image."""
    if tuple(st.tile) == (16, 16):
        return int(st.image.n_contrib.to(torch.int64).sum().item())
    ctx = lobe.Context(tile=(16, 16))
    _, _, img = lobe.forward(ctx, st.batch, sync=True)
    n = int(img.n_contrib.to(torch.int64).sum().item())
    del img, ctx
    torch.cuda.empty_cache()
    return n


def stage_algorithmic_work(torch, st, nc):
    """Algorithmic bytes / FLOP of one step's stages (the units of the per-stage rooflines);
    nc = the reference pair count (reference_pairs)."""
    b = st.batch
    radius = st.proj.radius
    vis_entry = int((radius > 0).sum().item())
    n_entries = b.n_entries
    seen_any, n_total = 0, 0
    for si, g in enumerate(b.sets):
        seen = torch.zeros(g.n, dtype=torch.bool, device="cuda")
        for i, (s, _, _) in enumerate(b.items):
            if s == si:
                e0 = b.entry_off[i]
                seen |= radius[e0:e0 + g.n] > 0
        seen_any += int(seen.sum().item())
        n_total += g.n
    n_isect = int(st.bins.n_isect.item())
    proj = n_total * PROJ_IN_CULLED + seen_any * (PARAM_BYTES - PROJ_IN_CULLED) + vis_entry * PROJ_OUT_VISIBLE + \
        (n_entries - vis_entry) * PROJ_OUT_CULLED
    proj_bwd = seen_any * (2 * PARAM_BYTES + SD_BYTES) + (n_total - seen_any) * PARAM_BYTES + n_entries * 4 + \
        vis_entry * GRAD2D_BYTES
    return {"project": ("hbm", proj / 1e9, "GB/s"), "bin_sort": ("hbm", n_isect * SORT_BYTES_PAIR / 1e9, "GB/s"),
            "render_fwd": ("alu", nc * FLOP_FWD_PAIR / 1e12, "TFLOP/s"),
            "render_bwd": ("alu", nc * FLOP_BWD_PAIR / 1e12, "TFLOP/s"),
            "project_bwd": ("hbm", proj_bwd / 1e9, "GB/s")}, \
        {"visible_entries": vis_entry, "entries": n_entries, "gaussians_seen": seen_any, "gaussians": n_total,
         "n_contrib_sum_16x16": nc, "intersections": n_isect}


def time_graph(torch, st, K, flush, stream):
    """K graph replays, L2 flushed before each, CUDA events on the step's stream."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            st.graph.replay()
            b.record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in evs])


def time_stages(torch, st, K, flush):
    """K eager steps (the graph's kernels, launched one by one) with an event between stages."""
    import paper_2510_01767_b300 as lobe
    c, b, s = st.ctx, st.batch, st.stream
    fns = [lambda: lobe.project(c, b, st.proj), lambda: lobe.bin_sort(c, b, st.proj, st.bins, sync=False),
           lambda: lobe.render_fwd(c, b, st.proj, st.bins, st.image),
           lambda: lobe.render_bwd(c, b, st.proj, st.bins, st.image, st.dL, st.grad2d),
           lambda: lobe.project_bwd(c, b, st.proj, st.grad2d, st.grads, accumulate=False)]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    with torch.cuda.stream(s):
        for k in range(K):
            flush.zero_()
            evs[k][0].record(s)
            for i, f in enumerate(fns):
                f()
                evs[k][i + 1].record(s)
    torch.cuda.synchronize()
    return np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(5)] for k in range(K)])


def stage_table(stage_ms, work, hbm_peak, fp32_peak):
    names = ["project", "bin_sort", "render_fwd", "render_bwd", "project_bwd"]
    mean_ms = stage_ms.mean(axis=0)
    stages = {}
    for i, n in enumerate(names):
        bound, w, unit = work[n]
        peak = hbm_peak if bound == "hbm" else fp32_peak
        ach = w / (mean_ms[i] / 1e3)
        stages[n] = {"ms": round(float(mean_ms[i]), 4), "bound": bound, "achieved": round(ach, 3), "unit": unit,
                     "peak": round(peak, 2), "frac": round(ach / peak, 4)}
    return stages, names[int(np.argmax(mean_ms))]


_COMMENT = re.compile(r"//[^\n]*|/\*.*?\*/", re.S)


def source_digest(paths):
    """sha1 (16 hex digits) of the code of the given package source files, in order, with
    comments and whitespace removed (an edit of a comment does not change a kernel): the
    traffic files record it for the kernels they were captured from."""
    h = hashlib.sha1()
    for rel in paths:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            code = _COMMENT.sub(" ", f.read())
        h.update("".join(code.split()).encode())
    return h.hexdigest()[:16]


def traffic_of(name, workload):
    """DRAM bytes per launch from profiles/traffic_<stage>_<workload>.json, or None when absent
    or when the kernel sources changed since the capture (the file's source digest)."""
    tf = os.path.join(ROOT, "profiles", f"traffic_{name}_{workload}.json")
    if not os.path.exists(tf):
        return None
    t = json.load(open(tf))
    if "sources" in t and source_digest(t["sources"]) != t.get("source_sha1"):
        return None
    return t


def e2e_pipelined(torch, st, K, params, world):
    """The step through host memory: every step uploads its inputs from pinned host buffers
    and downloads its results, with the copies inside the timed region. Inputs: dL/dC of every
    view (a training loop's per-view input, standing in for the target images); with
    ``params`` also every set's parameters. Results: the rendered images; with ``params`` also
    every parameter gradient. The graph reads and writes fixed device buffers, so each step's
    inputs land in one of two device staging buffers (uploaded on a copy stream while the
    previous step runs) and are copied device-to-device into place at the start of the step;
    results leave the same way. Returns (Mpix/s, h2d bytes, d2h bytes)."""
    import paper_2510_01767_b300 as lobe
    stream = st.stream
    ins = [st.dL]
    outs = [st.image.rgb]
    if params:
        for s in st.batch.sets:
            ins += [getattr(s, k) for k in lobe.PARAM_KEYS]
        for g in st.grads:
            outs += [g[k] for k in lobe.PARAM_KEYS]
    host_in = [t.detach().cpu().pin_memory() for t in ins]
    host_out = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs] for _ in range(2)]
    stage_in = [[torch.empty_like(t) for t in ins] for _ in range(2)]
    stage_out = [[torch.empty_like(t) for t in outs] for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]

    def one(i):
        b = i & 1
        with torch.cuda.stream(up):
            up.wait_event(ev_used[b])  # step i-2 has copied these staging inputs into place
            for h, d in zip(host_in, stage_in[b]):
                d.copy_(h, non_blocking=True)
            ev_in[b].record(up)
        with torch.cuda.stream(stream):
            stream.wait_event(ev_in[b])
            for d, t in zip(stage_in[b], ins):
                t.copy_(d, non_blocking=True)
            ev_used[b].record(stream)
            st.graph.replay()
            stream.wait_event(ev_done[b])  # step i-2's results have left this staging buffer
            for t, d in zip(outs, stage_out[b]):
                d.copy_(t, non_blocking=True)
            ev_out[b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev_out[b])
            for d, h in zip(stage_out[b], host_out[b]):
                h.copy_(d, non_blocking=True)
            ev_done[b].record(down)

    for i in range(2):
        one(i)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(up)  # before the first upload
    for i in range(K):
        one(i)
    for ev in ev_done:
        stream.wait_event(ev)
    e1.record(stream)  # after the last download
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        s = float(t.item())
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    d2h = sum(t.numel() * t.element_size() for t in host_out[0])
    del stage_in, stage_out, host_in, host_out
    return st.batch.n_pixels * K * world / s / 1e6, h2d, d2h


def kernels_per_step(st):
    """Kernels one step launches (counted on an eager run of the captured sequence)."""
    import torch
    from paper_2510_01767_b300 import _abi
    L = _abi.lib()
    n0 = L.lobe_kernel_launches()
    with torch.cuda.stream(st.stream):
        st.run()
    st.stream.synchronize()
    return int(L.lobe_kernel_launches() - n0)


# --------------------------------------------------------------------------- other measurements

def fcs_benchmark(reps=5):
    """Fast camera selection (Sec. 3.2) over a coarse model: a 2M-Gaussian city, 16 KD blocks
    and 64 aerial cameras of 800x600, 16 cameras per batch: project, bin, composite with the
    depth channel, back-project and count per block. Returns a dict for the JSON line."""
    import torch
    import paper_2510_01767_b300 as lobe

    g = scenes.city_layout(11, 2_000_000)
    blocks = [box for _, box in scenes.kd_median_leaves(g.means, 4)]
    rng = np.random.default_rng(12)
    cams = [scenes.aerial_camera((rng.uniform(-200, 200), rng.uniform(-200, 200), 0.0), rng.uniform(120, 180),
                                 rng.uniform(35, 60), rng.uniform(0, 360), 800, 600, 880.0) for _ in range(64)]
    sets = [lobe.GaussianSet.from_numpy(g)]
    per = 16
    batches = [lobe.Batch(sets, cams[i:i + per], [(0, c, -1) for c in range(len(cams[i:i + per]))])
               for i in range(0, len(cams), per)]
    ctx = lobe.Context(tile=(16, 16))
    state = []
    for b in batches:  # bins sized once
        proj, bins, _ = lobe.forward(ctx, b, sync=True)
        ctx.reserve(b.n_entries, int(bins.count * 1.25) + 4096, b.tiles((16, 16))[0])
        bins = lobe.raster.empty_bins(int(bins.count * 1.25) + 4096, b.tiles((16, 16))[0])
        state.append((b, proj, bins, lobe.raster.empty_image(b.n_pixels),
                      torch.empty(b.n_pixels, dtype=torch.float32, device="cuda")))
    stream = torch.cuda.current_stream()

    def run():
        out = []
        for b, proj, bins, img, depth in state:
            lobe.project(ctx, b, proj)
            lobe.bin_sort(ctx, b, proj, bins, sync=False)
            lobe.render_depth(ctx, b, proj, bins, img, depth)
            out.append(lobe.fcs_coverage(ctx, b, img, depth, blocks))
        return out

    for _ in range(2):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        res = run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    counts = torch.cat([c for c, _ in res]).cpu()
    npts = torch.cat([n for _, n in res]).cpu()
    V, assign = lobe.fcs_select(counts, npts, tau=0.1)
    pixels = sum(b.n_pixels for b, *_ in state)
    # the load-balanced KD partition into 16 blocks over the same depth maps (Alg. 1)
    from paper_2510_01767_b300.partition import CameraDepths, kd_partition, workloads
    depths = CameraDepths.from_maps(ctx, cams, torch.cat([d for *_, d in state]),
                                    torch.cat([img.T_final for _, _, _, img, _ in state]))
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    leaves = kd_partition(g.means, root, 16, depths)
    part_ms = (time.perf_counter() - t0) * 1e3
    median = kd_partition(g.means, root, 16, depths, steps=1)  # no refinement: median cuts
    return {"workload": "fcs_city_2M_64cams_800x600_16blocks", "cameras": len(cams), "blocks": len(blocks),
            "ms": round(ms, 3), "cameras_per_s": round(len(cams) / ms * 1e3, 1),
            "mpix_s": round(pixels / ms / 1e3, 1),
            "cameras_per_block": [len(a) for a in assign],
            "kd_partition": {"blocks": 16, "ms": round(part_ms, 1), "workloads": workloads(leaves),
                             "max_workload": max(workloads(leaves)),
                             "max_workload_median_cuts": max(workloads(median))}}


def densify_benchmark(reps=5):
    """Selective densification (Sec. 3.3) of a 2M-Gaussian block with a synthetic SD statistic
    (60% of the Gaussians inside the block): classify, scan, emit. Returns a dict."""
    import torch
    import paper_2510_01767_b300 as lobe

    rng = np.random.default_rng(21)
    n = 2_000_000
    g = scenes.uniform_gaussians(rng, n, 10.0, 5.0, 50.0, logscale_shift=math.log(10.0))
    g.opacity_logits[:] = rng.normal(0.0, 3.0, n).astype(np.float32)
    cnt = np.where(rng.uniform(size=n) < 0.6, rng.integers(1, 8, n), 0).astype(np.int32)
    acc = (rng.exponential(2e-4, n) * np.maximum(cnt, 1)).astype(np.float32)
    gs = lobe.GaussianSet.from_numpy(g)
    acc_t, cnt_t = torch.as_tensor(acc).cuda(), torch.as_tensor(cnt).cuda()
    normals = torch.randn((n, 2, 3), device="cuda")
    ctx = lobe.Context()
    for _ in range(2):
        out, _ = lobe.densify(ctx, gs, acc_t, cnt_t, normals, scene_extent=20.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        out, _ = lobe.densify(ctx, gs, acc_t, cnt_t, normals, scene_extent=20.0)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / reps * 1e3
    # bytes: parameters + statistic read, outputs written (236 B a Gaussian each way)
    gb = (n * (236 + 8) + out.n * 236) / 1e9
    return {"workload": "densify_2M", "gaussians_in": n, "gaussians_out": out.n, "ms": round(ms, 3),
            "gaussians_per_s": round(n / ms * 1e3, 1), "achieved_gbs": round(gb / ms * 1e3, 1),
            "note": "host-timed around the call (it synchronises once to size the output)"}


ADAM_BYTES = 59 * 4 * 7  # per Gaussian: p, g, m, v read, p, m, v written (59 floats each)


def adam_benchmark(ctx, batch, proj, grad2d, hbm_peak, reps=10):
    """Adam (appendix "3DGS Training") on the bench's set: the projection adjoint followed by the
    standalone update, the two fused (standard and sparse Adam), the standalone update alone
    (HBM roofline), torch's fused Adam on the same tensors for context, and the standalone
    update over a 4M-Gaussian set (a whole coarse city model before visibility cropping).
    CUDA events around each variant, L2 flushed before each rep. Returns a dict."""
    import torch
    import paper_2510_01767_b300 as lobe

    sets = [lobe.GaussianSet(**{k: getattr(s, k).clone() for k in lobe.PARAM_KEYS}, crop_mask=s.crop_mask)
            for s in batch.sets]
    cb = lobe.Batch(sets, batch.cameras, batch.items, batch.blocks)
    n = sum(s.n for s in sets)
    opts = [lobe.Adam(s) for s in sets]
    grads = lobe.zero_grads(cb, sd=False)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    def unfused():
        lobe.project_bwd(ctx, cb, proj, grad2d, grads)
        for o, gr in zip(opts, grads):
            o.step(ctx, gr)

    def adam_only():
        for o, gr in zip(opts, grads):
            o.step(ctx, gr)

    t_unfused = timed(unfused)
    t_adj = timed(lambda: lobe.project_bwd(ctx, cb, proj, grad2d, grads))
    t_dense = timed(lambda: lobe.project_bwd_adam(ctx, cb, proj, grad2d, opts, sparse=False))
    t_sparse = timed(lambda: lobe.project_bwd_adam(ctx, cb, proj, grad2d, opts, sparse=True))
    t_adam = timed(adam_only)
    # torch's fused Adam (library kernels) on the same tensors, one group per array
    tparams = [getattr(s, k) for s in sets for k in lobe.PARAM_KEYS]
    for tp, gr in zip(tparams, [g[k] for g in grads for k in lobe.PARAM_KEYS]):
        tp.grad = gr
    topt = torch.optim.Adam([{"params": [tp]} for tp in tparams], lr=1e-3, eps=1e-15, fused=True)
    t_torch = timed(topt.step)
    for tp in tparams:
        tp.grad = None
    del topt
    # the whole coarse model: 4M Gaussians
    big_n = 4_000_000
    big = lobe.GaussianSet(**{k: torch.randn((big_n,) + tuple(getattr(sets[0], k).shape[1:]), device="cuda")
                              for k in lobe.PARAM_KEYS})
    big_g = {k: torch.randn_like(getattr(big, k)) * 1e-3 for k in lobe.PARAM_KEYS}
    big_opt = lobe.Adam(big)
    t_big = timed(lambda: big_opt.step(ctx, big_g))
    del big, big_g, big_opt
    torch.cuda.empty_cache()
    gbs = ADAM_BYTES * n / 1e9 / (t_adam / 1e3)
    gbs_big = ADAM_BYTES * big_n / 1e9 / (t_big / 1e3)
    return {"workload": f"{batch.sets[0].n}-gaussian set of the step", "gaussians": n,
            "adjoint_then_adam_ms": round(t_unfused, 4), "adjoint_ms": round(t_adj, 4),
            "fused_adjoint_adam_ms": round(t_dense, 4), "fused_adjoint_sparse_adam_ms": round(t_sparse, 4),
            "fused_saving": round(1.0 - t_dense / t_unfused, 4),
            "adam_ms": round(t_adam, 4), "torch_fused_adam_ms": round(t_torch, 4),
            "adam_roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": round(hbm_peak, 1), "unit": "GB/s",
                              "frac": round(gbs / hbm_peak, 4), "bytes_per_gaussian": ADAM_BYTES},
            "adam_4M": {"gaussians": big_n, "ms": round(t_big, 4), "achieved_gbs": round(gbs_big, 1),
                        "frac": round(gbs_big / hbm_peak, 4)}}


def training_benchmark(steps=200, warm=20):
    """A training step of the per-block fine training (config-5 style): a 2M-Gaussian city block
    fitted to 16 target views at 1280x720 with L1 + 0.2 (1 - SSIM), one view a step, 3DGS
    learning rates. Two variants, stepped alternately so that both see the same GPU state:
    (a) the autograd.Function with torch's fused Adam, (b) Rasterizer.train_step, whose
    projection adjoint applies the Adam update itself. Each step is bracketed by CUDA events
    on the current stream (a step synchronises once, to size its bins, so the events also
    see the host's part). Reports medians over `steps` steps of each after `warm`."""
    import torch
    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300.losses import l1_ssim_loss

    gt, init, cams, block = scenes.training_scene(n=2_000_000, n_views=16)
    keys = lobe.PARAM_KEYS
    with torch.no_grad():
        r = lobe.Rasterizer(gt.n)
        gtp = [torch.as_tensor(gt.arrays()[k]).cuda().contiguous() for k in keys]
        targets = [lobe.rasterize(*gtp, c.as_dict(), r).clone() for c in cams]
        del gtp, r
    extent = float(np.linalg.norm(gt.means.max(0) - gt.means.min(0)))
    lrs = [1.6e-4 * extent, 5e-3, 1e-3, 5e-2, 2.5e-3]
    order = np.random.default_rng(0).permutation(np.arange(steps + warm) % len(cams))
    variants = {}
    for name in ("torch_adam", "fused_adam"):
        raster = lobe.Rasterizer(init.n, tile=(16, 16), block=block)
        ps = [torch.as_tensor(init.arrays()[k]).cuda().contiguous() for k in keys]
        if name == "torch_adam":
            ps = [p.requires_grad_(True) for p in ps]
            opt = torch.optim.Adam([{"params": [p], "lr": lr} for p, lr in zip(ps, lrs)], eps=1e-15, fused=True)
        else:
            opt = lobe.Adam(lobe.GaussianSet(*ps), lr=dict(zip(("means", "log_scales", "quats", "opacity_logits",
                                                                 "sh_dc"), lrs), sh_rest=lrs[4]), eps=1e-15)
        variants[name] = (raster, ps, opt, [], [])
    stream = torch.cuda.current_stream()
    for it in range(steps + warm):
        k = int(order[it])
        for name, (raster, ps, opt, times, losses) in variants.items():
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if name == "torch_adam":
                loss = l1_ssim_loss(lobe.rasterize(*ps, cams[k].as_dict(), raster), targets[k])
                opt.zero_grad(set_to_none=True)
                loss.backward()
                opt.step()
            else:
                loss = raster.train_step(opt, cams[k].as_dict(), lambda v: l1_ssim_loss(v[0], targets[k]))
            b.record(stream)
            if it >= warm:
                times.append((a, b))
            if it in (0, steps + warm - 1):
                losses.append(round(float(loss.detach()), 5))
    torch.cuda.synchronize()
    out = {"workload": "city_block_2M_16views_1280x720", "gaussians": init.n, "steps": steps,
           "timing": "CUDA events around each step, the two variants alternating; medians"}
    for name, (_, _, _, times, losses) in variants.items():
        ms = [a.elapsed_time(b) for a, b in times]
        out[name + "_ms_per_step"] = round(float(np.median(ms)), 3)
        out[name + "_ms_p10_p90"] = [round(float(np.percentile(ms, 10)), 3), round(float(np.percentile(ms, 90)), 3)]
        out[name + "_loss_first_last"] = losses
    del variants
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------------------- batched vs plain

def plain_stage_ms(torch, plain, reps):
    """Where the plain path's time goes: each stage run for every view in turn (every view's
    buffers are its own, so the stages can be grouped), CUDA events between the groups; mean
    ms a step per stage, summed over the views."""
    import paper_2510_01767_b300 as lobe
    stream = torch.cuda.current_stream()
    names = ["project", "bin_sort", "render_fwd", "render_bwd", "project_bwd"]

    def stage(i, p):
        c, b = p.ctx, p.batch
        return [lambda: lobe.project(c, b, p.proj), lambda: lobe.bin_sort(c, b, p.proj, p.bins, sync=False),
                lambda: lobe.render_fwd(c, b, p.proj, p.bins, p.image),
                lambda: lobe.render_bwd(c, b, p.proj, p.bins, p.image, p.dL, p.grad2d),
                lambda: lobe.project_bwd(c, b, p.proj, p.grad2d, p.grads, accumulate=False)][i]()

    tot = np.zeros(5)
    for r in range(reps + 1):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        evs[0].record(stream)
        for i in range(5):
            for p in plain.steps:
                stage(i, p)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        if r > 0:  # the first round warms up
            tot += [evs[i].elapsed_time(evs[i + 1]) for i in range(5)]
    return {n: round(float(t / reps), 4) for n, t in zip(names, tot)}


def batched_vs_plain(lobe, torch, wl, sets, st, batched_ms, reps=5, batched_stages=None):
    """The batched graph step (already timed) against the plain path on the same batch: one
    view per call sequence, eager, same tile shape, pixels per lane, persistent choice and
    staging batch; and against the
    autograd.Function called view by view (host-timed: each forward synchronises once to size
    its bins)."""
    from paper_2510_01767_b300.batched import PlainSteps, _time
    cams = [c.as_dict() for c in wl.cameras]
    gen = torch.Generator(device="cuda").manual_seed(7)
    plain = PlainSteps(sets, cams, wl.items, wl.blocks, tile=st.tile, px=st.px, persistent=st.persistent,
                       batch=st.batch_size)
    for p in plain.steps:
        p.dL.copy_(torch.randn(p.dL.shape, generator=gen, device="cuda"))
    plain_ms = _time(plain.run, reps, torch.cuda.current_stream())
    plain_stages = plain_stage_ms(torch, plain, reps)
    del plain
    torch.cuda.empty_cache()
    params = [[getattr(s, k).clone().requires_grad_(True) for k in lobe.PARAM_KEYS] for s in sets]
    rasters = {(si, b): lobe.Rasterizer(sets[si].n, tile=st.tile, block=wl.blocks[b] if b >= 0 else None)
               for si, _, b in wl.items}
    dls = [torch.randn((3, cams[c]["height"], cams[c]["width"]), generator=gen, device="cuda") for _, c, _ in wl.items]

    def per_view():
        for (si, c, b), dl in zip(wl.items, dls):
            lobe.rasterize(*params[si], cams[c], rasters[(si, b)]).backward(dl)

    per_view()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        per_view()
    torch.cuda.synchronize()
    autograd_ms = (time.perf_counter() - t0) / reps * 1e3
    del params, rasters, dls
    torch.cuda.empty_cache()
    pixels = st.batch.n_pixels
    return {"workload": wl.name, "tile": list(st.tile), "px_per_lane": list(st.px), "persistent": st.persistent,
            "staging_batch": list(st.batch_size), "batched_ms": round(batched_ms, 3), "plain_ms": round(plain_ms, 3),
            "batched_mpix_s": round(pixels / batched_ms / 1e3, 1), "plain_mpix_s": round(pixels / plain_ms / 1e3, 1),
            "ratio": round(plain_ms / batched_ms, 3),
            "plain_stages_ms": plain_stages,
            "batched_stages_ms": {k: v["ms"] for k, v in (batched_stages or {}).items()},
            "autograd_per_view_ms": round(autograd_ms, 3), "ratio_vs_autograd_per_view": round(autograd_ms / batched_ms, 3),
            "note": "ratio: against the eager one-view-per-call library path (no host synchronisation); "
                    "ratio_vs_autograd_per_view: against the autograd.Function called view by view (host-timed)"}


def single_view_extra(lobe, torch, args, rank, flush, hbm_peak, fp32_peak, K=10):
    """The single-view medium workload (200k Gaussians, 1600x1066) through the same graph
    step: a context figure next to the headline batch. Returns (dict, step) -- the step is
    reused by the Adam measurement."""
    wl = build_workload("medium", rank)
    st, tuning, sets, n_input = make_step(lobe, wl, args, rank)
    for _ in range(3):
        st.replay()
    torch.cuda.synchronize()
    ms = time_graph(torch, st, K, flush, st.stream)
    stage_ms = time_stages(torch, st, K, flush)
    work, counts = stage_algorithmic_work(torch, st, reference_pairs(lobe, torch, st))
    stages, dom = stage_table(stage_ms, work, hbm_peak, fp32_peak)
    return {"workload": wl.name, "value": round(st.batch.n_pixels / float(ms.mean()) / 1e3, 3), "unit": UNIT,
            "ms_per_step": round(float(ms.mean()), 4), "tile": list(st.tile), "px_per_lane": list(st.px),
            "persistent": st.persistent, "staging_batch": list(st.batch_size), "staging_batch_ms": st.batch_times,
            "tuning_ms": {k: round(v, 4) for k, v in (tuning or {}).items()}, "stages": stages, **counts}, st


# --------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    wl = build_workload(args.workload, seed=rank)
    sampler = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sampler = OracleSampler(wl)  # the oracle's process pool starts before any CUDA call
        sampler.start_pool()

    import torch
    import torch.distributed as dist
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300 import _abi

    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    hbm_source = "measured hbm_gbs (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks else "fallback 6400 GB/s"
    dev = probe_peaks(_abi, torch)
    fp32_peak = dev["fp32_tflops"]

    tile = px = None
    if args.tile != "auto":
        tile, px = tuple(int(x) for x in args.tile.split("x")), tuple(int(x) for x in args.px.split(","))
    st, tuning, sets, n_input = make_step(lobe, wl, args, rank, tile=tile, px=px)
    K = args.steps
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    per_step_kernels = kernels_per_step(st)
    for _ in range(max(3, args.warmup)):
        st.replay()
    torch.cuda.synchronize()
    st.ctx.status()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    clk.wait_first_sample()
    step_ms = time_graph(torch, st, K, flush, st.stream)
    total_s = float(step_ms.sum()) / 1e3
    if world > 1:
        dist.barrier()
        t = torch.tensor([total_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    pixels = st.batch.n_pixels * K * world
    value = pixels / total_s / 1e6
    gaussians_per_s = n_input * K * world / total_s
    stage_ms = time_stages(torch, st, min(K, 10), flush)
    e2e_value, h2d, d2h = e2e_pipelined(torch, st, K, False, world)
    e2e_hp_value, h2d_hp, d2h_hp = e2e_pipelined(torch, st, max(4, K // 4), True, world)
    clk.__exit__(None, None, None)  # sampled over the timed regions
    st.ctx.status()

    work, counts = stage_algorithmic_work(torch, st, reference_pairs(lobe, torch, st))
    stages, dom = stage_table(stage_ms, work, hbm_peak, fp32_peak)
    st_tile, st_px, st_persistent = st.tile, st.px, st.persistent
    tb = traffic_of("bin_sort", wl.name)
    if tb:
        stages["bin_sort"]["dram_bytes_per_call"] = tb["bytes_per_launch"]
        stages["bin_sort"]["dram_achieved_gbs"] = round(tb["bytes_per_launch"] / 1e9 / (stages["bin_sort"]["ms"] / 1e3), 1)
        stages["bin_sort"]["dram_frac"] = round(stages["bin_sort"]["dram_achieved_gbs"] / hbm_peak, 4)
        stages["bin_sort"]["dram_note"] = "DRAM bytes of one call's kernels from one ncu capture (profiles/)"
    stages["bin_sort"]["work_note"] = ("achieved/frac count 44 B per intersection: the duplication + pair sort + "
                                       "ranges of the 3DGS design, a work-equivalent this binning does not run")
    tr = traffic_of(dom, wl.name)
    if tr and "tile" in tr and (list(tr["tile"]) != list(st_tile) or list(tr["px"]) != list(st_px) or
                                bool(tr["persistent"]) != bool(st_persistent)):
        tr = None  # captured with another kernel configuration than the one timed
    roof = {"stage": dom, "bound": stages[dom]["bound"], "achieved": stages[dom]["achieved"],
            "peak": stages[dom]["peak"], "unit": stages[dom]["unit"], "frac": stages[dom]["frac"],
            "traffic": tr.get("bytes_per_launch") if tr else None,
            "peak_source": (hbm_source if stages[dom]["bound"] == "hbm" else
                            "measured FP32 FMA rate of this GPU (lobe_peak_probe, packed f32x2), FMA = 2 FLOP")}
    csum = clk.summary()

    cpu = None
    extras = {}
    if sampler is not None:
        cpu = cpu_baseline(wl, sampler)
        sampler.close()
    if world == 1 and not args.no_extras:
        extras["batched_vs_plain"] = batched_vs_plain(lobe, torch, wl, sets, st, float(np.median(step_ms)),
                                                      batched_stages=stages)
    graph_tile, graph_px, graph_persistent, graph_batch = st.tile, st.px, st.persistent, st.batch_size
    graph_batch_times = st.batch_times
    del st
    torch.cuda.empty_cache()
    if world == 1 and not args.no_extras and args.workload != "medium":
        extras["medium_view"], mst = single_view_extra(lobe, torch, args, rank, flush, hbm_peak, fp32_peak)
        with torch.cuda.stream(mst.stream):  # the step's context launches on its own stream
            extras["adam"] = adam_benchmark(mst.ctx, mst.batch, mst.proj, mst.grad2d, hbm_peak)
        del mst
        torch.cuda.empty_cache()
        extras["fast_camera_selection"] = fcs_benchmark()
        torch.cuda.empty_cache()
        extras["selective_densification"] = densify_benchmark()
        torch.cuda.empty_cache()
        extras["training_step"] = training_benchmark()

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(float(step_ms.mean()), 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "gaussians": sum(s.n for s in sets), "gaussians_input": n_input,
                       "views": len(wl.items), "pixels": st_pixels(wl),
                       "tile": list(graph_tile), "px_per_lane": {"fwd": graph_px[0] or "default",
                                                                  "bwd": graph_px[1] or "default"},
                       "persistent_compositing": graph_persistent,
                       "staging_batch": {"fwd": graph_batch[0] or 32, "bwd": graph_batch[1] or 32,
                                         "tuning_ms": graph_batch_times},
                       "tuning_ms": ({k: round(v, 4) for k, v in tuning.items()} if tuning else None),
                       "sh_degree": 3, **counts,
                       "step": "one CUDA graph replay: projection (each set once for all its views), binning of "
                               "all views' tiles, composite, adjoint, projection adjoint summed per set",
                       "bwd_mode": "recompute" if args.recompute else "store",
                       "l2": "flushed between timed steps (2x126 MB write); the step's inputs also exceed L2",
                       "dL_dC": "L1+0.2(1-SSIM) vs a render of a perturbed copy, computed once before timing",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "gaussians_per_s": round(gaussians_per_s, 1),
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "reading": "training loop: parameters and their gradients stay resident (the optimizer "
                               "consumes the gradients on the device); per step every view's dL/dC up and every "
                               "rendered image down"},
            "e2e_host_params": {"value": round(e2e_hp_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d_hp),
                                "d2h_bytes_per_step": int(d2h_hp),
                                "reading": "caller-owned parameters: per step also every parameter up and every "
                                           "parameter gradient down"},
            "gpu_launches": int(per_step_kernels * K),
            "gpu_launches_note": f"{per_step_kernels} kernels a step (counted on one eager run of the captured "
                                 f"sequence) x {K} graph replays",
            "clocks": {k: csum[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "device_peaks": dev,
            "roofline": roof,
            "stages": stages,
            "cpu_baseline": cpu,
            **extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def st_pixels(wl):
    return int(sum(wl.cameras[c].as_dict()["width"] * wl.cameras[c].as_dict()["height"] for _, c, _ in wl.items))


if __name__ == "__main__":
    main()
