#!/usr/bin/env python3
"""Throughput of the differentiable tile rasterizer: one step = project -> bin/sort ->
render fwd -> render bwd -> project bwd over one synthetic view (the per-block training
step's rasterizer pass; the loss gradient dL/dC is computed once before timing).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lobe|reference] [--workload NAME]

Default workload: 200k Gaussians in a 20 m box, one 1600x1066 pinhole view (fx=fy=1200),
16x16 tiles, SH degree 3, dL/dC of L1 + 0.2 (1 - SSIM) against a render of a perturbed copy.
Prints ONE JSON line (rank 0). Under torchrun every rank renders its own independent
replica (a different seeded block): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
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
PROJ_BYTES_VISIBLE = 236 + 56   # params in, splat record + radius + tile count out
PROJ_BYTES_CULLED = 44 + 8      # mean/scale/quat/logit in, radius + count out
PROJ_BWD_BYTES = 236 + 48 + 236 + 8  # params + 2D grads in, param grads + radius/opacity out
SORT_BYTES_PAIR = 12 + 12 + 12 + 8  # per intersection for duplication + pair sort + ranges (key/value written,
#                                     read, sorted and written, range read); this binning moves fewer (see traffic)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lobe", choices=["lobe", "reference"])
    ap.add_argument("--workload", default="medium", choices=["medium", "small", "city", "multi"])
    ap.add_argument("--tile", default="auto", help="WxH, or auto: tile shape and pixels per lane by the autotuner")
    ap.add_argument("--px", default="0,0", help="with --tile WxH: pixels per lane of the composite and its adjoint")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain multi-block measurement")
    ap.add_argument("--no-fcs", action="store_true", help="skip the fast-camera-selection, densification, Adam and training-step measurements")
    ap.add_argument("--recompute", action="store_true")
    return ap.parse_args()


def build_workload(name, seed):
    if name == "small":
        return scenes.small_scene(seed=seed)
    if name == "medium":
        return scenes.medium_scene(seed=seed)
    if name == "city":
        return scenes.city_block_scene(seed=seed)
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

def oracle_sample(wl, win=128, seed=0):
    """Runs the FP64 oracle's fwd+bwd on a win x win pixel window of the workload's first item
    (every Gaussian projected, only the window's tiles binned and rendered). Returns
    (seconds, pixels, gaussians)."""
    import oracle
    s, c, b = wl.items[0]
    g = oracle.set_dict(wl.sets[s])
    cam = wl.cameras[c].as_dict()
    W, H = cam["width"], cam["height"]
    w = min(win, W, H)
    x0, y0 = (W - w) // 2, (H - w) // 2
    dL = np.zeros((3, H, W))
    dL[:, y0:y0 + w, x0:x0 + w] = np.random.default_rng(seed).standard_normal((3, w, w))
    t0 = time.perf_counter()
    with oracle.window(x0, y0, x0 + w, y0 + w):
        f = oracle.forward(g, cam, wl.tile)
        oracle.backward(g, cam, f, dL, wl.tile, aabb=wl.blocks[b] if b >= 0 and wl.blocks else None)
    return time.perf_counter() - t0, w * w, g["means"].shape[0]


def cpu_baseline(wl, budget_s=15.0):
    done, t, px, gs = 0, 0.0, 0, 0
    while t < budget_s and done < 50:
        dt, p, n = oracle_sample(wl, seed=done)
        t += dt
        px += p
        gs += n
        done += 1
    return {"value": px / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} steps of the FP64 C oracle (single thread) on a 128x128 pixel window of the "
                      f"workload's view: all {gs // done} Gaussians projected, the window's tiles binned, "
                      f"composited and differentiated; {t:.1f} s total",
            "gaussians_per_s": gs / t}


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = build_workload(args.workload, 0)
    for _ in range(args.warmup):
        oracle_sample(wl)
    times, px = [], 0
    for k in range(args.steps):
        dt, p, _ = oracle_sample(wl, seed=k)
        times.append(dt)
        px = p
    tot = sum(times)
    value = px * args.steps / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "sample": "128x128 pixel window per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "128x128 pixel window of the workload's view per step, FP64 C oracle, "
                                       "single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- batched vs plain

def batched_vs_plain(reps=5):
    """Multi-block workload (4 KD blocks of 0.5/1/2/3 M Gaussians, 16 views of uneven
    resolution, 4 per block): one autotuned CUDA-graph step over all views vs the plain path
    (one view per call sequence, eager, same tile shape). Returns a dict for the JSON line."""
    import torch
    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300.batched import PlainSteps, _time, autotune

    wl = scenes.multi_block_scene(seed=0)
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    cams = [c.as_dict() for c in wl.cameras]
    gen = torch.Generator(device="cuda").manual_seed(7)

    def fill(st):
        st.dL.copy_(torch.randn(st.dL.shape, generator=gen, device="cuda"))

    best, times = autotune(sets, cams, wl.items, wl.blocks, reps=reps, use_cache=False, dL_init=fill)
    batched_ms = _time(best.replay, reps, best.stream)
    pixels = best.batch.n_pixels
    tile, best_px = best.tile, best.px
    n_isect = best.n_isect
    del best
    torch.cuda.empty_cache()
    plain = PlainSteps(sets, cams, wl.items, wl.blocks, tile=tile, px=best_px)
    for st in plain.steps:
        fill(st)
    plain_ms = _time(plain.run, reps, torch.cuda.current_stream())
    del plain
    torch.cuda.empty_cache()
    # the per-view path of a training loop: the autograd.Function view by view (each forward
    # synchronises once to size its bins), parameters as leaf tensors; host-timed, since the
    # device idles during the synchronisations
    params = [[getattr(s, k).clone().requires_grad_(True) for k in lobe.PARAM_KEYS] for s in sets]
    rasters = {(si, b): lobe.Rasterizer(sets[si].n, tile=tile, block=wl.blocks[b] if b >= 0 else None)
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
    return {"workload": wl.name, "gaussians": sum(s.n for s in sets), "views": len(cams), "pixels": pixels,
            "intersections": n_isect, "tile": list(tile), "px_per_lane": list(best_px), "autotune_ms": {k: round(v, 3) for k, v in times.items()},
            "batched_ms": round(batched_ms, 3), "plain_ms": round(plain_ms, 3),
            "batched_mpix_s": round(pixels / batched_ms / 1e3, 1), "plain_mpix_s": round(pixels / plain_ms / 1e3, 1),
            "ratio": round(plain_ms / batched_ms, 3),
            "autograd_per_view_ms": round(autograd_ms, 3), "ratio_vs_autograd_per_view": round(autograd_ms / batched_ms, 3),
            "note": "ratio: against the eager one-view-per-call library path (no host synchronisation); "
                    "ratio_vs_autograd_per_view: against the autograd.Function called view by view (host-timed)"}


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


def training_benchmark(steps=60, warm=20):
    """A training step of the per-block fine training (config-5 style): a 2M-Gaussian city block
    fitted to 16 target views at 1280x720 with L1 + 0.2 (1 - SSIM), one view a step, 3DGS
    learning rates. Per-step time (a) through the autograd.Function with torch's fused Adam and
    (b) through Rasterizer.train_step, whose projection adjoint applies the Adam update itself.
    Host-timed over `steps` steps after `warm` (each step synchronises once to size its bins).
    Returns a dict."""
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
    out = {"workload": "city_block_2M_16views_1280x720", "gaussians": init.n, "steps": steps}
    for variant in ("torch_adam", "fused_adam"):
        raster = lobe.Rasterizer(init.n, tile=(16, 16), block=block)
        ps = [torch.as_tensor(init.arrays()[k]).cuda().contiguous() for k in keys]
        if variant == "torch_adam":
            ps = [p.requires_grad_(True) for p in ps]
            opt = torch.optim.Adam([{"params": [p], "lr": lr} for p, lr in zip(ps, lrs)], eps=1e-15, fused=True)
        else:
            gs = lobe.GaussianSet(*ps)
            opt = lobe.Adam(gs, lr=dict(zip(("means", "log_scales", "quats", "opacity_logits", "sh_dc"), lrs),
                                        sh_rest=lrs[4]), eps=1e-15)
        losses = []
        for it in range(steps + warm):
            if it == warm:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            k = int(order[it])
            if variant == "torch_adam":
                loss = l1_ssim_loss(lobe.rasterize(*ps, cams[k].as_dict(), raster), targets[k])
                opt.zero_grad(set_to_none=True)
                loss.backward()
                opt.step()
            else:
                loss = raster.train_step(opt, cams[k].as_dict(), lambda v: l1_ssim_loss(v[0], targets[k]))
            if it in (0, steps + warm - 1):
                losses.append(round(float(loss), 5))
        torch.cuda.synchronize()
        out[variant + "_ms_per_step"] = round((time.perf_counter() - t0) / steps * 1e3, 3)
        out[variant + "_loss_first_last"] = losses
        del raster, ps, opt
        torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2510_01767_b300 as lobe
    from paper_2510_01767_b300 import _abi
    from paper_2510_01767_b300.losses import loss_and_grad

    from paper_2510_01767_b300.batched import autotune, config_name

    wl = build_workload(args.workload, seed=rank)
    sets = [lobe.GaussianSet.from_numpy(s) for s in wl.sets]
    batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    n_input = sum(s.n for s in sets)
    if args.workload == "city":
        # visibility cropping (Sec. 3.3): once per block, before its fine training, the Gaussians
        # no camera of the block sees are removed; every training step then renders the rest
        mask = lobe.visibility_crop(lobe.Context(), batch)[0]
        kept = lobe.crop_compact({k: getattr(sets[0], k) for k in lobe.PARAM_KEYS}, mask)
        sets = [lobe.GaussianSet(**kept)]
        batch = lobe.Batch(sets, wl.cameras, wl.items, wl.blocks)
    tuning = None
    if args.tile == "auto":
        best, tuning = autotune(sets, [c.as_dict() for c in wl.cameras], wl.items, wl.blocks, reps=3, use_cache=False,
                                recompute_T=args.recompute)
        tile, px = best.tile, best.px
        del best
        torch.cuda.empty_cache()
    else:
        tile, px = tuple(int(x) for x in args.tile.split("x")), tuple(int(x) for x in args.px.split(","))
    wl.tile = tile
    ctx = lobe.Context(tile=tile, recompute_T=args.recompute, px_fwd=px[0], px_bwd=px[1])

    # one-time: bins sized from a first pass, dL/dC of the training loss against a target
    proj, bins, img = lobe.forward(ctx, batch, sync=True)
    n_isect = bins.count
    n_tiles, _ = batch.tiles(tile)
    ctx.reserve(batch.n_entries, int(n_isect * 1.25) + 4096, batch.tiles(tile)[0])
    bins = lobe.raster.empty_bins(int(n_isect * 1.25) + 4096, n_tiles)
    tgt_sets = [lobe.GaussianSet.from_numpy(scenes.perturbed_copy(s, seed=2 + rank)) for s in wl.sets]
    tbatch = lobe.Batch(tgt_sets, wl.cameras, wl.items, wl.blocks)
    _, _, timg = lobe.forward(ctx, tbatch, sync=True)
    dL = torch.empty_like(img.rgb)
    for v, t, d in zip(batch.image_views(img.rgb), tbatch.image_views(timg.rgb), batch.image_views(dL)):
        d.copy_(loss_and_grad(v, t)[1])
    grad2d = torch.empty((batch.n_entries, 12), dtype=torch.float32, device="cuda")
    grads = lobe.zero_grads(batch, sd=True)
    image = lobe.raster.empty_image(batch.n_pixels)
    stream = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        lobe.project(ctx, batch, proj)
        if ev:
            ev[1].record(stream)
        lobe.bin_sort(ctx, batch, proj, bins, sync=False)
        if ev:
            ev[2].record(stream)
        lobe.render_fwd(ctx, batch, proj, bins, image)
        if ev:
            ev[3].record(stream)
        lobe.render_bwd(ctx, batch, proj, bins, image, dL, grad2d)
        if ev:
            ev[4].record(stream)
        lobe.project_bwd(ctx, batch, proj, grad2d, grads, accumulate=False)  # fresh gradients, as autograd returns
        if ev:
            ev[5].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ctx.status()

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(K)]
    launches0 = _abi.lib().lobe_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    clk.wait_first_sample()
    for k in range(K):
        flush.zero_()  # inputs of the next step start cold in L2
        step(evs[k])
    torch.cuda.synchronize()
    launches = _abi.lib().lobe_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    ctx.status()
    stage_ms = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(5)] for k in range(K)])
    step_ms = stage_ms.sum(axis=1)
    total_s = float(step_ms.sum()) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    pixels = batch.n_pixels * K * world
    gaussians = sum(s.n for s in sets) * K * world
    value = pixels / total_s / 1e6

    # ---- end to end through host buffers (pinned), copies inside the timed region. Two readings:
    # (1) `e2e`, a training loop's: the parameters (and their gradients, which the optimizer
    # consumes on the device) stay resident; every step uploads its per-view input (dL/dC,
    # standing in for the view's target image: 3 floats a pixel) and downloads its rendered
    # image; (2) `e2e_host_params`, the rasterizer as a service whose caller owns the
    # parameters: every step also uploads all parameters and downloads all gradients. Device
    # buffers are doubled so that step i+1's uploads and step i-1's downloads run on their own
    # streams (copy engines) while step i's kernels run.
    host_params = [{k: getattr(s, k).detach().cpu().pin_memory() for k in lobe.PARAM_KEYS} for s in sets]
    host_crop = [s.crop_mask.cpu().pin_memory() if s.crop_mask is not None else None for s in sets]
    host_dL = dL.cpu().pin_memory()
    host_rgb = [torch.empty_like(image.rgb, device="cpu").pin_memory() for _ in range(2)]
    host_grads = [[{k: torch.empty_like(g[k], device="cpu").pin_memory() for k in lobe.PARAM_KEYS} for g in grads]
                  for _ in range(2)]
    bsets = [[lobe.GaussianSet(**{k: torch.empty_like(getattr(s, k)) for k in lobe.PARAM_KEYS},
                               crop_mask=torch.empty_like(s.crop_mask) if s.crop_mask is not None else None)
              for s in sets] for _ in range(2)]
    bbatch = [lobe.Batch(bs, wl.cameras, wl.items, wl.blocks) for bs in bsets]
    bdL = [torch.empty_like(dL) for _ in range(2)]
    bimage = [lobe.raster.empty_image(batch.n_pixels) for _ in range(2)]
    bgrads = [lobe.zero_grads(batch, sd=False) for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]    # inputs of buffer b uploaded
    ev_used = [torch.cuda.Event() for _ in range(2)]  # kernels done with buffer b
    ev_out = [torch.cuda.Event() for _ in range(2)]   # results of buffer b downloaded

    def e2e_step(i, params):
        b = i & 1
        with torch.cuda.stream(up):
            up.wait_event(ev_used[b])  # step i-2 finished reading these inputs
            if params:
                for s, hp, hc in zip(bsets[b], host_params, host_crop):
                    for k in lobe.PARAM_KEYS:
                        getattr(s, k).copy_(hp[k], non_blocking=True)
                    if hc is not None:
                        s.crop_mask.copy_(hc, non_blocking=True)
            bdL[b].copy_(host_dL, non_blocking=True)
            ev_in[b].record(up)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])  # step i-2's results have left these buffers
        bt, gr = (bbatch[b], bgrads[b]) if params else (batch, grads)
        lobe.project(ctx, bt, proj)
        lobe.bin_sort(ctx, bt, proj, bins, sync=False)
        lobe.render_fwd(ctx, bt, proj, bins, bimage[b])
        lobe.render_bwd(ctx, bt, proj, bins, bimage[b], bdL[b], grad2d)
        lobe.project_bwd(ctx, bt, proj, grad2d, gr, accumulate=False)
        ev_used[b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev_used[b])
            host_rgb[b].copy_(bimage[b].rgb, non_blocking=True)
            if params:
                for g, hg in zip(bgrads[b], host_grads[b]):
                    for k in lobe.PARAM_KEYS:
                        hg[k].copy_(g[k], non_blocking=True)
            ev_out[b].record(down)

    def run_e2e(params):
        for i in range(2):
            e2e_step(i, params)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(up)  # before the first upload
        for i in range(K):
            e2e_step(i, params)
        for ev in ev_out:
            stream.wait_event(ev)
        e1.record(stream)  # after the last download
        torch.cuda.synchronize()
        e2e_s = e0.elapsed_time(e1) / 1e3
        if world > 1:
            t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = host_dL.numel() * 4
        d2h = host_rgb[0].numel() * 4
        if params:
            h2d += sum(t.numel() * t.element_size() for d in host_params for t in d.values())
            h2d += sum(c.numel() for c in host_crop if c is not None)
            d2h += sum(t.numel() * t.element_size() for d in host_grads[0] for t in d.values())
        return pixels / e2e_s / 1e6, h2d, d2h

    e2e_value, h2d, d2h = run_e2e(False)
    e2e_hp_value, h2d_hp, d2h_hp = run_e2e(True)
    clk.__exit__(None, None, None)  # sampled over both timed regions

    # ---- roofline of the dominant stage
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    csum = clk.summary()
    sm_mhz = csum["sm_mhz"] or peaks.get("sm_max_mhz", 2032.0)
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    alu_peak_tflops = 2 * 128 * 148 * sm_mhz * 1e6 / 1e12  # FP32 FMA lanes x SMs x clock, FMA = 2 FLOP
    torch.cuda.synchronize()
    nc = int(image.n_contrib.to(torch.int64).sum().item())
    vis = int((proj.tiles > 0).sum().item())
    n_entries = batch.n_entries
    n_isect = int(bins.n_isect.item())
    mean_ms = stage_ms.mean(axis=0)
    names = ["project", "bin_sort", "render_fwd", "render_bwd", "project_bwd"]
    units = {
        "project": ("hbm", (vis * PROJ_BYTES_VISIBLE + (n_entries - vis) * PROJ_BYTES_CULLED) / 1e9, "GB/s", hbm_peak),
        "bin_sort": ("hbm", n_isect * SORT_BYTES_PAIR / 1e9, "GB/s", hbm_peak),
        "render_fwd": ("alu", nc * FLOP_FWD_PAIR / 1e12, "TFLOP/s", alu_peak_tflops),
        "render_bwd": ("alu", nc * FLOP_BWD_PAIR / 1e12, "TFLOP/s", alu_peak_tflops),
        "project_bwd": ("hbm", vis * PROJ_BWD_BYTES / 1e9, "GB/s", hbm_peak),
    }
    stages = {}
    for i, n in enumerate(names):
        bound, work, unit, peak = units[n]
        ach = work / (mean_ms[i] / 1e3)
        stages[n] = {"ms": round(float(mean_ms[i]), 4), "bound": bound, "achieved": round(ach, 3), "unit": unit,
                     "peak": round(peak, 2), "frac": round(ach / peak, 4)}
    dom = names[int(np.argmax(mean_ms))]
    traffic = None
    tf = os.path.join(ROOT, "profiles", f"traffic_{dom}_{wl.name}.json")
    if os.path.exists(tf):
        traffic = json.load(open(tf)).get("bytes_per_launch")
    roof = {"stage": dom, "bound": stages[dom]["bound"], "achieved": stages[dom]["achieved"],
            "peak": stages[dom]["peak"], "unit": stages[dom]["unit"], "frac": stages[dom]["frac"],
            "traffic": traffic,
            "peak_source": ("measured hbm_gbs (MEASURED_PEAKS.json)" if stages[dom]["bound"] == "hbm" else
                            "derived: 2 x 128 FP32 lanes x 148 SMs x median SM clock sampled in the timed region")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)
    adam = None
    if world == 1 and not args.no_fcs:
        adam = adam_benchmark(ctx, batch, proj, grad2d, hbm_peak)
    bvp = None
    if world == 1 and not args.no_batched:
        del proj, bins, image, grad2d, grads, flush
        torch.cuda.empty_cache()
        bvp = batched_vs_plain()
    fcs = dens = train = None
    if world == 1 and not args.no_fcs:
        torch.cuda.empty_cache()
        fcs = fcs_benchmark()
        torch.cuda.empty_cache()
        dens = densify_benchmark()
        torch.cuda.empty_cache()
        train = training_benchmark()

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(float(step_ms.mean()), 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "gaussians": sum(s.n for s in sets), "gaussians_input": n_input,
                       "pixels": batch.n_pixels,
                       "tile": list(tile), "px_per_lane": {"fwd": px[0] or "default", "bwd": px[1] or "default"},
                       "tuning_ms": ({k: round(v, 4) for k, v in tuning.items()} if tuning else None),
                       "sh_degree": 3, "intersections": n_isect, "visible": vis,
                       "visibility_crop": ("applied once before the timed steps (Gaussians no view of the block "
                                           "sees removed)") if args.workload == "city" else None,
                       "bwd_mode": "recompute" if args.recompute else "store",
                       "l2": "flushed between timed steps (2x126 MB write)",
                       "dL_dC": "L1+0.2(1-SSIM) vs perturbed-copy render, computed once before timing",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "gaussians_per_s": round(gaussians / total_s, 1),
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "reading": "training loop: parameters resident; per step dL/dC up, the image down"},
            "e2e_host_params": {"value": round(e2e_hp_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d_hp),
                                "d2h_bytes_per_step": int(d2h_hp),
                                "reading": "caller-owned parameters: per step also all parameters up, all gradients down"},
            "gpu_launches": int(launches),
            "clocks": {k: csum[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "roofline": roof,
            "stages": stages,
            "cpu_baseline": cpu,
            "batched_vs_plain": bvp,
            "fast_camera_selection": fcs,
            "selective_densification": dens,
            "adam": adam,
            "training_step": train,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
