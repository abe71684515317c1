"""Benchmark of the active-set OIT splat renderer (forward + backward) on GB300.

Workload (one step = one training iteration of the active-set loop: forward
of the active set over its view's frozen sums with the fused L1 loss, and the
backward to compact active gradients): 1,000,000 splats of the unbounded
synthetic scene (70 % in a radius-2 ball, 30 % log-uniform out to radius 50),
one 1297 x 840 view, 5 % active set chosen by the seeded gradient-magnitude
proxy, FP32.  The same library's full-set path (100 % active) and the 1 / 20 %
fractions are timed in the same run, as are the active-set update (mask
compaction) and the delayed frozen-sum update.

value = splat-pixel evaluations per second = E / step time, E = number of
(active splat, pixel) pairs with alpha >= 1/255 in the view (counted by the
forward raster in an untimed pass).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms per fwd+bwd iteration & splat-pixel evals/s at 1M splats, active vs full set"
UNIT = "splat-pixel evals/s"
FRACTIONS = (0.01, 0.05, 0.20, 1.0)
HEADLINE_FRACTION = 0.05
WORKLOAD = "unbounded scene, 1M splats, one 1297x840 view, 5% active (gradient proxy), fused L1, fwd+bwd"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 flops (an FMA counts 2, exp2 / reciprocal / min 1 each) of one
# contributing (splat, pixel) pair in the algorithm the kernels run: forward
# 22 = offsets 2, u 2, e1 1, e2 1, s 3, log2 alpha 1, exp2 1, clamp 1,
# P 6, Q 2, T 2; backward 38 = the same 12 up to the clamp,
# D = (B g).c - B g.F 6, 1 - a 1, reciprocal 1, dL/da = A/(1 - a) + w D 3,
# dL/dw += a D 2, dL/dc += a (B g) 6, da 1, chain sums 6.
FLOPS_FWD_PER_EVAL = 22
FLOPS_BWD_PER_EVAL = 38


# Source files of each kernel: the DRAM traffic recorded in profiles/dram_traffic.txt is reported
# only while the digest of these files still matches the one recorded with it.
KERNEL_SOURCES = {
    "raster_bwd": ("raster_bwd.cu", "pair_eval.cuh", "common.cuh"),
    "raster_fwd": ("raster_fwd.cu", "pair_eval.cuh", "common.cuh"),
    "project": ("project.cu", "common.cuh"),
    "scatter": ("project.cu", "common.cuh"),
}


def _code_only(src: str) -> str:
    """C/CUDA source without comments and blank lines (a comment edit changes no counter)."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def kernel_digest(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2605_13855_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from profiles/dram_traffic.txt (lines: kernel bytes digest workload),
    or None when absent or recorded for other sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if kernel not in KERNEL_SOURCES or not os.path.exists(path):
        return None
    digest = kernel_digest(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel and parts[2] == digest:
            return float(parts[1])
    return None


def algorithmic_bytes(n_active: int, pairs: int, pixels: int, tiles: int) -> dict:
    """Unique HBM bytes each kernel of one step must move (FP32 parameters: 75 floats = 300 B per
    splat; screen record 48 B + extent 16 B; 4 B per (splat, tile) pair id; per pixel 20 B of frozen
    sums, 12 B target, 12 B image, 20 B of pixel state; 40 B of screen-space gradients per splat)."""
    na, m, p = n_active, pairs, pixels
    return {
        "project": na * (4 + 300 + 64) + 4 * tiles,
        "scan_tiles": 8 * tiles,
        "scatter": na * (4 + 64) + 4 * m + 4 * tiles,
        "raster_fwd": 4 * m + 48 * na + p * (20 + 12 + 12 + 20),
        "raster_bwd": 4 * m + 48 * na + p * 20 + 40 * na,
        "project_bwd": na * (4 + 300 + 40 + 300),
    }


def hbm_report(per_kernel: dict, n_active: int, pairs: int, pixels: int, tiles: int, ms_step: float,
               peaks: dict, peak_kind: str) -> dict:
    peak = float(peaks.get("hbm_gbs", 6800.0))
    ab = algorithmic_bytes(n_active, pairs, pixels, tiles)
    out = {"peak_gbs": peak, "peak_source": f"hbm_gbs ({peak_kind})", "per_kernel": {}}
    for k, b in ab.items():
        if k in per_kernel and per_kernel[k]["avg_ms"] > 0:
            gbs = b / (per_kernel[k]["avg_ms"] * 1e-3) / 1e9
            out["per_kernel"][k] = {"bytes": int(b), "gbs": gbs, "frac": gbs / peak}
    tot = sum(ab.values())
    out["step_bytes"] = int(tot)
    out["step_gbs"] = tot / (ms_step * 1e-3) / 1e9
    out["step_frac"] = out["step_gbs"] / peak
    out["floor_ms"] = tot / (peak * 1e9) * 1e3
    return out


def fp32_peak_tflops(sm_mhz: float, n_sms: int = 152) -> float:
    # SMs x 128 FP32 lanes x 2 flops (FMA) x clock
    return n_sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def device_sms(torch, dev) -> int:
    """Streaming multiprocessors of the device (152 on a GB300)."""
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def _clock_dir() -> str:
    """Where the nvidia-smi samples of the timed region are written (SPARSEOIT_CLOCKS_DIR, else the
    system temporary directory)."""
    import tempfile
    return os.environ.get("SPARSEOIT_CLOCKS_DIR") or tempfile.gettempdir()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [line.split(",") for line in open(self.path).read().strip().splitlines() if line.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if len(r) >= 9]
        mx = [float(r[2]) for r in rows if len(r) >= 9]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_camera_seeds(rank: int, base_seed: int):
    """Weak scaling over views: rank k renders its own view of the same scene
    (camera seed base + 3 + 17 k, target seed base + 1 + 17 k)."""
    return base_seed + 3 + 17 * rank, base_seed + 1 + 17 * rank


def reduce_over_ranks(ms: float, evals: float, device="cpu"):
    """Whole-job figures over the ranks: the max step time and the summed evals."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(e)
    return float(t.item()), float(e.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _centred_window(cam, area_px):
    W, H = cam["width"], cam["height"]
    a = max(16 * 16, min(area_px, W * H))
    w = int(min(W, max(16, round((a * W / H) ** 0.5))))
    h = int(min(H, max(16, round(a / w))))
    x0, y0 = (W - w) // 2, (H - h) // 2
    return (x0, y0, x0 + w, y0 + h)


def _oracle_step(scene, cam, target, mask, frozen, win):
    """One fwd+bwd of the active set over the frozen sums, restricted to win, by the FP64 oracle."""
    import oracle
    r = oracle.render(scene, cam, subset=mask, frozen_sums=frozen, window=win)
    diff = r["image"] - target.astype(np.float64)
    g = np.zeros_like(diff)
    x0, y0, x1, y1 = win
    HW = cam["width"] * cam["height"]
    g[y0:y1, x0:x1] = np.sign(diff[y0:y1, x0:x1]) / (3 * HW)
    oracle.backward(scene, cam, r["sums"], g, active=mask, window=win)
    return r["pairs"]


def _calibrated_window(scene, cam, target, mask, seconds):
    """Centred window whose oracle fwd+bwd takes about `seconds` (from a 64x64 probe)."""
    import oracle
    area = 64 * 64
    win = _centred_window(cam, area)
    for _ in range(4):  # the per-call overhead makes one probe underestimate: refine
        frozen, _, _ = oracle.render_sums(scene, cam, subset=~mask, window=win)
        t = time.perf_counter()
        _oracle_step(scene, cam, target, mask, frozen, win)
        dt = time.perf_counter() - t
        if dt >= 0.5 * seconds or (win[2] - win[0]) * (win[3] - win[1]) >= cam["width"] * cam["height"]:
            break
        area = int(area * min(64.0, max(1.5, seconds / max(dt, 1e-3))))
        win = _centred_window(cam, area)
    return win


def _oracle_timing(scene, cam, target, mask, win, steps, warmup):
    import oracle
    frozen, _, _ = oracle.render_sums(scene, cam, subset=~mask, window=win)
    times, evals = [], 0
    for k in range(warmup + steps):
        t = time.perf_counter()
        evals = _oracle_step(scene, cam, target, mask, frozen, win)
        if k >= warmup:
            times.append(time.perf_counter() - t)
    return float(np.mean(times)), evals


def _sample_text(win, evals, dt, reps):
    return (f"fwd+bwd of the 5% active set (all 1M splats given, complement as precomputed sums) on a centred "
            f"{win[2]-win[0]}x{win[3]-win[1]} px window of the 1297x840 view (E={evals} pairs), FP64, "
            f"{reps} timed rep(s) of {dt:.2f} s")


def run_reference(args):
    """The FP64 oracle timed on the host cores on a bounded sample of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2605_13855_gb300 import scenes
    scene, cam, target = scenes.unbounded_workload()
    mask = scenes.unbounded_active_mask(scene, HEADLINE_FRACTION).astype(bool)
    per_step = min(8.0, 150.0 / max(1, args.steps + args.warmup))
    win = _calibrated_window(scene, cam, target, mask, per_step)
    mean, evals = _oracle_timing(scene, cam, target, mask, win, args.steps, args.warmup)
    value = evals / mean
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (FP64 oracle on a window sample)",
                       "active_fraction": HEADLINE_FRACTION, "window": list(win)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": _sample_text(win, evals, mean, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(scene, cam, target, mask, budget_s=15.0):
    """The oracle as it stands, timed on the host cores: fwd+bwd on a window sized to ~budget_s
    (repeated when even the whole view takes less)."""
    import oracle
    win = _calibrated_window(scene, cam, target, mask, budget_s)
    dt, evals = _oracle_timing(scene, cam, target, mask, win, 1, 0)
    reps = 1
    if dt < 0.5 * budget_s:
        reps = int(min(20, max(1, budget_s // max(dt, 1e-3))))
        dt, evals = _oracle_timing(scene, cam, target, mask, win, reps, 0)
    return {"value": evals / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": _sample_text(win, evals, dt, reps)}


def _graph_time(torch, stream, flush, fn, steps, warmup):
    """Capture fn() once as a CUDA graph; mean CUDA-event time of `steps` replays (L2 flushed between)."""
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        g.replay()
        stream.synchronize()
        times = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            stream.synchronize()
            times.append(a.elapsed_time(b))
    del g
    return float(np.mean(times))


def _grad_out(torch, rows, dev):
    out = {k: torch.zeros((rows,) + s, dtype=torch.float32, device=dev) for k, s in
           (("means", (3,)), ("quats", (4,)), ("log_scales", (3,)), ("opacity_logits", ()),
            ("sh_color", (16, 3)), ("sh_weight", (16,)))}
    out["sigma"] = torch.zeros(1, dtype=torch.float32, device=dev)
    return out


def measure_single_view(torch, dev, scene, cam, target, masks, steps, warmup, stream, flush):
    """fwd (fused L1) + bwd of one view for each active mask of `masks` (label -> uint8 numpy
    mask), the complement's sums committed first; CUDA-graph replay, L2 flushed between steps.
    Returns label -> {ms, evals, pairs, n_active, value, commit_recompute_ms}."""
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams
    n = int(scene["means"].shape[0])
    W, H = cam["width"], cam["height"]
    sp = SplatParams.from_numpy(scene, device=dev)
    tg = torch.as_tensor(target, device=dev)
    img = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    res = {}
    with torch.cuda.stream(stream):
        r = Renderer(n, [(W, H)], max_pairs=1 << 27)
        for label, m in masks.items():
            r.set_active(torch.as_tensor(m, device=dev), stream=stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            b.record(stream)
            out = _grad_out(torch, r.n_active, dev)

            def step():
                r.forward(sp, [cam], [0], targets=[tg], stream=stream, images=[img], loss=loss)
                r.backward(sp, stream=stream, out=out)

            r.set_counting(True)
            step()
            r.status(stream)
            r.set_counting(False)
            M, E = r.last_counts(stream)
            ms = _graph_time(torch, stream, flush, step, steps, warmup)
            r.status(stream)
            res[label] = {"ms": ms, "evals": int(E), "pairs": int(M), "n_active": int(r.n_active),
                          "value": E / (ms * 1e-3), "commit_recompute_ms": a.elapsed_time(b)}
        r.close()
    return res


def measure_tiny(args, torch, dev, stream, flush):
    """Tiny workload: 4,096 splats uniform in [-1, 1]^3, one 128x128 view, every splat active, L1
    against the render of a second seeded splat set (rendered by the library)."""
    from paper_2605_13855_gb300 import scenes
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams
    scene, tscene, cam = scenes.tiny_workload()
    n, W, H = scenes.TINY["n"], cam["width"], cam["height"]
    with torch.cuda.stream(stream):
        rt = Renderer(n, [(W, H)])
        rt.set_active(torch.ones(n, dtype=torch.uint8, device=dev), stream=stream)
        rt.commit_frozen(SplatParams.from_numpy(tscene, device=dev), cam, 0, mode="recompute", stream=stream)
        imgs, _ = rt.forward(SplatParams.from_numpy(tscene, device=dev), [cam], [0], stream=stream)
        target = imgs[0].cpu().numpy()
        rt.close()
    res = measure_single_view(torch, dev, scene, cam, target, {"all_active": np.ones(n, np.uint8)}, args.steps,
                              args.warmup, stream, flush)["all_active"]
    return {"workload": "tiny: 4,096 splats uniform in [-1,1]^3, one 128x128 view, all active, fused L1 against "
                        "the render of a second seeded splat set", **res}


def measure_clustered(args, torch, dev, stream, flush):
    """Clustered workload: 200k splats in 32 anisotropic blobs, one 800x800 view, a seeded random 10 %
    active set over the complement's committed sums, against the same library's full set."""
    from paper_2605_13855_gb300 import scenes
    scene, mask, cam, target = scenes.clustered_workload()
    n = scenes.CLUSTERED["n"]
    res = measure_single_view(torch, dev, scene, cam, target, {"active_10pct": mask, "full_set": np.ones(n, np.uint8)},
                              args.steps, args.warmup, stream, flush)
    return {"workload": "clustered: 200k splats in 32 anisotropic normal blobs, one 800x800 view, seeded random "
                        "10% active over the complement's sums, fused L1", "active_10pct": res["active_10pct"],
            "full_set": res["full_set"], "speedup_active_vs_full": res["full_set"]["ms"] / res["active_10pct"]["ms"]}


def run_small(args, which):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if which == "tiny":
        r = measure_tiny(args, torch, dev, stream, flush)
        ms, value = r["ms"], r["value"]
    else:
        r = measure_clustered(args, torch, dev, stream, flush)
        ms, value = r["active_10pct"]["ms"], r["active_10pct"]["value"]
    line = {"metric": f"ms per fwd+bwd iteration & splat-pixel evals/s, {which} workload", "value": value,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"], "l2": "flushed between timed steps (256 MiB write)"},
            "result": r}
    print(json.dumps(line), flush=True)


def run_batched(args):
    print(json.dumps(measure_batched(args)), flush=True)


def measure_batched(args):
    """3M splats, 16 views of four sizes in one call (CUDA-graph replay), 5 % active:
    autotuned forward strip vs one pixel per thread vs 16 separate calls."""
    import torch
    import __graft_entry__
    from paper_2605_13855_gb300 import scenes
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    c = scenes.BATCHED
    n = c["n"]
    scene = scenes.unbounded_scene(n, c["seed"])
    cams = scenes.batched_cameras()
    sizes = [(cm["width"], cm["height"]) for cm in cams]
    views = list(range(len(cams)))
    mask = torch.as_tensor(scenes.proxy_active_mask(scene["means"], c["active"], c["seed"] + 2), device=dev)
    sp = SplatParams.from_numpy(scene, device=dev)
    targets = [torch.as_tensor(scenes.uniform_target(c["seed"] + 1 + 17 * k, W, H), device=dev)
               for k, (W, H) in enumerate(sizes)]
    imgs = [torch.empty((H, W, 3), dtype=torch.float32, device=dev) for (W, H) in sizes]
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    with torch.cuda.stream(stream):
        rA = Renderer(n, sizes, max_pairs=1 << 27)
        rA.set_active(mask, stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for v, cm in enumerate(cams):
            rA.commit_frozen(sp, cm, v, mode="recompute", stream=stream)
        b.record(stream)
        stream.synchronize()
        res["commit_recompute_16_views_ms"] = a.elapsed_time(b)
        out = _grad_out(torch, rA.n_active, dev)
        rA.set_counting(True)
        rA.forward(sp, cams, views, targets=targets, stream=stream, images=imgs, loss=loss)
        rA.status(stream)
        rA.set_counting(False)
        M, E = rA.last_counts(stream)
        tune = rA.autotune(sp, cams, views, targets=targets, stream=stream)

        def batched_step(r=rA):
            r.forward(sp, cams, views, targets=targets, stream=stream, images=imgs, loss=loss)
            r.backward(sp, stream=stream, out=out)

        res["autotuned_ms"] = _graph_time(torch, stream, flush, batched_step, args.steps, args.warmup)
        rA.set_profiling(True)
        rA.get_profile()
        for _ in range(args.steps):
            flush.zero_()
            batched_step()
        stream.synchronize()
        res["per_kernel_ms"] = {k: v[1] / max(1, v[0]) for k, v in rA.get_profile().items()}
        rA.set_profiling(False)

        def separate_step():
            for k in views:
                rA.forward(sp, [cams[k]], [k], targets=[targets[k]], stream=stream, images=[imgs[k]], loss=loss)
                rA.backward(sp, stream=stream, out=out, accumulate=k > 0)

        res["separate_calls_ms"] = _graph_time(torch, stream, flush, separate_step, args.steps, args.warmup)
        rA.status(stream)
        rA.close()
        rB = Renderer(n, sizes, max_pairs=1 << 27, fwd_pixels_per_thread=1)
        rB.set_active(mask, stream=stream)
        for v, cm in enumerate(cams):
            rB.commit_frozen(sp, cm, v, mode="recompute", stream=stream)
        res["fixed_1px_ms"] = _graph_time(torch, stream, flush, lambda: batched_step(rB), args.steps, args.warmup)
        rB.status(stream)
        rB.close()
        # persistent rasters (blocks that take the 16 views' tiles from one queue), autotuned strip
        rC = Renderer(n, sizes, max_pairs=1 << 27, fwd_pixels_per_thread=tune["fwd_pixels_per_thread"],
                      raster_persistent=1)
        rC.set_active(mask, stream=stream)
        for v, cm in enumerate(cams):
            rC.commit_frozen(sp, cm, v, mode="recompute", stream=stream)
        res["persistent_ms"] = _graph_time(torch, stream, flush, lambda: batched_step(rC), args.steps, args.warmup)
        rC.status(stream)
        rC.close()
    ms = res["autotuned_ms"]
    line = {"metric": "ms per fwd+bwd iteration & splat-pixel evals/s, 3M splats, 16 views of uneven size, 5% active",
            "value": E / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched: 3M splats (unbounded scene), 16 views (4 x 640x480, 800x800, 1297x840, "
                                   "1600x1064), 5% active, fused L1, one call + CUDA graph",
                       "evals_per_step": E, "pairs_per_step": M, "n_active": int(mask.sum().item())},
            "variants_ms": {"autotuned_one_call": ms, "fixed_1px_per_thread_one_call": res["fixed_1px_ms"],
                            "persistent_rasters_one_call": res["persistent_ms"],
                            "16_separate_calls": res["separate_calls_ms"]},
            "autotune": tune, "commit_recompute_16_views_ms": res["commit_recompute_16_views_ms"],
            "per_kernel_ms": res["per_kernel_ms"]}
    return line


def run_active_update(args):
    print(json.dumps(measure_active_update(args)), flush=True)


def measure_active_update(args):
    """The periodic active-set update of Alg. 1 (sparseoit_update_active_set): 1M splats (unbounded
    scene), 60 training views of 1297x840, 30 picked by farthest point sampling, full-set fwd+bwd
    with the fused L1 loss on each, gradients summed, Eq. 8 against per-group thresholds."""
    import torch
    import __graft_entry__
    from paper_2605_13855_gb300 import scenes
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams, activeness
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    c = scenes.ACTIVE_UPDATE
    n, W, H, V, S = c["n"], c["width"], c["height"], c["views"], c["n_sub"]
    scene = scenes.unbounded_scene(n, c["seed"])
    cams = scenes.training_cameras(V, c["camera_seed"], W, H)
    rng = np.random.default_rng(c["camera_seed"] + 1)
    sp = SplatParams.from_numpy(scene, device=dev)
    targets = [torch.as_tensor(scenes.uniform_target(c["camera_seed"] + 100 + k, W, H), device=dev) for k in range(V)]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        r = Renderer(n, [(W, H)] * V, max_pairs=1 << 26)
        r.set_active(torch.ones(n, dtype=torch.uint8, device=dev), stream=stream)
        # thresholds: the 99th percentile of each group's nonzero norms after one update pass
        inf = [float("inf")] * 6
        _, _, scratch = r.update_active_set(sp, cams, targets, inf, S, int(rng.integers(V)), stream=stream)
        _, norms = activeness(scratch, inf, stream=stream, with_norms=True)
        nz = norms[norms.max(dim=1).values > 0]
        eps = [float(torch.quantile(nz[:, k], 0.99).item()) for k in range(6)]
        mask = torch.empty(n, dtype=torch.uint8, device=dev)
        for _ in range(args.warmup):
            r.update_active_set(sp, cams, targets, eps, S, int(rng.integers(V)), stream=stream, scratch=scratch,
                                mask=mask)
        stream.synchronize()
        # the delayed frozen-sum updates of a stage: every view committed under the current set, then
        # one more update, then every view brought up to date incrementally (against a recompute)
        for v in range(V):
            r.commit_frozen(sp, cams[v], v, mode="recompute", stream=stream)
        r.update_active_set(sp, cams, targets, eps, S, int(rng.integers(V)), stream=stream, scratch=scratch,
                            mask=mask)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for v in range(V):
            r.commit_frozen(sp, cams[v], v, mode="incremental", stream=stream)
        b.record(stream)
        stream.synchronize()
        commit_inc_ms = a.elapsed_time(b)
        r.set_active(mask, stream=stream)  # the same set again: every view stale, recompute timed
        a.record(stream)
        for v in range(V):
            r.commit_frozen(sp, cams[v], v, mode="recompute", stream=stream)
        b.record(stream)
        stream.synchronize()
        commit_rec_ms = a.elapsed_time(b)
        times, fracs = [], []
        with ClockSampler(os.path.join(_clock_dir(), "clocks_active_update.csv")) as clk:
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                first = int(rng.integers(V))
                a.record(stream)
                r.update_active_set(sp, cams, targets, eps, S, first, stream=stream, scratch=scratch, mask=mask)
                b.record(stream)
                stream.synchronize()
                times.append(a.elapsed_time(b))
                fracs.append(r.n_active / n)
        clocks = clk.summary()
        r.close()
    ms = float(np.mean(times))
    line = {"metric": "ms per periodic active-set update (30 of 60 views, full-set fwd+bwd, Eq. 8), 1M splats",
            "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "active-set update: unbounded scene, 1M splats, 60 views 1297x840, 30 picked by "
                                   "farthest point sampling, fused L1, thresholds = 99th percentile of each group's "
                                   "nonzero norms", "l2": "inputs (60 x 13 MB targets, 300 MB gradients) exceed L2"},
            "ms_per_subsampled_view": ms / S, "active_fraction_after": float(np.mean(fracs)), "eps": eps,
            "amortised_ms_per_iteration_at_interval_500": ms / 500.0,
            "commit_all_views_after_update_ms": {"incremental": commit_inc_ms, "recompute": commit_rec_ms},
            "stage_overhead_ms_per_iteration_at_interval_500": (ms + commit_inc_ms) / 500.0, "clocks": clocks}
    return line


def run_bwd_ablation(args):
    """Backward ablation (the paper's Tab. 2 analogue) on the headline workload: the step and the
    backward raster with per-splat lanes (this library's design), per-pixel threads with warp-reduced
    atomics, and per-pixel threads with one set of atomics per contributing pair (the 3DGS scheme)."""
    import torch
    import __graft_entry__
    from paper_2605_13855_gb300 import scenes
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    c = scenes.UNBOUNDED
    scene, cam, target_np = scenes.unbounded_workload()
    n, W, H = c["n"], c["width"], c["height"]
    sp = SplatParams.from_numpy(scene, device=dev)
    target = torch.as_tensor(target_np, device=dev)
    img = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for frac in (0.05, 1.0):
        mask = torch.as_tensor(scenes.unbounded_active_mask(scene, frac), device=dev)
        for mode, name in ((1, "per_splat"), (2, "per_pixel_warp_reduced"), (3, "per_pixel_atomics")):
            with torch.cuda.stream(stream):
                r = Renderer(n, [(W, H)], max_pairs=1 << 26, bwd_parallel=mode)
                r.set_active(mask, stream=stream)
                r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
                out = _grad_out(torch, r.n_active, dev)

                def step(r=r, out=out):
                    r.forward(sp, [cam], [0], targets=[target], stream=stream, images=[img], loss=loss)
                    r.backward(sp, stream=stream, out=out)

                ms = _graph_time(torch, stream, flush, step, args.steps, args.warmup)
                r.set_profiling(True)
                r.get_profile()
                for _ in range(args.steps):
                    flush.zero_()
                    step()
                stream.synchronize()
                prof = r.get_profile()
                r.set_profiling(False)
                r.status(stream)
                r.close()
            bw = prof.get("raster_bwd", (1, 0.0))
            res[f"{frac}"] = res.get(f"{frac}", {})
            res[f"{frac}"][name] = {"step_ms": ms, "raster_bwd_ms": bw[1] / max(1, bw[0])}
    head = res["0.05"]
    line = {"metric": "backward ablation: ms per fwd+bwd step and backward-raster ms, 1M splats, 1297x840",
            "value": head["per_pixel_atomics"]["step_ms"] / head["per_splat"]["step_ms"],
            "unit": "step speedup of per-splat over per-pixel atomics (5% active)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["per_splat"]["step_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fractions": [0.05, 1.0]}, "modes": res}
    print(json.dumps(line), flush=True)


def _err_stats(gpu, ref):
    d = np.abs(gpu - ref)
    return {"max_rel": float(d.max() / max(np.abs(ref).max(), 1e-30)),
            "mean_rel": float(d.mean() / max(np.abs(ref).mean(), 1e-30))}


def run_precision(args):
    print(json.dumps(measure_precision(args)), flush=True)


def measure_precision(args, oracle_views=None):
    """3M splats, 8 views 1297x840, 5 % active: BF16-stored SH vs FP32, time and error against
    the FP64 oracle on the centred 256x256 crop of every view (dL/dC zero outside it), or of the
    first `oracle_views` views (the gradient compared is then that of those views' loss alone)."""
    import torch
    import __graft_entry__
    import oracle
    from paper_2605_13855_gb300 import scenes
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    c = scenes.PRECISION
    n = c["n"]
    scene = scenes.unbounded_scene(n, c["seed"])
    cams = scenes.precision_cameras()
    W, H = c["width"], c["height"]
    views = list(range(len(cams)))
    mask_np = scenes.proxy_active_mask(scene["means"], c["active"], c["seed"] + 2)
    mask = torch.as_tensor(mask_np, device=dev)
    x0, y0, x1, y1 = c["crop"]
    rng = np.random.default_rng(c["seed"] + 9)
    gs = []
    for _ in views:
        g = np.zeros((H, W, 3))
        g[y0:y1, x0:x1] = rng.normal(size=(y1 - y0, x1 - x0, 3))
        gs.append(g)
    n_ref = len(views) if oracle_views is None else max(1, min(len(views), int(oracle_views)))
    for v in range(n_ref, len(views)):
        gs[v][:] = 0.0  # the compared gradient is that of the first n_ref views' loss
    gts = [torch.as_tensor(g, dtype=torch.float32, device=dev) for g in gs]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    imgs = [torch.empty((H, W, 3), dtype=torch.float32, device=dev) for _ in views]
    results = {}
    sc16 = dict(scene)
    for k in ("sh_color", "sh_weight"):
        sc16[k] = torch.as_tensor(scene[k]).to(torch.bfloat16).float().numpy()
    act = mask_np.astype(bool)
    rows = np.where(act)[0]
    for label, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
        sp = SplatParams.from_numpy(scene, device=dev, sh_dtype=dt)
        with torch.cuda.stream(stream):
            r = Renderer(n, [(W, H)] * len(views), max_pairs=1 << 27)
            r.set_active(mask, stream=stream)
            for v, cm in enumerate(cams):
                r.commit_frozen(sp, cm, v, mode="recompute", stream=stream)
            out = _grad_out(torch, r.n_active, dev)

            def step():
                r.forward(sp, cams, views, stream=stream, images=imgs)
                r.backward(sp, gts, stream=stream, out=out)

            ms = _graph_time(torch, stream, flush, step, args.steps, args.warmup)
            step()
            stream.synchronize()
            r.status(stream)
        img_np = [im.cpu().numpy().astype(np.float64) for im in imgs]
        grads = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
        r.close()
        del sp
        results[label] = {"ms": ms, "img": img_np, "grads": grads}
    # FP64 oracle on the crops, with FP32 and with BF16-rounded coefficients
    # Pairs within a relative 3e-4 of the 1/255 cut (or of the 0.99 clamp) may be decided
    # differently in FP32 and FP64: each pixel / gradient element is allowed the oracle's bound
    # on what those pairs can change ("flip"); the raw maximum is reported beside.  Splats at a
    # max(0, .) kink or the near plane are excluded and counted.
    errs = {}
    for ref_label, ref_scene in (("oracle_fp32_inputs", scene), ("oracle_bf16_inputs", sc16)):
        ref_imgs, flips, tot = [], [], None
        for v, cm in enumerate(cams[:n_ref]):
            rr_ = oracle.render(ref_scene, cm, window=c["crop"], amb_band=3e-4)
            ref_imgs.append(rr_["image"][y0:y1, x0:x1])
            flips.append(rr_["flip"][y0:y1, x0:x1])
            rg = oracle.backward_full(ref_scene, cm, rr_["sums"], gs[v], active=act, window=c["crop"],
                                      amb_band=3e-4, want_flip=True)
            if tot is None:
                tot = {"grads": rg["grads"][rows], "flip": rg["flip"][rows], "amb": rg["amb"][rows]}
            else:
                tot["grads"] += rg["grads"][rows]
                tot["flip"] += rg["flip"][rows]
                tot["amb"] |= rg["amb"][rows]
        groups = dict(means=(0, 3), quats=(3, 7), log_scales=(7, 10), opacity_logits=(10, 11),
                      sh_color=(11, 59), sh_weight=(59, 75))
        keep = (tot["amb"] & 2) == 0
        ri, fl = np.stack(ref_imgs), np.stack(flips)
        for label in ("fp32", "bf16"):
            gi = np.stack([im[y0:y1, x0:x1] for im in results[label]["img"][:n_ref]])
            d = np.abs(gi - ri).max(axis=3)
            dm = np.maximum(d - fl, 0.0)
            e = {"image": {"max_rel": float(dm.max() / np.abs(ri).max()),
                           "mean_rel": float(d.mean() / np.abs(ri).mean()),
                           "raw_max_rel": float(d.max() / np.abs(ri).max()),
                           "pixels_with_allowance": float((fl > 0).mean())}}
            for name, (lo, hi) in groups.items():
                gg = results[label]["grads"][name].reshape(len(rows), -1)[keep]
                rr = tot["grads"][keep, lo:hi]
                dd = np.abs(gg - rr)
                fl_g = tot["flip"][keep, lo:hi]
                sc_g = max(np.abs(rr).max(), 1e-30)
                over = dd > 1e-4 * sc_g
                e[name] = {"max_rel": float(np.maximum(dd - fl_g, 0.0).max() / sc_g),
                           "mean_rel": float(dd.mean() / max(np.abs(rr).mean(), 1e-30)),
                           "raw_max_rel": float(dd.max() / sc_g),
                           "raw_max_rel_no_allowance_elems": float(dd[fl_g == 0].max(initial=0.0) / sc_g),
                           "elems_over_1e-4_raw": float(over.mean()),
                           "splats_over_1e-4_raw": float(over.any(axis=1).mean())}
            e["kink_excluded_splats"] = float(1.0 - keep.mean())
            errs[f"{label}_vs_{ref_label}"] = e
    line = {"metric": "ms per fwd+bwd iteration, 3M splats, 8 views 1297x840, 5% active: BF16 vs FP32 SH storage",
            "value": results["fp32"]["ms"] / results["bf16"]["ms"], "unit": "speedup of BF16 SH over FP32 SH",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": results["bf16"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 SH, f32 math",
            "data": "synthetic",
            "config": {"workload": "precision: 3M splats (unbounded scene), 8 views 1297x840, 5% active, linear "
                                   "loss on the 256x256 crop [520,776)x[292,548) of each view",
                       "oracle_views": n_ref,
                       "ms_fp32_sh": results["fp32"]["ms"], "ms_bf16_sh": results["bf16"]["ms"]},
            "errors": errs}
    return line


def config_summaries(args, torch, dev):
    """Compact results of the other four workloads (tiny, clustered, batched, precision) and of the
    periodic active-set update, for the default line; each timed like its own --workload run with
    fewer steps, the precision errors against the oracle on two of the eight views."""
    import copy
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    a = copy.copy(args)
    a.steps, a.warmup = min(args.steps, 10), 3
    out, t0 = {}, time.perf_counter()
    out["tiny"] = measure_tiny(a, torch, dev, stream, flush)
    out["clustered"] = measure_clustered(a, torch, dev, stream, flush)
    del flush
    torch.cuda.empty_cache()
    b = measure_batched(a)
    out["batched"] = {"workload": b["config"]["workload"], "value": b["value"], "unit": b["unit"],
                      "ms": b["ms_per_step"], "variants_ms": b["variants_ms"], "autotune": b["autotune"],
                      "evals_per_step": b["config"]["evals_per_step"]}
    torch.cuda.empty_cache()
    pr = measure_precision(a, oracle_views=2)
    out["precision"] = {"workload": pr["config"]["workload"], "ms_fp32_sh": pr["config"]["ms_fp32_sh"],
                        "ms_bf16_sh": pr["config"]["ms_bf16_sh"], "bf16_speedup": pr["value"],
                        "oracle_views": pr["config"]["oracle_views"], "errors": pr["errors"]}
    torch.cuda.empty_cache()
    u = copy.copy(a)
    u.steps, u.warmup = 2, 1
    au = measure_active_update(u)
    out["active_update"] = {"workload": au["config"]["workload"], "ms": au["ms_per_step"],
                            "ms_per_subsampled_view": au["ms_per_subsampled_view"],
                            "active_fraction_after": au["active_fraction_after"],
                            "commit_all_views_after_update_ms": au["commit_all_views_after_update_ms"],
                            "stage_overhead_ms_per_iteration_at_interval_500":
                                au["stage_overhead_ms_per_iteration_at_interval_500"]}
    torch.cuda.empty_cache()
    out["wall_s"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--quick", action="store_true", help="smaller scene (debug only)")
    ap.add_argument("--fractions", default=None,
                    help="comma list of active fractions to time (default 0.01,0.05,0.2,1); must include 0.05")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end and stage-update timings")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the summaries of the tiny, clustered, batched, precision and update workloads")
    ap.add_argument("--fwd-strip", type=int, default=0, help="forward raster pixels per thread (1, 2, 4; 0 = default)")
    ap.add_argument("--proj-lanes", type=int, default=0, help="projection lanes per splat (4, 16; 0 = default)")
    ap.add_argument("--bwd-walk", type=int, default=0, help="backward raster splat order (1 sorted by first row, 2 arena order, 0 default)")
    ap.add_argument("--persistent", type=int, default=0,
                    help="rasters as persistent blocks over a tile queue (1 on, -1 off, 0 default)")
    ap.add_argument("--tile-order", type=int, default=0, help="rasters take tiles heaviest first (1 on, -1 off, 0 default)")
    ap.add_argument("--workload", default="unbounded", choices=["unbounded", "batched", "precision", "active_update",
                                                                  "bwd_ablation", "tiny", "clustered"],
                    help="unbounded (default line): 1M splats, one view; batched: 3M splats, 16 views; "
                         "precision: 3M splats, 8 views, BF16 vs FP32 SH")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return
    if args.workload == "active_update":
        run_active_update(args)
        return
    if args.workload == "bwd_ablation":
        run_bwd_ablation(args)
        return
    if args.workload in ("tiny", "clustered"):
        run_small(args, args.workload)
        return

    import torch
    import __graft_entry__
    from paper_2605_13855_gb300 import scenes
    from paper_2605_13855_gb300.renderer import Renderer, SplatParams

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2605_13855_gb300 import _lib
    _lib.load()
    dev = torch.device("cuda", local)

    n = 100_000 if args.quick else scenes.UNBOUNDED["n"]
    W, H = scenes.UNBOUNDED["width"], scenes.UNBOUNDED["height"]
    scene = scenes.unbounded_scene(n, scenes.UNBOUNDED["seed"])
    # weak scaling: every rank renders its own view of the same scene
    cam_seed, target_seed = rank_camera_seeds(rank, scenes.UNBOUNDED["seed"])
    cam = scenes.random_camera(cam_seed, W, H)
    target_np = scenes.uniform_target(target_seed, W, H)
    sp = SplatParams.from_numpy(scene, device=dev)
    target = torch.as_tensor(target_np, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def make(fraction, seed_shift=0):
        m = scenes.proxy_active_mask(scene["means"], fraction, scenes.UNBOUNDED["seed"] + 2 + seed_shift)
        return torch.as_tensor(m, device=dev)

    r = Renderer(n, [(W, H)], max_pairs=1 << 27, fwd_pixels_per_thread=args.fwd_strip,
                 proj_lanes_per_splat=args.proj_lanes, bwd_walk=args.bwd_walk,
                 raster_tile_order=args.tile_order, raster_persistent=args.persistent)
    img = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)

    def grads_for(na):
        out = {k: torch.empty((na,) + s, dtype=torch.float32, device=dev) for k, s in
               (("means", (3,)), ("quats", (4,)), ("log_scales", (3,)), ("opacity_logits", ()),
                ("sh_color", (16, 3)), ("sh_weight", (16,)))}
        out["sigma"] = torch.empty(1, dtype=torch.float32, device=dev)
        return out

    def step(out, p):
        r.forward(p, [cam], [0], targets=[target], stream=stream, images=[img], loss=loss)
        r.backward(p, stream=stream, out=out)

    def timed(fraction, steps, warmup, profile=False):
        """The step on the stage layout: the active rows are gathered once when the active set is set
        (the active set, and so the gathered rows, stay fixed for the update interval of Sec. 4.1;
        the gather is reported, not timed in the step)."""
        mask = make(fraction)
        with torch.cuda.stream(stream):
            r.set_active(mask, stream=stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            ev1.record(stream)
            stream.synchronize()
            commit_ms = ev0.elapsed_time(ev1)
            ev0.record(stream)
            p = r.gather_active(sp, stream=stream)
            ev1.record(stream)
            stream.synchronize()
            gather_ms = ev0.elapsed_time(ev1)
            out = grads_for(r.n_active)
            # size the pair arena, count E and M (untimed)
            r.set_counting(True)
            step(out, p)
            r.status(stream)
            r.set_counting(False)
            M, E = r.last_counts(stream)
            for _ in range(warmup):
                step(out, p)
            stream.synchronize()
            # CUDA graph of one step (no host work between the kernels)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                step(out, p)
            for _ in range(2):
                g.replay()
            stream.synchronize()
            times = []
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.replay()
                b.record(stream)
                stream.synchronize()
                times.append(a.elapsed_time(b))
            prof = None
            if profile:
                r.set_profiling(True)
                r.get_profile()
                for _ in range(steps):
                    flush.zero_()
                    step(out, p)
                stream.synchronize()
                prof = r.get_profile()
                r.set_profiling(False)
            r.status(stream)
            del g
        return dict(ms=float(np.mean(times)), ms_min=float(np.min(times)), E=E, M=M, n_active=r.n_active,
                    commit_recompute_ms=commit_ms, gather_ms=gather_ms, prof=prof, out=out, mask=mask, p=p)

    results = {}
    clock_path = os.path.join(_clock_dir(), f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clock_path), exist_ok=True)
    fr_list = [HEADLINE_FRACTION, 1.0] if args.no_sweep else list(FRACTIONS)
    if args.fractions:
        fr_list = sorted({float(x) for x in args.fractions.split(",")} | {HEADLINE_FRACTION})
    with ClockSampler(clock_path) as clk:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for f in fr_list:
            results[f] = timed(f, args.steps, args.warmup, profile=(f in (HEADLINE_FRACTION, 1.0)))
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    clocks = clk.summary()

    head = results[HEADLINE_FRACTION]
    ms = head["ms"]
    if ws > 1:
        ms, total_E = reduce_over_ranks(ms, head["E"], device=dev)
    else:
        total_E = float(head["E"])
    value = total_E / (ms * 1e-3)

    set_active_ms = commit_inc_ms = async_host_ms = async_dev_ms = sync_host_ms = None
    e2e_ms, h2d, d2h = None, 0, 0
    train = dssim = None
    if not args.no_e2e:
        # active-set update (compaction of a changed mask) and the delayed,
        # incremental frozen-sum update it implies
        with torch.cuda.stream(stream):
            r.set_active(make(HEADLINE_FRACTION), stream=stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            m2 = make(HEADLINE_FRACTION, seed_shift=1)
            m3 = make(HEADLINE_FRACTION, seed_shift=2)
            stream.synchronize()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            # a GPU sleep ahead of the events keeps the stream busy while the host enqueues the
            # call, so that the events time the device work alone (the host time is taken apart)
            torch.cuda._sleep(2_000_000)
            a.record(stream)
            r.set_active(m2, stream=stream)
            b.record(stream)
            r.commit_frozen(sp, cam, 0, mode="incremental", stream=stream)
            c.record(stream)
            stream.synchronize()
            set_active_ms, commit_inc_ms = a.elapsed_time(b), b.elapsed_time(c)
            # the same update without the host wait (sparseoit_set_active_async); then the
            # headline's changed set again
            torch.cuda._sleep(2_000_000)
            a.record(stream)
            t0 = time.perf_counter()
            r.set_active(m3, stream=stream, asynchronous=True)
            async_host_ms = (time.perf_counter() - t0) * 1e3
            b.record(stream)
            stream.synchronize()
            async_dev_ms = a.elapsed_time(b)
            # host time of the synchronising call on an idle stream (back to the changed set)
            t0 = time.perf_counter()
            r.set_active(m2, stream=stream)
            sync_host_ms = (time.perf_counter() - t0) * 1e3
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            stream.synchronize()

        # end to end through the public API with host buffers, on the stage layout of the headline
        # step: every step copies the active rows (the parameters the step trains) and the target from
        # pinned host memory and reads back the compact gradients and the loss; the complement enters
        # as its committed frozen sums, which stay on the device for the whole active stage
        def e2e_time(params, host, host_target):
            out = grads_for(r.n_active)
            host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
            host_loss = torch.empty(1).pin_memory()
            h2d_ = sum(v.numel() * v.element_size() for v in host.values()) + host_target.numel() * 4
            d2h_ = sum(v.numel() * v.element_size() for v in out.values()) + 4

            def e2e_step():
                for k, v in host.items():
                    getattr(params, k).copy_(v, non_blocking=True)
                target.copy_(host_target, non_blocking=True)
                step(out, params)
                for k, v in out.items():
                    host_out[k].copy_(v, non_blocking=True)
                host_loss.copy_(loss, non_blocking=True)

            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    e2e_step()
                stream.synchronize()
                e_times = []
                for _ in range(args.steps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    e2e_step()
                    b.record(stream)
                    stream.synchronize()
                    e_times.append(a.elapsed_time(b))
            return float(np.mean(e_times)), h2d_, d2h_

        def e2e_pipelined(params, host, host_target):
            """The same step streamed: each step's inputs are copied in on a copy stream while the
            previous step computes, and its results copied out on a third stream while the next
            computes (two device slots of inputs, gradients and loss, ordered by events). The L2
            flush is written before every step inside the timed region. Returns ms per step."""
            from paper_2605_13855_gb300.renderer import SplatParams
            slots = []
            for sidx in range(2):
                pp = params if sidx == 0 else SplatParams(*[getattr(params, k).clone() for k in PARAM_NAMES],
                                                         params.sigma, params.bg, active_rows=params.active_rows)
                o = grads_for(r.n_active)
                slots.append(dict(p=pp, t=torch.empty_like(target), o=o, l=torch.zeros(1, device=dev),
                                  ho={k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in o.items()},
                                  hl=torch.empty(1).pin_memory()))
            s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
            ev_in = [torch.cuda.Event() for _ in range(2)]
            ev_done = [torch.cuda.Event() for _ in range(2)]
            ev_out = [torch.cuda.Event() for _ in range(2)]

            def issue(k):
                sl = slots[k % 2]
                with torch.cuda.stream(s_in):
                    if k >= 2:
                        s_in.wait_event(ev_done[k % 2])  # step k - 2 has read this slot's inputs
                    for name, v in host.items():
                        getattr(sl["p"], name).copy_(v, non_blocking=True)
                    sl["t"].copy_(host_target, non_blocking=True)
                    ev_in[k % 2].record(s_in)
                with torch.cuda.stream(stream):
                    stream.wait_event(ev_in[k % 2])
                    if k >= 2:
                        stream.wait_event(ev_out[k % 2])  # step k - 2's results have been copied out
                    flush.zero_()
                    r.forward(sl["p"], [cam], [0], targets=[sl["t"]], stream=stream, images=[img], loss=sl["l"])
                    r.backward(sl["p"], stream=stream, out=sl["o"])
                    ev_done[k % 2].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[k % 2])
                    for name, v in sl["o"].items():
                        sl["ho"][name].copy_(v, non_blocking=True)
                    sl["hl"].copy_(sl["l"], non_blocking=True)
                    ev_out[k % 2].record(s_out)

            for k in range(args.warmup):
                issue(k)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s_in)
            for k in range(args.steps):
                issue(k)
            b.record(s_out)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / args.steps

        from paper_2605_13855_gb300.renderer import PARAM_NAMES
        host_target = target.cpu().pin_memory()
        with torch.cuda.stream(stream):
            r.set_active(make(HEADLINE_FRACTION), stream=stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            spa_e = r.gather_active(sp, stream=stream)
            stream.synchronize()
        host_a = {k: getattr(spa_e, k).cpu().pin_memory() for k in PARAM_NAMES}
        e2e_serial_ms, h2d, d2h = e2e_time(spa_e, host_a, host_target)
        e2e_ms = e2e_pipelined(spa_e, host_a, host_target)
        # the same with the whole parameter arrays (rows by splat, 1M splats) copied every step
        host_full = {k: getattr(sp, k).cpu().pin_memory() for k in PARAM_NAMES}
        e2e_full_serial_ms, h2d_full, d2h_full = e2e_time(sp, host_full, host_target)
        e2e_full_ms = e2e_pipelined(sp, host_full, host_target)
        del host_full
        if ws > 1:
            e2e_ms, _ = reduce_over_ranks(e2e_ms, 0.0, device=dev)

        # a whole training iteration of the active-set loop: the step plus the sparse Adam update
        # of the active rows (in place on copies of the parameters, moments by splat)
        from paper_2605_13855_gb300.renderer import PARAM_NAMES, SplatParams
        spt = SplatParams(*[getattr(sp, k).clone() for k in PARAM_NAMES], sp.sigma, sp.bg)
        P = {k: getattr(spt, k) for k in PARAM_NAMES}
        P["sigma"] = torch.tensor([sp.sigma], dtype=torch.float32, device=dev)
        Mo = {k: torch.zeros_like(v) for k, v in P.items()}
        Vo = {k: torch.zeros_like(v) for k, v in P.items()}
        lr = [1.6e-4, 1e-3, 5e-3, 1e-2, 2.5e-3, 1.25e-4, 5e-3, 0.1]
        with torch.cuda.stream(stream):
            r.set_active(make(HEADLINE_FRACTION), stream=stream)
            r.commit_frozen(spt, cam, 0, mode="recompute", stream=stream)
            out = grads_for(r.n_active)

        def train_step():
            r.forward(spt, [cam], [0], targets=[target], stream=stream, images=[img], loss=loss)
            r.backward(spt, stream=stream, out=out)
            r.adam_step(out, P, Mo, Vo, lr, 100, stream=stream)

        train_ms = _graph_time(torch, stream, flush, train_step, args.steps, args.warmup)
        with torch.cuda.stream(stream):
            r.set_profiling(True)
            r.get_profile()
            for _ in range(args.steps):
                flush.zero_()
                r.adam_step(out, P, Mo, Vo, lr, 100, stream=stream)
            stream.synchronize()
            adam_prof = r.get_profile().get("adam", (1, 0.0))
            r.set_profiling(False)
        adam_ms = adam_prof[1] / max(1, adam_prof[0])
        adam_bytes = r.n_active * (4 + 300 + 3 * 600)  # index, compact grads, (p, m, v) read + write
        # the same step with the 3DGS loss (0.8 L1 + 0.2 D-SSIM) instead of the fused L1
        def dssim_step():
            r.forward(spt, [cam], [0], stream=stream, images=[img])
            r.loss_l1_dssim([target], 0.2, stream=stream, loss=loss)
            r.backward(spt, stream=stream, out=out)

        dssim_ms = _graph_time(torch, stream, flush, dssim_step, args.steps, args.warmup)
        with torch.cuda.stream(stream):
            r.set_profiling(True)
            r.get_profile()
            for _ in range(args.steps):
                flush.zero_()
                dssim_step()
            stream.synchronize()
            ssim_prof = r.get_profile().get("ssim", (1, 0.0))
            r.set_profiling(False)
        ssim_ms = ssim_prof[1] / max(1, ssim_prof[0])
        # per pixel: image + target read twice (x, y) = 48 B, 9 maps written and read = 72 B,
        # (F, T, Q) read and the state written = 40 B
        ssim_bytes = W * H * (48 + 72 + 40)
        dssim = {"step_ms": dssim_ms, "ssim_kernels_ms": ssim_ms,
                 "ssim_gbs": ssim_bytes / (ssim_ms * 1e-3) / 1e9, "ssim_algorithmic_bytes": ssim_bytes}
        # the stage layout: the active rows gathered once per stage, the step and Adam on them
        with torch.cuda.stream(stream):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            spa = r.gather_active(spt, stream=stream)
            ev1.record(stream)
            stream.synchronize()
            gather_ms = ev0.elapsed_time(ev1)
            Pa = {k: getattr(spa, k) for k in PARAM_NAMES}
            Pa["sigma"] = P["sigma"]
            Ma = {k: torch.zeros_like(v) for k, v in Pa.items()}
            Va = {k: torch.zeros_like(v) for k, v in Pa.items()}

        def step_active_rows():
            r.forward(spa, [cam], [0], targets=[target], stream=stream, images=[img], loss=loss)
            r.backward(spa, stream=stream, out=out)

        def train_active_rows():
            step_active_rows()
            r.adam_step(out, Pa, Ma, Va, lr, 100, stream=stream)

        step_rows_ms = _graph_time(torch, stream, flush, step_active_rows, args.steps, args.warmup)
        train_rows_ms = _graph_time(torch, stream, flush, train_active_rows, args.steps, args.warmup)
        with torch.cuda.stream(stream):
            r.set_profiling(True)
            r.get_profile()
            for _ in range(args.steps):
                flush.zero_()
                train_active_rows()
            stream.synchronize()
            prof_rows = r.get_profile()
            r.set_profiling(False)
        # end to end on the stage layout: each step copies the active rows (not the whole scene) and
        # the target from pinned host memory and reads back the compact gradients and the loss
        host_a = {k: getattr(spa, k).cpu().pin_memory() for k in PARAM_NAMES}
        host_target = target.cpu().pin_memory()
        host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
        host_loss = torch.empty(1).pin_memory()
        h2d_a = sum(v.numel() * v.element_size() for v in host_a.values()) + host_target.numel() * 4
        d2h_a = sum(v.numel() * v.element_size() for v in out.values()) + 4

        def e2e_rows_step():
            for k, v in host_a.items():
                getattr(spa, k).copy_(v, non_blocking=True)
            target.copy_(host_target, non_blocking=True)
            step_active_rows()
            for k, v in out.items():
                host_out[k].copy_(v, non_blocking=True)
            host_loss.copy_(loss, non_blocking=True)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                e2e_rows_step()
            stream.synchronize()
            e_t = []
            for _ in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                e2e_rows_step()
                b.record(stream)
                stream.synchronize()
                e_t.append(a.elapsed_time(b))
        active_rows = {"gather_ms_per_stage": gather_ms, "step_ms": step_rows_ms, "train_iteration_ms": train_rows_ms,
                       "per_kernel_ms": {k: v[1] / max(1, v[0]) for k, v in prof_rows.items()},
                       "e2e": {"ms_per_step": float(np.mean(e_t)), "value": head["E"] / (float(np.mean(e_t)) * 1e-3),
                               "unit": UNIT, "h2d_bytes_per_step": int(h2d_a), "d2h_bytes_per_step": int(d2h_a)}}
        train = {"ms": train_ms, "adam_ms": adam_ms, "adam_gbs": adam_bytes / (adam_ms * 1e-3) / 1e9,
                 "adam_hbm_frac": adam_bytes / (adam_ms * 1e-3) / 1e9 / float(_peaks()[0].get("hbm_gbs", 6800.0)),
                 "adam_algorithmic_bytes": adam_bytes, "active_rows_layout": active_rows}

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, peak_kind = _peaks()
    prof = head["prof"] or {}
    per_kernel = {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0])} for k, v in prof.items()}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["avg_ms"]) if per_kernel else None
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = device_sms(torch, dev)
    peak_tf = fp32_peak_tflops(sm_max, n_sms)
    roofline = None
    if dom is not None:
        avg_s = per_kernel[dom]["avg_ms"] * 1e-3
        flops = head["E"] * (FLOPS_BWD_PER_EVAL if dom == "raster_bwd" else FLOPS_FWD_PER_EVAL)
        if dom in ("raster_bwd", "raster_fwd"):
            ach = flops / avg_s / 1e12
            roofline = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                        "frac": ach / peak_tf, "traffic": recorded_traffic(dom),
                        "peak_source": f"{n_sms} SMs (device properties) x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz of "
                                       f"MEASURED_PEAKS.json, {peak_kind})",
                        "algorithmic": f"E={head['E']} pairs x {FLOPS_BWD_PER_EVAL if dom == 'raster_bwd' else FLOPS_FWD_PER_EVAL} FP32 ops"}
    # FP32 issue-bound rasters: achieved flops of both against the FP32 peak
    fp32 = {}
    for k, per in (("raster_fwd", FLOPS_FWD_PER_EVAL), ("raster_bwd", FLOPS_BWD_PER_EVAL)):
        if k in per_kernel and per_kernel[k]["avg_ms"] > 0:
            ach = head["E"] * per / (per_kernel[k]["avg_ms"] * 1e-3) / 1e12
            fp32[k] = {"achieved_tflops": ach, "frac": ach / peak_tf, "flops_per_pair": per}
    gpu_launches = 6 * args.steps  # project, scan, scatter, raster_fwd, raster_bwd, project_bwd
    n_tiles = ((W + 15) // 16) * ((H + 15) // 16)
    hbm = hbm_report(per_kernel, head["n_active"], head["M"], W * H, n_tiles, ms, peaks, peak_kind)

    configs = None
    if not args.no_configs and ws == 1:
        configs = config_summaries(args, torch, dev)

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_sample(scene, cam, target_np, head["mask"].cpu().numpy().astype(bool))

    full = results.get(1.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_splats": n, "width": W, "height": H,
                   "active_fraction": HEADLINE_FRACTION, "n_active": head["n_active"],
                   "evals_per_step": head["E"], "pairs_per_step": head["M"],
                   "evals_tile_per_step": 256 * head["M"],
                   "l2": "flushed between timed steps (256 MiB write)", "timing": "CUDA graph replay, CUDA events",
                   "layout": "stage layout: the active rows gathered once when the active set is set (fixed for "
                             "the update interval, Sec. 4.1), the complement as committed frozen sums",
                   "parallelism": f"dp{ws} (one view per rank)"},
        "active_vs_full": None if full is None else {
            "ms_active": ms, "ms_full": full["ms"], "speedup": full["ms"] / ms,
            "evals_full": full["E"], "value_full": full["E"] / (full["ms"] * 1e-3)},
        "fractions": {str(f): {"ms": v["ms"], "ms_min": v["ms_min"], "evals": v["E"], "pairs": v["M"],
                               "n_active": v["n_active"], "commit_recompute_ms": v["commit_recompute_ms"],
                               "gather_active_rows_ms": v["gather_ms"]}
                      for f, v in results.items()},
        "per_kernel_ms_full": None if full is None or not full["prof"] else {
            k: {"launches": n_, "avg_ms": t_ / max(1, n_)} for k, (n_, t_) in full["prof"].items()},
        "stage_update": {"set_active_ms": set_active_ms, "set_active_host_call_ms": sync_host_ms,
                         "commit_incremental_ms": commit_inc_ms,
                         "set_active_async": {"host_call_ms": async_host_ms, "device_ms": async_dev_ms},
                         "timing": "device times from CUDA events with the call queued behind a GPU sleep; "
                                   "host call times with perf_counter"},
        "per_kernel_ms": per_kernel,
        "roofline": roofline,
        "fp32": {"peak_tflops": peak_tf, "per_kernel": fp32},
        "train_iteration_with_sparse_adam": train,
        "step_with_l1_dssim_loss": dssim,
        "evals_tile_per_s": 256 * head["M"] / (ms * 1e-3),
        "hbm": hbm,
        "cpu_baseline": cpu,
        "e2e": None if e2e_ms is None else {
            "value": total_E / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "copies": "the active rows of every parameter array and the target in, the compact gradients and "
                      "the loss out, each step (stage layout)",
            "pipelining": "each step's copies in on a copy stream during the previous step, its results out on a "
                          "third stream during the next (two device slots, event-ordered); L2 flushed before every "
                          "step inside the timed region",
            "serial": {"value": total_E / (e2e_serial_ms * 1e-3), "ms_per_step": e2e_serial_ms,
                       "note": "copies in, step, copies out, one step at a time"},
            "full_parameter_copy": {"value": total_E / (e2e_full_ms * 1e-3), "ms_per_step": e2e_full_ms,
                                    "serial_ms_per_step": e2e_full_serial_ms,
                                    "h2d_bytes_per_step": int(h2d_full), "d2h_bytes_per_step": int(d2h_full)}},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
