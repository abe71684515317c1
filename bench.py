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


# FP32 operations of one contributing (splat, pixel) pair, counted from the
# arithmetic of the kernels' algorithm ("Roofline"): forward
# 16 (offset 2, quadratic form 5, threshold 1, exp 1, clamp 1, weight 1,
# P/Q 4, T 1), backward 44 (forward part 10, Eq. 10 terms 16, chain to the
# screen parameters 10, accumulation 8).
FLOPS_FWD_PER_EVAL = 16
FLOPS_BWD_PER_EVAL = 44


def fp32_peak_tflops(sm_mhz: float) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


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
    """The oracle as it stands, timed on the host cores: one fwd+bwd on a window sized to ~budget_s."""
    import oracle
    win = _calibrated_window(scene, cam, target, mask, budget_s)
    dt, evals = _oracle_timing(scene, cam, target, mask, win, 1, 0)
    return {"value": evals / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": _sample_text(win, evals, dt, 1)}


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
    ap.add_argument("--fwd-strip", type=int, default=0, help="forward raster pixels per thread (1, 2, 4; 0 = default)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
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
    cam = scenes.random_camera(scenes.UNBOUNDED["seed"] + 3 + 17 * rank, W, H)
    target_np = scenes.uniform_target(scenes.UNBOUNDED["seed"] + 1 + 17 * rank, W, H)
    sp = SplatParams.from_numpy(scene, device=dev)
    target = torch.as_tensor(target_np, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def make(fraction, seed_shift=0):
        m = scenes.proxy_active_mask(scene["means"], fraction, scenes.UNBOUNDED["seed"] + 2 + seed_shift)
        return torch.as_tensor(m, device=dev)

    r = Renderer(n, [(W, H)], max_pairs=1 << 27, fwd_pixels_per_thread=args.fwd_strip)
    img = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)

    def grads_for(na):
        out = {k: torch.empty((na,) + s, dtype=torch.float32, device=dev) for k, s in
               (("means", (3,)), ("quats", (4,)), ("log_scales", (3,)), ("opacity_logits", ()),
                ("sh_color", (16, 3)), ("sh_weight", (16,)))}
        out["sigma"] = torch.empty(1, dtype=torch.float32, device=dev)
        return out

    def step(out):
        r.forward(sp, [cam], [0], targets=[target], stream=stream, images=[img], loss=loss)
        r.backward(sp, stream=stream, out=out)

    def timed(fraction, steps, warmup, profile=False):
        mask = make(fraction)
        with torch.cuda.stream(stream):
            r.set_active(mask, stream=stream)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            ev1.record(stream)
            stream.synchronize()
            commit_ms = ev0.elapsed_time(ev1)
            out = grads_for(r.n_active)
            # size the pair arena, count E and M (untimed)
            r.set_counting(True)
            step(out)
            r.status(stream)
            r.set_counting(False)
            M, E = r.last_counts(stream)
            for _ in range(warmup):
                step(out)
            stream.synchronize()
            # CUDA graph of one step (no host work between the kernels)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                step(out)
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
                    step(out)
                stream.synchronize()
                prof = r.get_profile()
                r.set_profiling(False)
            r.status(stream)
            del g
        return dict(ms=float(np.mean(times)), ms_min=float(np.min(times)), E=E, M=M, n_active=r.n_active,
                    commit_recompute_ms=commit_ms, prof=prof, out=out, mask=mask)

    results = {}
    clock_path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clock_path), exist_ok=True)
    fr_list = [HEADLINE_FRACTION, 1.0] if args.no_sweep else list(FRACTIONS)
    if args.fractions:
        fr_list = sorted({float(x) for x in args.fractions.split(",")} | {HEADLINE_FRACTION})
    with ClockSampler(clock_path) as clk:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for f in fr_list:
            results[f] = timed(f, args.steps, args.warmup, profile=(f == HEADLINE_FRACTION))
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    clocks = clk.summary()

    head = results[HEADLINE_FRACTION]
    ms = head["ms"]
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        e = torch.tensor([float(head["E"])], device=dev)
        dist.all_reduce(e)
        total_E = float(e.item())
    else:
        total_E = float(head["E"])
    value = total_E / (ms * 1e-3)

    set_active_ms = commit_inc_ms = None
    e2e_ms, h2d, d2h = None, 0, 0
    if not args.no_e2e:
        # active-set update (compaction of a changed mask) and the delayed,
        # incremental frozen-sum update it implies
        with torch.cuda.stream(stream):
            r.set_active(make(HEADLINE_FRACTION), stream=stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            m2 = make(HEADLINE_FRACTION, seed_shift=1)
            stream.synchronize()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            r.set_active(m2, stream=stream)
            b.record(stream)
            r.commit_frozen(sp, cam, 0, mode="incremental", stream=stream)
            c.record(stream)
            stream.synchronize()
            set_active_ms, commit_inc_ms = a.elapsed_time(b), b.elapsed_time(c)

        # end to end through the public API with host buffers: every step copies
        # the full parameter arrays and the target from pinned host memory and
        # reads back the compact gradients and the loss
        host = {k: getattr(sp, k).cpu().pin_memory() for k in
                ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight")}
        host_target = target.cpu().pin_memory()
        with torch.cuda.stream(stream):
            r.set_active(make(HEADLINE_FRACTION), stream=stream)
            r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
            out = grads_for(r.n_active)
            host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
            host_loss = torch.empty(1).pin_memory()
            h2d = sum(v.numel() * v.element_size() for v in host.values()) + host_target.numel() * 4
            d2h = sum(v.numel() * v.element_size() for v in out.values()) + 4

            def e2e_step():
                for k, v in host.items():
                    getattr(sp, k).copy_(v, non_blocking=True)
                target.copy_(host_target, non_blocking=True)
                step(out)
                for k, v in out.items():
                    host_out[k].copy_(v, non_blocking=True)
                host_loss.copy_(loss, non_blocking=True)

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
        e2e_ms = float(np.mean(e_times))
        if ws > 1:
            import torch.distributed as dist
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, peak_kind = _peaks()
    prof = head["prof"] or {}
    per_kernel = {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0])} for k, v in prof.items()}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["avg_ms"]) if per_kernel else None
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tf = fp32_peak_tflops(sm_max)
    roofline = None
    if dom is not None:
        avg_s = per_kernel[dom]["avg_ms"] * 1e-3
        flops = head["E"] * (FLOPS_BWD_PER_EVAL if dom == "raster_bwd" else FLOPS_FWD_PER_EVAL)
        if dom in ("raster_bwd", "raster_fwd"):
            ach = flops / avg_s / 1e12
            roofline = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                        "frac": ach / peak_tf, "traffic": None,
                        "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz of "
                                       f"MEASURED_PEAKS.json, {peak_kind})",
                        "algorithmic": f"E={head['E']} pairs x {FLOPS_BWD_PER_EVAL if dom == 'raster_bwd' else FLOPS_FWD_PER_EVAL} FP32 ops"}
    gpu_launches = 6 * args.steps  # project, scan, scatter, raster_fwd, raster_bwd, project_bwd

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
                   "l2": "flushed between timed steps (256 MiB write)", "timing": "CUDA graph replay, CUDA events",
                   "parallelism": f"dp{ws} (one view per rank)"},
        "active_vs_full": None if full is None else {
            "ms_active": ms, "ms_full": full["ms"], "speedup": full["ms"] / ms,
            "evals_full": full["E"], "value_full": full["E"] / (full["ms"] * 1e-3)},
        "fractions": {str(f): {"ms": v["ms"], "ms_min": v["ms_min"], "evals": v["E"], "pairs": v["M"],
                               "n_active": v["n_active"], "commit_recompute_ms": v["commit_recompute_ms"]}
                      for f, v in results.items()},
        "stage_update": {"set_active_ms": set_active_ms, "commit_incremental_ms": commit_inc_ms},
        "per_kernel_ms": per_kernel,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": None if e2e_ms is None else {
            "value": total_E / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
