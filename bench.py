#!/usr/bin/env python
"""Benchmark of the CaRtGS mapping iteration on GB300.

Workload: a 16-view 1200x680 keyframe window of a 300k-Gaussian SH-degree-3 room
scene (opacity logits N(-1, 1.5)), synthetic and seeded.  One step = one batched
window iteration: preprocess, bin sort, forward blend + L1 RGB/depth loss, backward,
densification statistics, fused Adam -- replayed from a captured CUDA graph with
every input resident in HBM (the working set is several GB, larger than L2).

Prints ONE JSON line (rank 0).  Besides the timed value it reports the same
iteration in the plain per-view form, the end-to-end rate through the public API
with the window's inputs copied from pinned host memory every step, a per-stage
breakdown, the roofline of the dominant kernel, and the FP64 oracle timed on the
host cores as a CPU baseline.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

METRIC = "mapping window iterations/s (fwd+bwd+Adam)"
UNIT = "window_iter/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0

# Work model of the raster kernels, in FP32 instructions per (splat, pixel) pair, counted
# from the kernel source: evaluating a pair (offsets, exponent, exp, alpha, tests) and,
# for a blended pair, the extra blend / gradient work.
FWD_OPS_EVAL, FWD_OPS_BLEND = 13, 11
BWD_OPS_EVAL, BWD_OPS_BLEND = 13, 55


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--batch-depth", type=int, default=128, help="splats per staged batch, forward")
    ap.add_argument("--batch-depth-bwd", type=int, default=64, help="splats per staged batch, backward")
    ap.add_argument("--autotune", action="store_true", help="pick tile/batch depth by measurement first")
    ap.add_argument("--no-per-view", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stages", action="store_true")
    ap.add_argument("--no-splat", action="store_true", help="skip the splat-wise backward head-to-head")
    ap.add_argument("--no-ssim", action="store_true", help="skip the timing of the loss with its SSIM term")
    ap.add_argument("--lambda-ssim", type=float, default=0.2)
    return ap.parse_args()


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.proc = None
        self.out = None
        self.uuid = device_uuid

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------- oracle side

def oracle_view_iteration(sc, v, row0=0, rows=None, lambda_d=0.1):
    """One view-iteration of the FP64 oracle on rows [row0, row0+rows) of view v (a crop is
    the same sub-problem: cy shifted, tile-aligned rows).  Targets are the oracle's render
    of the perturbed copy.  Returns seconds spent on the timed part (fwd+bwd, not targets)."""
    from oracle import oracle as O
    H = sc.height if rows is None else rows
    cam = sc.cams[v:v + 1].astype(np.float64).copy()
    cam[0, 15] -= row0
    pre_t = O.preprocess(sc.params_target, sc.n, sc.sh_degree, cam, sc.width, H, sc.tile)
    r = pre_t["rec"]
    rg, vl = O.bin_lists(r[:, 0], r[:, 1], r[:, 9], pre_t["radius"], 1, sc.n, sc.width, H, sc.tile)
    tg = O.render_fwd(r, rg, vl, 1, sc.width, H, sc.tile, cam)
    t0 = time.perf_counter()
    O.iteration(sc.params, sc.n, sc.sh_degree, cam, sc.width, H, sc.tile, tg["img"], tg["depth"],
                lambda_d=lambda_d)
    return time.perf_counter() - t0


def oracle_adam_seconds(P):
    from oracle import oracle as O
    rng = np.random.default_rng(0)
    th, g = rng.normal(size=P), rng.normal(size=P)
    m, v = np.zeros(P), np.zeros(P)
    lr = np.full(P, 1e-3)
    t0 = time.perf_counter()
    O.adam(th, g, m, v, 1, lr)
    return time.perf_counter() - t0


def cpu_baseline(sc):
    """The oracle, as it stands, on a bounded sample: one full view-iteration of view 0
    (all Gaussians, full resolution) plus Adam on the whole parameter vector; scaled to
    window iterations/s (V view-iterations + one Adam per window)."""
    t_view = oracle_view_iteration(sc, 0)
    t_adam = oracle_adam_seconds(sc.params.size)
    t_window = sc.views * t_view + t_adam
    return {"value": 1.0 / t_window, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 of {sc.views} views at full resolution ({t_view:.2f} s) + Adam on all "
                      f"{sc.params.size} parameters ({t_adam:.2f} s), scaled to a {sc.views}-view window"}


def run_reference(args):
    """--impl reference: the FP64 oracle timed on the host cores on the same workload;
    each step is a bounded sample (a quarter-height, tile-aligned band of one view)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import make_scene
    sc = make_scene(args.config)
    band = (sc.height // 4 // sc.tile) * sc.tile
    bands = -(-sc.height // band)
    t_adam = oracle_adam_seconds(sc.params.size)
    for w in range(args.warmup):
        oracle_view_iteration(sc, w % sc.views, (w % bands) * band, min(band, sc.height - (w % bands) * band))
    ts = []
    for k in range(args.steps):
        b = k % bands
        rows = min(band, sc.height - b * band)
        ts.append(oracle_view_iteration(sc, k % sc.views, b * band, rows) * (sc.height / rows))
    t_window = sc.views * float(np.mean(ts)) + t_adam
    value = 1.0 / t_window
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_window,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded room scene, no dataset)",
        "config": workload_config(sc),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: a {band}-row band of one view at full width, all "
                                   f"{sc.n} Gaussians, fwd+bwd; scaled by {sc.height}/{band} rows and "
                                   f"{sc.views} views, plus Adam on all parameters ({t_adam:.2f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(sc, extra=None):
    cfg = {"workload": f"{sc.views}-view {sc.width}x{sc.height} window, {sc.n} Gaussians, SH degree "
                       f"{sc.sh_degree} (synthetic room, opacity logits N(-1,1.5))",
           "views": sc.views, "width": sc.width, "height": sc.height, "gaussians": sc.n,
           "sh_degree": sc.sh_degree, "parallelism": "replicas",
           "l2": "working set (params, Adam state, records, images, targets) > 129 MB L2; no flush"}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------- ours

def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's value (the job's timed region ends with its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps_per_rank: int, seconds: float) -> float:
    """Whole-job window iterations/s: every rank runs its own window (replicas), so the job
    completes world x steps windows in the slowest rank's time."""
    return world * steps_per_rank / seconds


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_00486_gb300 import _native as N
    from paper_2410_00486_gb300.window import MappingWindow
    from synth import make_scene

    sc = make_scene(args.config, seed=rank)   # independent replica per rank
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    params_t = torch.from_numpy(sc.params).to(dev)
    cams = torch.from_numpy(np.ascontiguousarray(sc.cams)).to(dev)

    # targets: the GPU render of the perturbed copy (set-up, untimed)
    tgt_win = MappingWindow(torch.from_numpy(sc.params_target).to(dev), n, sc.sh_degree, W, H, V,
                            tile=args.tile, batch_depth=args.batch_depth)
    tgt_win.set_window(cams, torch.zeros(V, 3, H, W), None)
    tgt_win.fit_capacity()
    tgt_win.forward(with_loss=False)
    tgt_rgb, tgt_d = tgt_win.img.clone(), tgt_win.depth.clone()
    del tgt_win

    tile, bd, bdb = args.tile, args.batch_depth, args.batch_depth_bwd
    tuned = None
    if args.autotune:
        from paper_2410_00486_gb300.autotune import autotune
        (tile, bd, bdb), res = autotune(params_t, n, sc.sh_degree, W, H, cams, tgt_rgb, tgt_d, log=log)
        tuned = {"x".join(map(str, c)): round(ms, 3) for c, ms in res.items()}

    win = MappingWindow(params_t.clone(), n, sc.sh_degree, W, H, V, tile=tile, batch_depth=bd,
                        batch_depth_bwd=bdb)
    win.set_window(cams, tgt_rgb, tgt_d)
    ninst = win.fit_capacity(1.25)
    win.capture()
    for _ in range(args.warmup):
        win.replay()
    torch.cuda.synchronize()
    if win.read_status()[0] != 0:
        raise SystemExit(f"device status {win.read_status()}")

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as clk:
        e0.record()
        for _ in range(args.steps):
            win.replay()
        e1.record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_max = max_over_ranks(e0.elapsed_time(e1), world, dev)
    value = job_throughput(world, args.steps, ms_max / 1e3)
    st = win.read_status()
    if st[0] != 0:
        raise SystemExit(f"device status after timing: {st}")
    # preprocess, count, scan, scatter, sort x2, order, fwd, loss reduce, raster bwd, preprocess bwd, adam,
    # step counter (the launch list of the captured iteration shows these 13 kernels per step)
    launches_per_step = 13
    gpu_launches = args.steps * launches_per_step

    # --- plain per-view form (same math, one view at a time), also graph-captured
    per_view = None
    if not args.no_per_view:
        pv = MappingWindow(params_t.clone(), n, sc.sh_degree, W, H, V, tile=tile, batch_depth=bd,
                           batch_depth_bwd=bdb, capacity=win.capacity)
        pv.set_window(cams, tgt_rgb, tgt_d)
        pv.step_per_view()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            pv.step_per_view()
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g):
            pv.step_per_view()
        for _ in range(args.warmup):
            g.replay()
        k = max(3, args.steps // 4)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(k):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        pv_ms = e0.elapsed_time(e1) / k
        per_view = {"value": 1e3 / pv_ms, "unit": UNIT, "ms_per_step": pv_ms, "steps": k,
                    "speedup_batched_vs_per_view": (value / world) / (1e3 / pv_ms)}
        del pv, g
        torch.cuda.empty_cache()

    # --- head to head: the paper's splat-wise backward (Fig. 4a) in the same iteration
    splat = None
    if not args.no_splat and tile in (8, 16):
        splat = splat_head_to_head(MappingWindow, params_t, sc, tile, bd, cams, tgt_rgb, tgt_d, win.capacity,
                                   max(3, args.steps // 4), args.warmup, value / world)

    # --- the same iteration with the SSIM term of Eq. 9 in the loss
    ssim = None
    if not args.no_ssim:
        ssim = ssim_variant(MappingWindow, params_t, sc, tile, (bd, bdb), cams, tgt_rgb, tgt_d, win.capacity,
                            max(3, args.steps // 4), args.warmup, args.lambda_ssim)

    # --- stage breakdown (eager, CUDA events on the launching stream)
    stages = None
    work = None
    if not args.no_stages:
        stages, work = stage_breakdown(win, N, reps=5)

    # --- end to end through the public API: inputs from pinned host memory every step,
    #     the per-view losses read back; keyframe weights from the adaptive scheduler
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(win, sc, cams, tgt_rgb, tgt_d, args, torch, N)
        if world > 1:
            e2e["value"] = job_throughput(world, e2e["steps"], max_over_ranks(e2e["seconds"], world, dev))

    roof = None
    if stages:
        work["workload"] = workload_config(sc)["workload"]
        roof = roofline(stages, work, clk.summary())
        roof["iteration_bound_ms"] = round(iteration_bound_ms(stages, work), 4)
        roof["iteration_frac"] = roof["iteration_bound_ms"] / (ms_max / args.steps)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc)

    if rank == 0:
        extra = {"tile": tile, "batch_depth": bd, "batch_depth_bwd": bdb, "tile_instances": ninst}
        if tuned:
            extra["autotune_ms"] = tuned
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded room scene)",
            "config": workload_config(sc, extra),
            "view_iters_per_s": value * V,
            "per_view_form": per_view,
            "splat_backward": splat,
            "ssim_loss_form": ssim,
            "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
            if e2e else None,
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "stages_ms": stages,
            "roofline": roof,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def splat_head_to_head(MappingWindow, params_t, sc, tile, bd, cams, tgt_rgb, tgt_d, capacity, k, warmup,
                       pixel_value):
    """Window iterations/s with the splat-wise backward (forward saving per-pixel states every
    32 splats), plus its forward and backward stage times."""
    import torch
    from paper_2410_00486_gb300 import _native as N
    w = MappingWindow(params_t.clone(), sc.n, sc.sh_degree, sc.width, sc.height, sc.views, tile=tile,
                      batch_depth=bd, capacity=capacity, backward="splat")
    w.set_window(cams, tgt_rgb, tgt_d)
    w.capture()
    for _ in range(warmup):
        w.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(k):
        w.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    st = w.read_status()
    if st[0] != 0:
        raise SystemExit(f"device status (splat-wise backward): {st}")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    N.cgs_preprocess(w.params, w.n, w.cams, w.V, w.cfg, w.rec, w.slot_grad, w.status)
    N.cgs_bin_sort(w.rec, w.n, w.V, w.cfg, w.bin_ws, w.capacity, w.vals, w.ranges, w.order, w.n_inst, w.status)
    ev[0].record()
    N.cgs_render_fwd_ckpt(w.rec, w.vals, w.ranges, w.order, w.V, w.cfg, w.view_weight, w.tgt_rgb, w.tgt_depth,
                          w.img, w.depth, w.t_final, w.last, w.loss_view, w.depth_count, w.fwd_ws, w.ckpt,
                          w.max_buckets, w.bucket_start, w.status)
    ev[1].record()
    N.cgs_raster_bwd_splat(w.rec, w.vals, w.ranges, w.order, w.V, w.cfg, w.view_weight, w.img, w.depth,
                           w.t_final, w.last, w.tgt_rgb, w.tgt_depth, w.depth_count, None, None, w.ckpt,
                           w.max_buckets, w.bucket_start, w.slot_grad, w.status)
    ev[2].record()
    torch.cuda.synchronize()
    out = {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "steps": k,
           "render_fwd_ckpt_ms": round(ev[0].elapsed_time(ev[1]), 4),
           "raster_bwd_splat_ms": round(ev[1].elapsed_time(ev[2]), 4),
           "checkpoint_buckets": int(w.bucket_start[-1].item()),
           "pixel_wise_over_splat_wise": pixel_value / (1e3 / ms)}
    del w
    torch.cuda.empty_cache()
    return out


def ssim_variant(MappingWindow, params_t, sc, tile, bd, cams, tgt_rgb, tgt_d, capacity, k, warmup, lam):
    """Window iterations/s with the loss of Eq. 9 including its SSIM term (weight lam), and the
    time of the SSIM loss stage alone."""
    import torch
    from paper_2410_00486_gb300 import _native as N
    w = MappingWindow(params_t.clone(), sc.n, sc.sh_degree, sc.width, sc.height, sc.views, tile=tile,
                      batch_depth=bd[0], batch_depth_bwd=bd[1], capacity=capacity, lambda_ssim=lam)
    w.set_window(cams, tgt_rgb, tgt_d)
    w.capture()
    for _ in range(warmup):
        w.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(k):
        w.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    st = w.read_status()
    if st[0] != 0:
        raise SystemExit(f"device status (SSIM loss): {st}")
    reps = 5
    e0.record()
    for _ in range(reps):
        N.cgs_ssim_loss(w.img, w.tgt_rgb, w.depth, w.tgt_depth, w.depth_count, w.V, w.cfg, w.view_weight, lam,
                        w.loss_view, w.dl_dimg, w.dl_ddepth, w.ssim_ws, w.status)
    e1.record()
    torch.cuda.synchronize()
    out = {"lambda_ssim": lam, "value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "steps": k,
           "ssim_loss_ms": round(e0.elapsed_time(e1) / reps, 4)}
    del w
    torch.cuda.empty_cache()
    return out


def stage_breakdown(win, N, reps=5):
    """Average ms per stage over `reps` eager iterations (no Adam updates between them
    change the work: Adam runs last)."""
    import torch
    names = ["preprocess", "bin_sort", "render_fwd", "raster_bwd", "preprocess_bwd", "adam"]
    acc = {k: 0.0 for k in names}
    c = win.cfg
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record()
        N.cgs_preprocess(win.params, win.n, win.cams, win.V, c, win.rec, win.slot_grad, win.status)
        ev[1].record()
        N.cgs_bin_sort(win.rec, win.n, win.V, c, win.bin_ws, win.capacity, win.vals, win.ranges, win.order,
                       win.n_inst, win.status)
        ev[2].record()
        N.cgs_render_fwd(win.rec, win.vals, win.ranges, win.order, win.V, c, win.view_weight, win.tgt_rgb,
                         win.tgt_depth, win.img, win.depth, win.t_final, win.last, win.loss_view,
                         win.depth_count, win.fwd_ws, win.status)
        ev[3].record()
        N.cgs_raster_bwd(win.rec, win.vals, win.ranges, win.order, win.V, c, win.view_weight, win.img, win.depth,
                         win.t_final, win.last, win.tgt_rgb, win.tgt_depth, win.depth_count, None, None,
                         win.slot_grad, win.status)
        ev[4].record()
        N.cgs_preprocess_bwd(win.params, win.n, win.cams, win.V, c, win.rec, win.slot_grad, win.grads, False,
                             win.accum, win.denom, win.max_r2d, win.status)
        ev[5].record()
        win.optimizer_step()
        ev[6].record()
        torch.cuda.synchronize()
        for i, k in enumerate(names):
            acc[k] += ev[i].elapsed_time(ev[i + 1]) / reps
    # work counts of this window (measurement only): one more forward over the same records
    # and lists with the blended-pair counter compiled in (the timed forward leaves it out)
    cc = type(c).from_buffer_copy(c)
    cc.count_work = 1
    N.cgs_render_fwd(win.rec, win.vals, win.ranges, win.order, win.V, cc, win.view_weight, win.tgt_rgb,
                     win.tgt_depth, win.img, win.depth, win.t_final, win.last, win.loss_view,
                     win.depth_count, win.fwd_ws, win.status)
    torch.cuda.synchronize()
    part = win.fwd_ws[: 4 * 5 * win.Ttot].view(torch.float32).view(win.Ttot, 5).double()
    rad = win.rec.view(torch.int32).view(-1, 12)[:, 7]
    work = {
        "pairs_fwd_eval": float(part[:, 3].sum()), "pairs_blend": float(part[:, 4].sum()),
        # every entry of a tile's list is staged (the binning keeps only splats that reach the
        # tile), so the backward evaluates each pixel's list up to its `last`
        "pairs_bwd_eval": float(win.last.double().sum()),
        "visible_slots": int((rad > 0).sum().item()), "instances": int(win.n_inst.item()),
        "params": win.P, "n": win.n, "slots": win.V * win.n, "pixels": win.V * win.W * win.H, "tiles": win.Ttot,
    }
    return {k: round(v, 4) for k, v in acc.items()}, work


def hbm_bytes(stage, w):
    """Algorithmic HBM bytes per launch: each input read once, each output written once."""
    P, S, M, I, X, T = w["params"], w["slots"], w["visible_slots"], w["instances"], w["pixels"], w["tiles"]
    if stage == "preprocess":
        return 4 * P + 4 * S + (48 + 48) * M          # params; radius of every slot; record + zeroed grad
    if stage == "bin_sort":
        return 4 * S + 12 * M + 8 * I + 8 * I + 4 * I + 8 * T   # scan rects, scatter keys, sort, vals, ranges
    if stage == "preprocess_bwd":
        return 4 * P + 4 * S + 48 * M + 4 * P + 24 * w["n"]   # params, radii, slot grads, grads, stats
    if stage == "adam":
        return 28 * P
    return None


TRAFFIC_PROFILE = ROOT / "profiles" / "k_render_bwd_traffic_window16_300k_1200x680.md"
RASTER_BWD_SOURCES = ("render_bwd.cu", "raster.cuh", "cgs_internal.cuh")


def raster_bwd_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in RASTER_BWD_SOURCES:
        h.update((ROOT / "paper_2410_00486_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()


def recorded_traffic(workload):
    """DRAM bytes per launch of k_render_bwd from the committed ncu capture, if it was taken on
    this workload and the kernel's sources are unchanged since (else None)."""
    if not TRAFFIC_PROFILE.exists():
        return None
    kv = {}
    for line in TRAFFIC_PROFILE.read_text().splitlines():
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("source_sha256") != raster_bwd_source_hash() or kv.get("workload") != workload:
        return None
    return float(kv["traffic_bytes_per_launch"])


def iteration_bound_ms(stages, work):
    """Time one iteration would take if every stage ran at its roofline: HBM stages at the
    measured copy bandwidth, raster stages at the FP32 lane peak (SURVEY-style combined bound)."""
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    bw = peaks.get("hbm_gbs", 6800.0) * 1e9
    alu = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6
    t = 0.0
    for st in stages:
        if st == "render_fwd":
            t += (FWD_OPS_EVAL * work["pairs_fwd_eval"] + FWD_OPS_BLEND * work["pairs_blend"]) / alu
        elif st == "raster_bwd":
            t += (BWD_OPS_EVAL * work["pairs_bwd_eval"] + BWD_OPS_BLEND * work["pairs_blend"]) / alu
        else:
            t += hbm_bytes(st, work) / bw
    return 1e3 * t


def roofline(stages, work, clocks):
    """Roofline of the dominant kernel: FP32-ALU bound for the raster kernels (peak = SMs x
    FP32 lanes x max SM clock), HBM bound for the rest (peak = measured copy bandwidth)."""
    dom = max(stages, key=stages.get)
    t = stages[dom] / 1e3
    peaks = {}
    mp = ROOT / "MEASURED_PEAKS.json"
    if mp.exists():
        peaks = json.loads(mp.read_text())
    if dom in ("render_fwd", "raster_bwd"):
        if dom == "render_fwd":
            ops = FWD_OPS_EVAL * work["pairs_fwd_eval"] + FWD_OPS_BLEND * work["pairs_blend"]
        else:
            ops = BWD_OPS_EVAL * work["pairs_bwd_eval"] + BWD_OPS_BLEND * work["pairs_blend"]
        peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
        ach = ops / t / 1e12
        traffic = recorded_traffic(work.get("workload")) if dom == "raster_bwd" else None
        return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Top/s",
                "frac": ach / peak, "traffic": traffic,
                "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (FP32 instructions/s), derived",
                "work": {k: work[k] for k in ("pairs_fwd_eval", "pairs_bwd_eval", "pairs_blend")},
                "ops_per_pair": {"fwd_eval": FWD_OPS_EVAL, "fwd_blend": FWD_OPS_BLEND, "bwd_eval": BWD_OPS_EVAL,
                                 "bwd_blend": BWD_OPS_BLEND}}
    b = hbm_bytes(dom, work)
    peak = peaks.get("hbm_gbs", 6800.0)
    ach = b / t / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}


def end_to_end(win, sc, cams, tgt_rgb, tgt_d, args, torch, N):
    """Steps through the public API: the adaptive scheduler (Eqs. 5-8) draws the window's
    view weights, the window's cameras, targets and weights are copied from pinned host
    memory (cameras and targets staged on a copy stream during the previous iteration),
    the captured iteration runs, and the per-view losses are read back and reported to the
    scheduler.  Every step copies the whole window's inputs."""
    from paper_2410_00486_gb300 import Scheduler
    V = sc.views
    h_cams = cams.cpu().pin_memory()
    h_rgb = tgt_rgb.cpu().pin_memory()
    h_d = tgt_d.cpu().pin_memory()
    h_w = torch.ones(V, dtype=torch.float32).pin_memory()
    h_loss = torch.zeros(V, dtype=torch.float32).pin_memory()
    sched = Scheduler(4)
    for v in range(V):
        sched.add(v, 8)
    rng = np.random.default_rng(0)

    done = torch.cuda.Event()

    def one_step():
        # the draws need the previous window's losses (reported below); the next window's
        # cameras and targets do not, so their copy is staged while this iteration runs
        counts = np.bincount(sched.draw_n(rng.integers(0, 2 ** 32, V, dtype=np.uint64).astype(np.uint32)),
                             minlength=V).astype(np.float32)
        h_w.copy_(torch.from_numpy(counts))
        win.set_view_weight(h_w)
        win.commit_window()
        win.replay()
        h_loss.copy_(win.loss_view, non_blocking=True)
        done.record()
        win.stage_window(h_cams, h_rgb, h_d)
        done.synchronize()
        drawn = np.nonzero(counts)[0]
        sched.report_n(drawn, h_loss.numpy()[drawn].astype(np.float64) / counts[drawn])

    win.stage_window(h_cams, h_rgb, h_d)
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = max(3, args.steps // 4)
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    h2d = h_cams.numel() * 4 + h_rgb.numel() * 4 + h_d.numel() * 4 + h_w.numel() * 4
    return {"value": steps / sec, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": V * 4,
            "seconds": sec, "steps": steps}


if __name__ == "__main__":
    main()
