#!/usr/bin/env python
"""Benchmark of the CaRtGS mapping iteration on GB300.

Default workload: a 16-view 1200x680 keyframe window of a 300k-Gaussian SH-degree-3
room scene (opacity logits N(-1, 1.5)), synthetic and seeded; --config 1-4 picks the
other workload shapes (2k-Gaussian 160x120 view, 100k-Gaussian 1200x680 view, 5k-Gaussian
320x240 view, 8-view 640x480 window of 200k Gaussians).  One step = one batched window
iteration: preprocess, bin sort, forward blend + L1 RGB/depth loss, backward,
densification statistics, fused Adam -- replayed from a captured CUDA graph with every
input resident in HBM.

Prints ONE JSON line (rank 0).  Besides the timed value it reports the same iteration in
the plain per-view form and in the paper's sequential loop (Adam after every view), the
end-to-end rate through the public API with the window's inputs copied from pinned host
memory every step, per-stage times with each stage's roofline fraction, the whole
iteration's fraction of the HBM roofline, the roofline of the dominant kernel, and the
FP64 oracle timed on the host cores as a CPU baseline.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference] [--config 1-5]
"""
from __future__ import annotations

import argparse
import dataclasses
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
FP32_LANES_PER_SM = 128
TRAFFIC_FILE = ROOT / "ncu_traffic.json"

# Work model of the raster kernels: formula operations per (splat, pixel) pair, as the
# blend and its derivative are written out (Eq. 1, Eqs. 2-4): evaluating a pair (offsets,
# exponent, exp, alpha, the two threshold tests) and, for a blended pair, the extra blend
# (forward) or gradient (backward) work.  The kernels execute fewer instructions than this
# (shared column terms, one dot product for the colour behind), so the achieved rate is
# formula operations per second.
FWD_OPS_EVAL, FWD_OPS_BLEND = 13, 11
BWD_OPS_EVAL, BWD_OPS_BLEND = 13, 55
# Replays timed for each alternative form of the iteration (per-view, paper loop, splat-wise
# backward, SSIM loss, end to end): at least this many, or --steps if larger.
MIN_FORM_STEPS = 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--batch-depth", type=int, default=128, help="splats per staged batch, forward")
    ap.add_argument("--batch-depth-bwd", type=int, default=32, help="splats per staged batch, backward")
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

BAND_TILE_ROWS = 5      # a CPU sample step covers this many tile rows of every view


def oracle_targets_band(sc, row0, rows):
    """The oracle's render of the perturbed copy on rows [row0, row0 + rows) of every view
    (a crop is the same sub-problem with cy shifted): the targets of a sample step."""
    from oracle import oracle as O
    cams = sc.cams.astype(np.float64).copy()
    cams[:, 15] -= row0
    pre = O.preprocess(sc.params_target, sc.n, sc.sh_degree, cams, sc.width, rows, sc.tile)
    rg, vl = O.bin_records(pre["rec"], pre["radius"], sc.views, sc.n, sc.width, rows, sc.tile)
    tg = O.render_fwd(pre["rec"], rg, vl, sc.views, sc.width, rows, sc.tile, cams)
    return cams, tg["img"], tg["depth"]


def oracle_band_step(sc, cams, tgt_rgb, tgt_d, rows, views=None, lambda_d=0.1):
    """One sample step of the FP64 oracle, as it stands: the iteration's steps (projection,
    rect lists, blend + L1 loss, hand-derived backward, chain rule to the parameters) on a
    band of `rows` rows of every view (or of `views`).  Returns (seconds of the projection,
    seconds of the whole step)."""
    from oracle import oracle as O
    if views is not None:
        cams, tgt_rgb, tgt_d = cams[views], tgt_rgb[views], tgt_d[views]
    V = cams.shape[0]
    t0 = time.perf_counter()
    pre = O.preprocess(sc.params, sc.n, sc.sh_degree, cams, sc.width, rows, sc.tile)
    t1 = time.perf_counter()
    rec = pre["rec"]
    rg, vl = O.bin_records(rec, pre["radius"], V, sc.n, sc.width, rows, sc.tile)
    fw = O.render_fwd(rec, rg, vl, V, sc.width, rows, sc.tile, cams, (0.0, 0.0, 0.0), tgt_rgb, tgt_d, lambda_d)
    sg = O.render_bwd(rec, rg, vl, V, sc.n, sc.width, rows, sc.tile, cams, fw["img"], fw["depth"], tgt_rgb, tgt_d,
                      fw["depth_count"], (0.0, 0.0, 0.0), lambda_d)
    O.preprocess_bwd(sc.params, sc.n, sc.sh_degree, cams, sc.width, rows, sc.tile, sg)
    return t1 - t0, time.perf_counter() - t0


def oracle_adam_seconds(P):
    from oracle import oracle as O
    rng = np.random.default_rng(0)
    th, g = rng.normal(size=P), rng.normal(size=P)
    m, v = np.zeros(P), np.zeros(P)
    lr = np.full(P, 1e-3)
    t0 = time.perf_counter()
    O.adam(th, g, m, v, 1, lr)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def band_rows(sc):
    return min(sc.height, BAND_TILE_ROWS * sc.tile)


def window_seconds_from_band(sc, t_pre, t_step, rows, t_adam):
    """A window iteration's oracle time from a band sample: the projection of every Gaussian
    is paid once per window (measured on the band), the rest scales with the image rows, and
    Adam runs once on all parameters."""
    return t_pre + (sc.height / rows) * (t_step - t_pre) + t_adam


def cpu_baseline(sc):
    """The oracle, as it stands, on bounded samples of the workload: a band of tile rows of
    every view on all host cores, and the same band of one view on one core; each scaled to
    a window iteration (window_seconds_from_band) with Adam on all parameters."""
    from oracle import oracle as O
    cores = host_cores()
    rows = band_rows(sc)
    cams, tr, td = oracle_targets_band(sc, 0, rows)
    t_adam = oracle_adam_seconds(sc.params.size)
    O.set_threads(cores)
    t_pre, t_step = oracle_band_step(sc, cams, tr, td, rows)
    t_win = window_seconds_from_band(sc, t_pre, t_step, rows, t_adam)
    O.set_threads(1)
    t_pre1, t_step1 = oracle_band_step(sc, cams, tr, td, rows, views=[0])
    t_win1 = sc.views * (t_pre1 + (sc.height / rows) * (t_step1 - t_pre1)) + t_adam
    O.set_threads(cores)
    return {"value": 1.0 / t_win, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"rows 0-{rows - 1} of all {sc.views} views, all {sc.n} Gaussians, fwd+bwd on {cores} "
                      f"threads ({t_step:.2f} s, projection {t_pre:.2f} s), scaled to {sc.height} rows; "
                      f"+ Adam on all {sc.params.size} parameters ({t_adam:.2f} s)",
            "value_1core": 1.0 / t_win1,
            "sample_1core": f"the same band of view 0 on 1 thread ({t_step1:.2f} s), scaled to {sc.height} rows "
                            f"and {sc.views} views, + Adam"}


def run_reference(args):
    """--impl reference: the FP64 oracle, as it stands, timed on all host cores on the same
    workload; each step is a bounded sample (a band of tile rows of every view, the bands
    taken in turn), and the value is the window iterations/s those samples imply."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from synth import make_scene
    sc = dataclasses.replace(make_scene(args.config), tile=args.tile)   # the GPU arm's tile size
    cores = host_cores()
    O.set_threads(cores)
    rows = band_rows(sc)
    nb = max(1, sc.height // rows)                  # whole bands only
    targets = {}
    t_adam = oracle_adam_seconds(sc.params.size)
    ts = []
    t_run0 = time.perf_counter()
    for k in range(args.warmup + args.steps):
        b = k % nb
        if b not in targets:
            targets[b] = oracle_targets_band(sc, b * rows, rows)
        cams, tr, td = targets[b]
        t_pre, t_step = oracle_band_step(sc, cams, tr, td, rows)
        if k >= args.warmup:
            ts.append((t_pre, t_step))
    wall = time.perf_counter() - t_run0
    t_pre = float(np.mean([a for a, _ in ts]))
    t_step = float(np.mean([b for _, b in ts]))
    t_window = window_seconds_from_band(sc, t_pre, t_step, rows, t_adam)
    value = 1.0 / t_window
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded scene, no dataset)",
        "config": arm_config(sc, args.tile, args.batch_depth, args.batch_depth_bwd, args.config),
        "ms_per_window": 1e3 * t_window, "wall_s": round(wall, 2),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: a {rows}-row band of all {sc.views} views (bands of rows taken "
                                   f"in turn), all {sc.n} Gaussians, fwd+bwd on {cores} threads "
                                   f"({1e3 * t_step:.0f} ms, projection {1e3 * t_pre:.0f} ms); window time = "
                                   f"projection + {sc.height}/{rows} x the rest + Adam on all parameters "
                                   f"({t_adam:.2f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


WORKLOAD_TEXT = {
    1: "synthetic box scene",
    2: "synthetic room, Replica-like shape",
    3: "synthetic box scene",
    4: "synthetic room, TUM-like path with uneven visibility",
    5: "synthetic room, opacity logits N(-1,1.5)",
}


def arm_config(sc, tile, bd, bdb, config_index, extra=None):
    """The `config` object of both arms' lines: the workload and the launch shape (measured
    quantities such as the tile-instance count sit outside it)."""
    cfg = workload_config(sc, {"tile": tile, "batch_depth": bd, "batch_depth_bwd": bdb, "config_index": config_index})
    if extra:
        cfg.update(extra)
    return cfg


def workload_config(sc, extra=None):
    kind = next((t for c, t in WORKLOAD_TEXT.items() if sc.name == _config_name(c)), "synthetic scene")
    cfg = {"workload": f"{sc.views}-view {sc.width}x{sc.height} window, {sc.n} Gaussians, SH degree "
                       f"{sc.sh_degree} ({kind})",
           "views": sc.views, "width": sc.width, "height": sc.height, "gaussians": sc.n,
           "sh_degree": sc.sh_degree, "parallelism": "replicas",
           "l2": "working set (params, Adam state, records, images, targets) > 129 MB L2; no flush"
           if sc.n * sc.views >= 100_000 else "small case: no L2 flush between steps"}
    if extra:
        cfg.update(extra)
    return cfg


def _config_name(c):
    from synth.scenes import CONFIG_NAMES
    return CONFIG_NAMES[c]


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


def timed_graph(fn, k, warmup):
    """ms per call of fn() captured in a CUDA graph: warm-up replays, then k replays bracketed
    by CUDA events on the launching stream."""
    import torch
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        fn()
    for _ in range(warmup):
        g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(k):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    del g
    return e0.elapsed_time(e1) / k


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
    props = torch.cuda.get_device_properties(dev)
    sm_count = int(props.multi_processor_count)

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
        t0 = time.perf_counter()
        (tile, bd, bdb), res = autotune(params_t, n, sc.sh_degree, W, H, cams, tgt_rgb, tgt_d, log=log)
        tuned = {"choice": [tile, bd, bdb], "seconds": round(time.perf_counter() - t0, 2),
                 "candidates_ms": {"x".join(map(str, c)): round(ms, 3) for c, ms in res.items()}}

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
        uuid = "GPU-" + str(props.uuid)
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
    # preprocess, count, scan x2 (with the work order), scatter, sort x3, fwd, loss reduce, raster bwd,
    # preprocess bwd, adam, step counter (the launch list of the captured iteration shows these 14 kernels
    # per step)
    launches_per_step = 14
    gpu_launches = args.steps * launches_per_step
    clocks = clk.summary()
    k_forms = max(MIN_FORM_STEPS, args.steps)

    # --- plain per-view form (same math, one view at a time), and the paper's sequential loop
    #     (Adam after every view), both graph-captured
    per_view = paper_loop = None
    if not args.no_per_view:
        pv = MappingWindow(params_t.clone(), n, sc.sh_degree, W, H, V, tile=tile, batch_depth=bd,
                           batch_depth_bwd=bdb, capacity=win.capacity)
        pv.set_window(cams, tgt_rgb, tgt_d)
        pv_ms = timed_graph(pv.step_per_view, k_forms, args.warmup)
        per_view = {"value": 1e3 / pv_ms, "unit": UNIT, "ms_per_step": pv_ms, "steps": k_forms,
                    "speedup_batched_vs_per_view": (value / world) / (1e3 / pv_ms)}
        pl_ms = timed_graph(lambda: pv.step_per_view(adam_every_view=True), k_forms, args.warmup)
        paper_loop = {"value": V * 1e3 / pl_ms, "unit": "view_iter/s", "ms_per_view_iteration": pl_ms / V,
                      "steps": k_forms, "what": f"{V} single-view iterations (fwd+bwd+Adam each), as the "
                                               "paper's mapping loop takes one keyframe per iteration"}
        if win.read_status()[0] != 0 or pv.read_status()[0] != 0:
            raise SystemExit(f"device status (per-view forms): {pv.read_status()}")
        del pv
        torch.cuda.empty_cache()

    # --- head to head: the paper's splat-wise backward (Fig. 4a) in the same iteration
    splat = None
    if not args.no_splat and tile in (8, 16):
        splat = splat_head_to_head(MappingWindow, params_t, sc, tile, bd, cams, tgt_rgb, tgt_d, win.capacity,
                                   k_forms, args.warmup, value / world)

    # --- the same iteration with the SSIM term of Eq. 9 in the loss
    ssim = None
    if not args.no_ssim:
        ssim = ssim_variant(MappingWindow, params_t, sc, tile, (bd, bdb), cams, tgt_rgb, tgt_d, win.capacity,
                            k_forms, args.warmup, args.lambda_ssim)

    # --- stage breakdown (eager, CUDA events on the launching stream)
    stages = work = None
    if not args.no_stages:
        stages, work = stage_breakdown(win, N, reps=10)

    # --- end to end through the public API: inputs from pinned host memory every step,
    #     the per-view losses read back; keyframe weights from the adaptive scheduler
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(win, sc, cams, tgt_rgb, tgt_d, args, torch, N, k_forms)
        if world > 1:
            e2e["value"] = job_throughput(world, e2e["steps"], max_over_ranks(e2e["seconds"], world, dev))

    roof = iteration = stage_roof = None
    if stages:
        work["workload"] = workload_config(sc)["workload"]
        peaks = Peaks(sm_count, clocks)
        stage_roof = stage_rooflines(stages, work, peaks)
        roof = roofline(stages, work, peaks, stage_roof)
        iteration = iteration_roofline(stages, work, peaks, ms_max / args.steps)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc)

    if rank == 0:
        extra = {"autotune": tuned} if tuned else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded scene)",
            "config": arm_config(sc, tile, bd, bdb, args.config, extra),
            "tile_instances": ninst,
            "view_iters_per_s": value * V,
            "per_view_form": per_view,
            "paper_loop_form": paper_loop,
            "splat_backward": splat,
            "ssim_loss_form": ssim,
            "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "steps")}
            if e2e else None,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "stages_ms": stages,
            "stage_roofline": stage_roof,
            "iteration_roofline": iteration,
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
    reps = MIN_FORM_STEPS
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
                         win.slot_grad, win.status, work=win.work)
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


class Peaks:
    """Roofline denominators: HBM = the measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs,
    else the 6.8 TB/s fallback); FP32 ALU = SMs (read from the device) x 128 FP32 lanes x the
    maximum SM clock (nvidia-smi clocks.max.sm sampled during the timed region, else
    MEASURED_PEAKS.json, else 2070 MHz)."""

    def __init__(self, sm_count, clocks):
        mp = ROOT / "MEASURED_PEAKS.json"
        measured = json.loads(mp.read_text()) if mp.exists() else {}
        self.hbm_gbs = float(measured.get("hbm_gbs") or 6800.0)
        self.hbm_source = "MEASURED_PEAKS.json hbm_gbs (of measured)" if measured.get("hbm_gbs") else \
            "fallback 6.8 TB/s (of fallback)"
        self.sm_count = int(sm_count)
        mhz, src = (clocks or {}).get("sm_max_mhz"), "nvidia-smi clocks.max.sm"
        if not mhz:
            mhz, src = measured.get("sm_max_mhz"), "MEASURED_PEAKS.json sm_max_mhz"
        if not mhz:
            mhz, src = 2070.0, "nominal 2070 MHz"
        self.sm_max_mhz = float(mhz)
        self.alu_tops = self.sm_count * FP32_LANES_PER_SM * self.sm_max_mhz * 1e6 / 1e12
        self.alu_source = (f"{self.sm_count} SMs (device) x {FP32_LANES_PER_SM} FP32 lanes x "
                           f"{self.sm_max_mhz:.0f} MHz ({src}), derived")


RASTER_STAGES = ("render_fwd", "raster_bwd")


def hbm_bytes(stage, w):
    """Algorithmic HBM bytes per launch of a stage: each input read once, each output written
    once (P parameters, S slots, M visible slots, I tile instances, X pixels, T tiles)."""
    P, S, M, I, X, T = w["params"], w["slots"], w["visible_slots"], w["instances"], w["pixels"], w["tiles"]
    if stage == "preprocess":
        return 4 * P + 4 * S + (48 + 48) * M          # params; radius of every slot; record + zeroed grad
    if stage == "bin_sort":
        return 4 * S + 12 * M + 8 * I + 8 * I + 4 * I + 8 * T   # scan rects, scatter keys, sort, vals, ranges
    if stage == "render_fwd":
        return 4 * I + 8 * T + 48 * M + 16 * X + 24 * X         # lists, ranges, records; targets; img/depth/T/last
    if stage == "raster_bwd":
        return 4 * I + 8 * T + 48 * M + 40 * X + 48 * M        # lists, records; fwd outputs + targets; slot grads
    if stage == "preprocess_bwd":
        return 4 * P + 4 * S + 48 * M + 4 * P + 24 * w["n"]   # params, radii, slot grads, grads, stats
    if stage == "adam":
        return 28 * P
    return None


def raster_ops(stage, w):
    if stage == "render_fwd":
        return FWD_OPS_EVAL * w["pairs_fwd_eval"] + FWD_OPS_BLEND * w["pairs_blend"]
    return BWD_OPS_EVAL * w["pairs_bwd_eval"] + BWD_OPS_BLEND * w["pairs_blend"]


def stage_rooflines(stages, work, pk):
    """Each stage against its own roof: the raster kernels against the FP32 ALU peak (formula
    operations/s), the others against the measured HBM copy bandwidth."""
    out = {}
    for st, ms in stages.items():
        t = ms / 1e3
        if st in RASTER_STAGES:
            ops = raster_ops(st, work)
            out[st] = {"bound": "alu", "ms": ms, "work": ops, "achieved": ops / t / 1e12, "peak": pk.alu_tops,
                       "unit": "Top/s", "frac": ops / t / 1e12 / pk.alu_tops,
                       "hbm_frac": hbm_bytes(st, work) / t / 1e9 / pk.hbm_gbs}
        else:
            b = hbm_bytes(st, work)
            out[st] = {"bound": "hbm", "ms": ms, "work": b, "achieved": b / t / 1e9, "peak": pk.hbm_gbs,
                       "unit": "GB/s", "frac": b / t / 1e9 / pk.hbm_gbs}
    return out


def iteration_roofline(stages, work, pk, ms_iter):
    """The whole iteration: its algorithmic HBM bytes over (iteration time x measured copy
    bandwidth), and the combined bound (each stage at the faster of its two roofs) over the
    iteration time."""
    total_bytes = sum(hbm_bytes(st, work) for st in stages)
    bound_s = 0.0
    for st in stages:
        t_hbm = hbm_bytes(st, work) / (pk.hbm_gbs * 1e9)
        t_alu = raster_ops(st, work) / (pk.alu_tops * 1e12) if st in RASTER_STAGES else 0.0
        bound_s += max(t_hbm, t_alu)
    return {"hbm_bytes": total_bytes, "hbm_frac": total_bytes / (ms_iter / 1e3) / (pk.hbm_gbs * 1e9),
            "hbm_peak_gbs": pk.hbm_gbs, "hbm_peak_source": pk.hbm_source,
            "combined_bound_ms": 1e3 * bound_s, "combined_frac": 1e3 * bound_s / ms_iter,
            "ms_per_iteration": ms_iter}


RASTER_BWD_SOURCES = ("render_bwd.cu", "raster.cuh", "cgs_internal.cuh")


def raster_bwd_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in RASTER_BWD_SOURCES:
        h.update((ROOT / "paper_2410_00486_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()


def recorded_traffic(workload):
    """DRAM bytes per launch of k_render_bwd from the committed ncu capture (ncu_traffic.json),
    if it was taken on this workload and the kernel's sources are unchanged since (else None)."""
    if not TRAFFIC_FILE.exists():
        return None
    rec = json.loads(TRAFFIC_FILE.read_text()).get("k_render_bwd")
    if not rec or rec.get("source_sha256") != raster_bwd_source_hash() or rec.get("workload") != workload:
        return None
    return float(rec["traffic_bytes_per_launch"])


def roofline(stages, work, pk, stage_roof):
    """Roofline of the dominant kernel (the stage with the largest time)."""
    dom = max(stages, key=stages.get)
    r = stage_roof[dom]
    out = {"kernel": {"raster_bwd": "k_render_bwd", "render_fwd": "k_render_fwd"}.get(dom, dom),
           "bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"], "unit": r["unit"], "frac": r["frac"],
           "traffic": recorded_traffic(work.get("workload")) if dom == "raster_bwd" else None}
    if r["bound"] == "alu":
        out["peak_source"] = pk.alu_source
        out["work"] = {k: work[k] for k in ("pairs_fwd_eval", "pairs_bwd_eval", "pairs_blend")}
        out["ops_per_pair"] = {"fwd_eval": FWD_OPS_EVAL, "fwd_blend": FWD_OPS_BLEND, "bwd_eval": BWD_OPS_EVAL,
                               "bwd_blend": BWD_OPS_BLEND}
    else:
        out["peak_source"] = pk.hbm_source
    return out


def end_to_end(win, sc, cams, tgt_rgb, tgt_d, args, torch, N, steps):
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
    for _ in range(steps):
        one_step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    h2d = h_cams.numel() * 4 + h_rgb.numel() * 4 + h_d.numel() * 4 + h_w.numel() * 4
    return {"value": steps / sec, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": V * 4,
            "seconds": sec, "steps": steps}


if __name__ == "__main__":
    main()
