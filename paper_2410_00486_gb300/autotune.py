"""Autotuner for the raster launch shape: tile edge B (8/16/32) and the batch depths
(splats staged per shared-memory batch) of the forward and of the backward.  Each
candidate runs the whole captured window iteration on the caller's scene; the fastest
(CUDA-event time) wins.  First every (tile, depth) pair with one depth for both kernels,
then, at the best tile, each kernel's depth on its own (the two kernels are separate
launches, so their best depths are independent).  Results are cached per workload shape
in memory and, when `cache_path` is given, in a JSON file.
"""
from __future__ import annotations

import json
from pathlib import Path

import torch

from .window import MappingWindow

CANDIDATES = [(t, bd) for t in (8, 16, 32) for bd in (32, 64, 128, 256)]
_memo: dict = {}


def shape_key(n, sh_degree, width, height, views) -> str:
    return f"n{n}_sh{sh_degree}_{width}x{height}_v{views}"


def time_window(win: MappingWindow, reps: int = 5, warmup: int = 2) -> float:
    """Average ms per captured window iteration."""
    win.capture()
    for _ in range(warmup):
        win.replay()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        win.replay()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def autotune(params: torch.Tensor, n: int, sh_degree: int, width: int, height: int, cams, tgt_rgb, tgt_depth,
             candidates=CANDIDATES, reps: int = 5, cache_path: str | Path | None = None, log=None, **kw):
    """Return ((tile, batch_depth, batch_depth_bwd), {candidate: ms}) for this workload."""
    views = int(cams.shape[0])
    key = shape_key(n, sh_degree, width, height, views)
    if cache_path and Path(cache_path).exists():
        disk = json.loads(Path(cache_path).read_text())
        if key in disk:
            return tuple(disk[key]["best"]), {tuple(map(int, k.split("x"))): v for k, v in disk[key]["ms"].items()}
    if key in _memo:
        return _memo[key]
    results = {}

    def measure(tile, bd, bdb):
        if (tile, bd, bdb) in results:
            return
        win = MappingWindow(params.clone(), n, sh_degree, width, height, views, tile=tile, batch_depth=bd,
                            batch_depth_bwd=bdb, **kw)
        win.set_window(cams, tgt_rgb, tgt_depth)
        win.fit_capacity(1.3)
        results[(tile, bd, bdb)] = time_window(win, reps)
        st = win.read_status()[0]
        if st != 0:                        # a candidate that fails is an error, not a slow one
            raise RuntimeError(f"autotune candidate tile={tile} batch_depth={bd}/{bdb}: device status {st}")
        if log:
            log(f"autotune tile={tile} batch_depth={bd} batch_depth_bwd={bdb}: {results[(tile, bd, bdb)]:.3f} ms")
        del win
        torch.cuda.empty_cache()

    for tile, bd in candidates:
        measure(tile, bd, bd)
    tile, bd, bdb = min(results, key=results.get)
    depths = sorted({b for _, b in candidates})
    for d in depths:                       # forward depth, backward depth held
        measure(tile, d, bdb)
    bd = min((d for d in depths), key=lambda d: results[(tile, d, bdb)])
    for d in depths:                       # backward depth, forward depth held
        measure(tile, bd, d)
    best = min(results, key=results.get)
    _memo[key] = (best, results)
    if cache_path:
        p = Path(cache_path)
        disk = json.loads(p.read_text()) if p.exists() else {}
        disk[key] = {"best": list(best), "ms": {"x".join(map(str, c)): v for c, v in results.items()}}
        p.write_text(json.dumps(disk, indent=1))
    return best, results
