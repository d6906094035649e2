"""Autotuner for the raster launch shape: tile edge B (8/16/32) and batch depth (splats
staged per shared-memory batch).  Each candidate runs the whole captured window
iteration on the caller's scene; the fastest (CUDA-event time) wins.  Results are
cached per workload shape in memory and, when `cache_path` is given, in a JSON file.
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
    """Return ((tile, batch_depth), {candidate: ms}) for this workload."""
    views = int(cams.shape[0])
    key = shape_key(n, sh_degree, width, height, views)
    if cache_path and Path(cache_path).exists():
        disk = json.loads(Path(cache_path).read_text())
        if key in disk:
            return tuple(disk[key]["best"]), {tuple(map(int, k.split("x"))): v for k, v in disk[key]["ms"].items()}
    if key in _memo:
        return _memo[key]
    results = {}
    for tile, bd in candidates:
        win = MappingWindow(params.clone(), n, sh_degree, width, height, views, tile=tile, batch_depth=bd, **kw)
        win.set_window(cams, tgt_rgb, tgt_depth)
        win.fit_capacity(1.3)
        results[(tile, bd)] = time_window(win, reps)
        if log:
            log(f"autotune tile={tile} batch_depth={bd}: {results[(tile, bd)]:.3f} ms")
        del win
        torch.cuda.empty_cache()
    best = min(results, key=results.get)
    _memo[key] = (best, results)
    if cache_path:
        p = Path(cache_path)
        disk = json.loads(p.read_text()) if p.exists() else {}
        disk[key] = {"best": list(best), "ms": {f"{t}x{b}": v for (t, b), v in results.items()}}
        p.write_text(json.dumps(disk, indent=1))
    return best, results
