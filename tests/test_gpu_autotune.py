"""The launch-shape autotuner: for each tile size it returns a valid (tile, batch depth,
backward batch depth) that is the fastest of what it measured, the choice runs the window
iteration with the same results as any other shape, and the on-disk cache round-trips."""
import numpy as np
import pytest

from synth import make_scene
from tests.gpu_util import native, torch_cuda

pytestmark = pytest.mark.gpu

DEPTHS = (32, 64, 128, 256)


def small_window(torch):
    sc = make_scene(4, n=20000, views=3)
    params = torch.from_numpy(sc.params).cuda()
    cams = torch.from_numpy(np.ascontiguousarray(sc.cams)).cuda()
    rng = np.random.default_rng(0)
    tgt = torch.from_numpy(rng.uniform(0, 1, (sc.views, 3, sc.height, sc.width)).astype(np.float32)).cuda()
    tgd = torch.from_numpy(rng.uniform(0.5, 5, (sc.views, sc.height, sc.width)).astype(np.float32)).cuda()
    return sc, params, cams, tgt, tgd


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_autotune_returns_a_valid_fastest_shape_per_tile(tile, tmp_path):
    torch = torch_cuda()
    native()
    from paper_2410_00486_gb300 import autotune as A
    sc, params, cams, tgt, tgd = small_window(torch)
    A._memo.clear()
    cache = tmp_path / "tune.json"
    best, res = A.autotune(params, sc.n, 3, sc.width, sc.height, cams, tgt, tgd,
                           candidates=[(tile, d) for d in DEPTHS], reps=2, cache_path=cache)
    t, bd, bdb = best
    assert t == tile and bd in DEPTHS and bdb in DEPTHS
    assert res[best] == min(res.values()) and all(ms > 0 for ms in res.values())
    # the cache round-trips: a fresh process state reads the same choice without measuring
    A._memo.clear()
    calls = []
    best2, res2 = A.autotune(params, sc.n, 3, sc.width, sc.height, cams, tgt, tgd,
                             candidates=[(tile, d) for d in DEPTHS], reps=2, cache_path=cache, log=calls.append)
    assert tuple(best2) == tuple(best) and not calls
    assert {tuple(k): v for k, v in res2.items()} == {tuple(k): v for k, v in res.items()}


def test_autotuned_shape_gives_the_same_iteration():
    torch = torch_cuda()
    native()
    from paper_2410_00486_gb300 import autotune as A
    from paper_2410_00486_gb300.window import MappingWindow
    sc, params, cams, tgt, tgd = small_window(torch)
    A._memo.clear()
    best, _ = A.autotune(params, sc.n, 3, sc.width, sc.height, cams, tgt, tgd, reps=2)
    wins = []
    for t, bd, bdb in (best, (16, 64, 64)):
        w = MappingWindow(params.clone(), sc.n, 3, sc.width, sc.height, sc.views, tile=t, batch_depth=bd,
                          batch_depth_bwd=bdb)
        w.set_window(cams, tgt, tgd)
        w.fit_capacity()
        w.forward()
        w.backward()
        torch.cuda.synchronize()
        assert w.read_status()[0] == 0
        wins.append(w)
    a, b = wins
    assert (a.img - b.img).abs().max().item() < 1e-5
    torch.testing.assert_close(a.loss_view, b.loss_view, rtol=1e-5, atol=0)
    rel = ((a.grads - b.grads).norm() / b.grads.norm()).item()
    assert rel < 1e-4
