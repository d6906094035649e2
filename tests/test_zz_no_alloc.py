"""cgs_render_fwd_noalloc: the forward render for callers that cannot allocate device
memory (or pass a workspace) -- e.g. a real-time mapping loop that must not allocate
once running.  Its scratch lives inside the library; its results must equal those of
cgs_render_fwd with a caller workspace, call after call.  Collected last on purpose."""
import numpy as np
import pytest

from synth import make_scene
from tests.gpu_util import PIX_TOL, native, torch_cuda

pytestmark = pytest.mark.gpu


def _setup(N, torch, sc, seed):
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    cfg = N.make_config(W, H, sc.tile, 64, sc.sh_degree, 0.2, (0.1, 0.2, 0.3), 0.1)
    params = torch.from_numpy(sc.params).cuda()
    cams = torch.from_numpy(np.ascontiguousarray(sc.cams)).cuda()
    rec = torch.zeros(V * n * 12, device="cuda")
    N.cgs_preprocess(params, n, cams, V, cfg, rec, None)
    cap = 1 << 23
    Tv = N.cgs_tiles_per_view(cfg)
    ws = torch.empty(N.cgs_bin_sort_workspace(cap, n, V, cfg), dtype=torch.uint8, device="cuda")
    vals = torch.zeros(cap, dtype=torch.int32, device="cuda")
    ranges = torch.zeros(2 * Tv * V, dtype=torch.int32, device="cuda")
    order = torch.zeros(Tv * V, dtype=torch.int32, device="cuda")
    ninst = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    N.cgs_bin_sort(rec, n, V, cfg, ws, cap, vals, ranges, order, ninst, status)
    rng = np.random.default_rng(seed)
    tgt_rgb = torch.from_numpy(rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)).cuda()
    tgt_d = torch.from_numpy(rng.uniform(0, 5, (V, H, W)).astype(np.float32)).cuda()
    tgt_d[:, : H // 8] = 0.0
    weight = torch.from_numpy(np.linspace(0.5, 2.0, V).astype(np.float32)).cuda()
    return cfg, rec, vals, ranges, order, tgt_rgb, tgt_d, weight, status


def _outputs(torch, V, H, W):
    return dict(img=torch.zeros(V, 3, H, W, device="cuda"), depth=torch.zeros(V, H, W, device="cuda"),
                T=torch.zeros(V, H, W, device="cuda"),
                last=torch.zeros(V, H, W, dtype=torch.int32, device="cuda"),
                loss=torch.zeros(V, device="cuda"), dcount=torch.zeros(V, dtype=torch.int32, device="cuda"))


def test_noalloc_forward_matches_workspace_forward_twice():
    torch = torch_cuda()
    N = native()
    # two different windows, one after the other: the second call must not see the first's
    # scratch contents
    for k, sc in enumerate([make_scene(4, n=20000, views=3), make_scene(1)]):
        V, H, W = sc.views, sc.height, sc.width
        cfg, rec, vals, ranges, order, tr, td, w, status = _setup(N, torch, sc, k)
        ref, got = _outputs(torch, V, H, W), _outputs(torch, V, H, W)
        ws = torch.empty(N.cgs_render_fwd_workspace(V, cfg), dtype=torch.uint8, device="cuda")
        N.cgs_render_fwd(rec, vals, ranges, order, V, cfg, w, tr, td, ref["img"], ref["depth"], ref["T"],
                         ref["last"], ref["loss"], ref["dcount"], ws, status)
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        N.cgs_render_fwd_noalloc(rec, vals, ranges, order, V, cfg, w, tr, td, got["img"], got["depth"],
                                 got["T"], got["last"], got["loss"], got["dcount"], status)
        torch.cuda.synchronize()
        if k > 0:   # after the first call's one-time set-up, a call allocates no device memory
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        assert int(status.item()) == 0
        for key in ("img", "depth", "T"):
            assert (got[key] - ref[key]).abs().max().item() <= PIX_TOL, key
        assert torch.equal(got["last"], ref["last"])
        assert torch.equal(got["dcount"], ref["dcount"])
        torch.testing.assert_close(got["loss"], ref["loss"], rtol=2e-5, atol=0)
        assert ref["loss"].min().item() > 0


def test_noalloc_forward_refuses_windows_above_its_limit():
    torch = torch_cuda()
    N = native()
    # 48 views of 1200x680 at 8x8 tiles = 48 * 12750 tiles > 65536: refused before launch
    cfg = N.make_config(1200, 680, 8, 64, 0)
    V = 48
    t = torch.zeros(16, device="cuda")
    ti = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(N.CgsError) as e:
        N.cgs_render_fwd_noalloc(t, ti, ti, None, V, cfg, None, None, None, t, t, t, ti, None, None)
    assert e.value.status == N.CGS_ERR_WORKSPACE
