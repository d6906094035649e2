"""Parity at the benchmark's workload size and launch configuration: 16 views of 1200x680,
300k Gaussians, SH degree 3, tile 16, staged batch depths 128 (forward) and 64 (backward),
all views in one launch per stage.  The oracle checks outputs it can compute one by one:
sampled Gaussians of the projection, two whole views of tile lists (bit-exact), sampled
pixels of the forward, sampled tiles of the raster backward (the full-size launch with
the other tiles' lists emptied) and sampled Gaussians of the preprocess backward (GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import make_scene
from synth.scenes import param_layout
from tests.gpu_util import GRAD_REL_TOL, PIX_TOL, native, rec_from_gpu, rel_l2, round32, sg_from_gpu, torch_cuda

pytestmark = pytest.mark.gpu

_S = {}


def window():
    """The full-size window after one forward and backward (set up once for the module)."""
    if _S:
        return _S
    torch = torch_cuda()
    native()
    from paper_2410_00486_gb300.window import MappingWindow
    sc = make_scene(5)
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    cams = torch.from_numpy(np.ascontiguousarray(sc.cams)).cuda()
    kw = dict(tile=16, batch_depth=128, batch_depth_bwd=64)
    tw = MappingWindow(torch.from_numpy(sc.params_target).cuda(), n, 3, W, H, V, **kw)
    tw.set_window(cams, torch.zeros(V, 3, H, W), None)
    tw.fit_capacity()
    tw.forward(with_loss=False)
    tgt_rgb, tgt_d = tw.img.clone(), tw.depth.clone()
    del tw
    win = MappingWindow(torch.from_numpy(sc.params).cuda(), n, 3, W, H, V, **kw)
    win.set_window(cams, tgt_rgb, tgt_d)
    win.fit_capacity(1.25)
    win.forward()
    win.backward()
    torch.cuda.synchronize()
    assert win.read_status()[0] == 0
    _S.update(sc=sc, win=win, tgt_rgb=tgt_rgb, tgt_d=tgt_d, ninst=int(win.n_inst.item()))
    return _S


def subset_params(P, n, deg, idx):
    """The parameter vector of Gaussians idx (same group layout, len(idx) Gaussians)."""
    K = (deg + 1) ** 2
    widths = [3, 3, 4, 1, 3, 3 * (K - 1)]
    out, off = [], 0
    for w in widths:
        grp = np.asarray(P[off: off + w * n]).reshape(n, w)
        out.append(grp[idx].ravel())
        off += w * n
    return np.concatenate(out)


def slot_rows(idx, n, V):
    """Slot indices (view-major) of Gaussians idx in every view, in the oracle's order."""
    return (np.arange(V)[:, None] * n + np.asarray(idx)[None, :]).ravel()


def test_fullsize_preprocess_sampled_gaussians():
    S = window()
    sc, win = S["sc"], S["win"]
    V, n = sc.views, sc.n
    idx = np.sort(np.random.default_rng(0).choice(n, 1500, replace=False))
    ref = O.preprocess(subset_params(sc.params, n, 3, idx), len(idx), 3, sc.cams, sc.width, sc.height, 16)
    rows = slot_rows(idx, n, V)
    g10, grad_r, gtau = rec_from_gpu(win.rec.view(-1, 12)[rows].reshape(-1))
    fr = ref["fragile"] > 0
    assert np.array_equal(grad_r[~fr], ref["radius"][~fr])
    both = (grad_r > 0) & (ref["radius"] > 0) & ~fr
    assert both.sum() > 1000
    e = np.abs(g10[both] - ref["rec"][both])
    r = ref["rec"][both]
    assert e[:, 0:2].max() < 2e-3
    assert (e[:, 2:5] / np.abs(r[:, 2:5]).max(1, keepdims=True)).max() < 1e-4
    assert e[:, 6:9].max() < 2e-5
    assert (e[:, 9] / r[:, 9]).max() < 1e-6
    assert np.abs(gtau[both] + np.log(255.0 * ref["rec"][both, 5])).max() < 1e-5


@pytest.mark.parametrize("view", [0, 11])
def test_fullsize_tile_lists_of_whole_views_bit_exact(view):
    S = window()
    sc, win = S["sc"], S["win"]
    n, W, H = sc.n, sc.width, sc.height
    rec = win.rec.view(-1, 12)[view * n:(view + 1) * n].cpu().numpy()
    u, v, z = rec[:, 0], rec[:, 1], rec[:, 6]
    radius = np.ascontiguousarray(rec[:, 7]).view(np.int32)
    # the GPU's own float32 records, conic and tau included: the reach test decides alike
    ranges_o, vals_o = O.bin_lists(u, v, z, radius, 1, n, W, H, 16, conic=rec[:, 2:5], tau=rec[:, 11])
    Tv = win.Tv
    rg = win.ranges.view(-1, 2)[view * Tv:(view + 1) * Tv].cpu().numpy().view(np.uint32).astype(np.int64)
    base = rg[0, 0]
    assert np.array_equal(rg - base, ranges_o)
    vals = win.vals[base: base + len(vals_o)].cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(vals - view * n, vals_o)


def test_fullsize_forward_sampled_pixels():
    S = window()
    sc, win = S["sc"], S["win"]
    V, W, H = sc.views, sc.width, sc.height
    rng = np.random.default_rng(1)
    k = 4000
    pix = np.stack([rng.integers(0, V, k), rng.integers(0, W, k), rng.integers(0, H, k)], 1).astype(np.int32)
    rec10, _, _ = rec_from_gpu(win.rec)
    ninst = S["ninst"]
    ranges = win.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    vals = win.vals[:ninst].cpu().numpy().view(np.uint32)
    ref = O.render_pixels(rec10, ranges, vals, W, H, 16, pix, tol=1e-5)
    vv, xx, yy = pix[:, 0], pix[:, 1], pix[:, 2]
    img = win.img.cpu().numpy()[vv, :, yy, xx]
    ok = ref["near"] == 0
    err = np.abs(img - ref["img"]).max(1)
    assert (1 - ok.mean()) < 2e-3
    assert err[ok].max() < PIX_TOL
    assert np.abs(win.t_final.cpu().numpy()[vv, yy, xx] - ref["T"])[ok].max() < PIX_TOL
    dscale = max(1.0, np.abs(ref["depth"]).max())
    assert (np.abs(win.depth.cpu().numpy()[vv, yy, xx] - ref["depth"])[ok] / dscale).max() < PIX_TOL
    assert np.array_equal(win.last.cpu().numpy().view(np.uint32)[vv, yy, xx][ok], ref["last"][ok])


def test_fullsize_raster_backward_sampled_tiles():
    """The raster backward launched on the whole window with every tile's list emptied but
    24 sampled ones: its slot gradients are those tiles' pixels' contributions, which the
    oracle computes from the same records, lists and forward outputs."""
    torch = torch_cuda()
    N = native()
    S = window()
    sc, win = S["sc"], S["win"]
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    rg = win.ranges.view(-1, 2).clone()
    lens = (rg[:, 1] - rg[:, 0]).cpu().numpy()
    busy = np.nonzero(lens > 0)[0]
    pick = np.random.default_rng(2).choice(busy, 24, replace=False)
    keep = torch.zeros(rg.shape[0], dtype=torch.bool, device="cuda")
    keep[torch.from_numpy(pick).cuda()] = True
    rg[:, 1] = torch.where(keep, rg[:, 1], rg[:, 0])
    sg = torch.zeros_like(win.slot_grad)
    N.cgs_raster_bwd(win.rec, win.vals, rg.reshape(-1), win.order, V, win.cfg, win.view_weight, win.img, win.depth,
                     win.t_final, win.last, win.tgt_rgb, win.tgt_depth, win.depth_count, None, None, sg)
    torch.cuda.synchronize()
    g = sg_from_gpu(sg)
    rec10, _, _ = rec_from_gpu(win.rec)
    ninst = S["ninst"]
    ref = O.render_bwd(rec10, rg.cpu().numpy().view(np.uint32), win.vals[:ninst].cpu().numpy().view(np.uint32),
                       V, n, W, H, 16, sc.cams, win.img.cpu().numpy(), win.depth.cpu().numpy(),
                       win.tgt_rgb.cpu().numpy(), win.tgt_depth.cpu().numpy(),
                       win.depth_count.cpu().numpy().astype(np.int64))
    touched = np.abs(ref).sum(1) > 0
    assert touched.sum() > 1000
    fields = ["u", "v", "A", "B", "C", "o", "r", "g", "b", "z"]
    errs = {f: rel_l2(g[touched, k], ref[touched, k]) for k, f in enumerate(fields)}
    print("[fullsize bwd] " + " ".join(f"{f}:{e:.1e}" for f, e in errs.items()))
    for f, e in errs.items():
        assert e < GRAD_REL_TOL, (f, e)
    assert np.all(g[~touched] == 0)


def test_fullsize_preprocess_backward_sampled_gaussians():
    """The window's parameter gradients of 1000 sampled Gaussians against the oracle's chain
    rule fed with the same (GPU) slot gradients of those Gaussians in all 16 views."""
    S = window()
    sc, win = S["sc"], S["win"]
    V, n = sc.views, sc.n
    idx = np.sort(np.random.default_rng(3).choice(n, 1000, replace=False))
    rows = slot_rows(idx, n, V)
    sg = round32(sg_from_gpu(win.slot_grad.view(-1, 12)[rows].reshape(-1)))
    pre = O.preprocess(subset_params(sc.params, n, 3, idx), len(idx), 3, sc.cams, sc.width, sc.height, 16)
    sg = sg * (pre["fragile"] == 0)[:, None]
    ref = O.preprocess_bwd(subset_params(sc.params, n, 3, idx), len(idx), 3, sc.cams, sc.width, sc.height, 16, sg)
    fr_g = np.zeros(n, bool)
    fr_g[idx[np.nonzero(pre["fragile"].reshape(V, -1).any(0))[0]]] = True
    if fr_g.any():     # Gaussians with a fragile slot: the GPU used that slot's gradient, the check did not
        keep = ~fr_g[idx]
    else:
        keep = np.ones(len(idx), bool)
    got = subset_params(win.grads.cpu().numpy().astype(np.float64), n, 3, idx)
    lay = param_layout(len(idx), 3)
    bounds = [("means", lay["means"], lay["log_scales"], 3), ("log_scales", lay["log_scales"], lay["quats"], 3),
              ("quats", lay["quats"], lay["opacity"], 4), ("opacity", lay["opacity"], lay["sh_dc"], 1),
              ("sh_dc", lay["sh_dc"], lay["sh_rest"], 3), ("sh_rest", lay["sh_rest"], lay["total"], 45)]
    for name, a, b, w in bounds:
        gg = got[a:b].reshape(len(idx), w)[keep]
        rr = ref[a:b].reshape(len(idx), w)[keep]
        e = rel_l2(gg, rr)
        print(f"[fullsize pre bwd] {name}: {e:.1e}")
        assert e < 1e-4, (name, e)
