"""Parity at the benchmark's workload size and launch configuration: 16 views of 1200x680,
300k Gaussians, SH degree 3, tile 16, staged batch depths 128 (forward) and 64 (backward),
all views in one launch per stage.  The oracle checks outputs it can compute one by one:
sampled Gaussians of the projection; two whole views of tile lists (rect lists bit-exact
with the oracle's, the culled lists checked against them by float64 brute force); the whole
window rendered from rect and from culled lists (bit-identical); sampled pixels of the
forward; sampled tiles of the raster backward and of the raster + preprocess backward
(the full-size launches with the other tiles' lists emptied; the oracle computes its own
slot gradients from its rect lists); and sampled Gaussians of the preprocess backward."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import make_scene
from synth.scenes import param_layout
from tests.gpu_util import (PIX_TOL, check_culled_lists, field_grad_check, gaussians_of_slots, grad_check,
                            last_slots, native, param_grad_check, rec_from_gpu, round32, sg_from_gpu, torch_cuda)

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


def view_records(view):
    """The GPU's float32 records of one view [n, 12] (slot ids local to the view)."""
    S = window()
    n = S["sc"].n
    return S["win"].rec.view(-1, 12)[view * n:(view + 1) * n].cpu().numpy()


def oracle_rect_lists(view):
    """The oracle's rect lists of one view, binned from the GPU's float32 records (cached)."""
    S = window()
    key = ("rect", view)
    if key not in S:
        sc = S["sc"]
        rec = view_records(view)
        radius = np.ascontiguousarray(rec[:, 7]).view(np.int32)
        S[key] = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 6], radius, 1, sc.n, sc.width, sc.height, 16)
    return S[key]


def rect_window():
    """The whole window binned with rect lists on the GPU and rendered from them (once)."""
    S = window()
    if "rect_win" in S:
        return S["rect_win"]
    torch = torch_cuda()
    N = native()
    sc, win = S["sc"], S["win"]
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    cfg = N.make_config(W, H, 16, 128, 3, 0.2, (0.0, 0.0, 0.0), 0.1, batch_depth_bwd=64, rect_lists=True)
    cap = sum(len(oracle_rect_lists(vw)[1]) for vw in range(V))     # rect instances of the window
    ws = torch.empty(N.cgs_bin_sort_workspace(cap, n, V, cfg), dtype=torch.uint8, device="cuda")
    vals = torch.zeros(cap, dtype=torch.int32, device="cuda")
    ranges = torch.zeros(2 * win.Ttot, dtype=torch.int32, device="cuda")
    order = torch.zeros(win.Ttot, dtype=torch.int32, device="cuda")
    ninst = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    N.cgs_bin_sort(win.rec, n, V, cfg, ws, cap, vals, ranges, order, ninst, status)
    del ws
    out = dict(vals=vals, ranges=ranges, order=order, ninst=int(ninst.item()), cap=cap)
    out["img"], out["depth"], out["T"] = torch.zeros_like(win.img), torch.zeros_like(win.depth), \
        torch.zeros_like(win.t_final)
    out["last"], out["loss"], out["dc"] = torch.zeros_like(win.last), torch.zeros_like(win.loss_view), \
        torch.zeros_like(win.depth_count)
    fws = torch.empty(N.cgs_render_fwd_workspace(V, cfg), dtype=torch.uint8, device="cuda")
    N.cgs_render_fwd(win.rec, vals, ranges, order, V, cfg, win.view_weight, win.tgt_rgb, win.tgt_depth, out["img"],
                     out["depth"], out["T"], out["last"], out["loss"], out["dc"], fws, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and out["ninst"] == cap
    S["rect_win"] = out
    return out


@pytest.mark.parametrize("view", [0, 11])
def test_fullsize_tile_lists_of_whole_views(view):
    """Rect lists of a whole view bit-exact with the oracle's; the window's culled lists of
    that view are ordered subsequences of them whose every dropped pair has alpha < 1/255 at
    each pixel centre of its tile (float64 brute force over all dropped pairs)."""
    S = window()
    sc, win = S["sc"], S["win"]
    n, W, H, Tv = sc.n, sc.width, sc.height, win.Tv
    ranges_o, vals_o = oracle_rect_lists(view)
    rw = rect_window()
    rg = rw["ranges"].view(-1, 2)[view * Tv:(view + 1) * Tv].cpu().numpy().view(np.uint32).astype(np.int64)
    base = rg[0, 0]
    assert np.array_equal(rg - base, ranges_o)
    vals = rw["vals"][base: base + len(vals_o)].cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(vals - view * n, vals_o)
    cg = win.ranges.view(-1, 2)[view * Tv:(view + 1) * Tv].cpu().numpy().view(np.uint32).astype(np.int64)
    cv = win.vals[cg[0, 0]: cg[-1, 1]].cpu().numpy().view(np.uint32).astype(np.int64)
    tot, kept, dropped = check_culled_lists(view_records(view), ranges_o, vals_o, cg, cv, W, H, 16,
                                            slot_base=view * n)
    assert dropped > 0.3 * tot
    print(f"[fullsize lists view {view}] rect {tot} kept {kept} dropped {dropped}")


def test_fullsize_rect_and_culled_renders_identical():
    """The whole window's forward from the rect lists and from the culled lists: images, depth,
    transmittance and per-view losses bit-identical; each pixel's last blended splat the same."""
    torch = torch_cuda()
    S = window()
    sc, win = S["sc"], S["win"]
    rw = rect_window()
    for k, w in (("img", win.img), ("depth", win.depth), ("T", win.t_final), ("loss", win.loss_view),
                 ("dc", win.depth_count)):
        assert torch.equal(rw[k], w), k
    la = last_slots(win.last.cpu().numpy(), win.ranges.cpu().numpy(), win.vals[:S["ninst"]].cpu().numpy(),
                    sc.width, sc.height, 16)
    lb = last_slots(rw["last"].cpu().numpy(), rw["ranges"].cpu().numpy(), rw["vals"][:rw["ninst"]].cpu().numpy(),
                    sc.width, sc.height, 16)
    assert np.array_equal(la, lb)
    print(f"[fullsize rect vs culled] instances rect {rw['ninst']} culled {S['ninst']}")


def test_fullsize_forward_sampled_pixels():
    """4000 pixels of four views blended by the oracle from its rect lists (float64) against
    the window's forward from its culled lists."""
    S = window()
    sc, win = S["sc"], S["win"]
    n, W, H = sc.n, sc.width, sc.height
    rng = np.random.default_rng(1)
    img, dep, tf = win.img.cpu().numpy(), win.depth.cpu().numpy(), win.t_final.cpu().numpy()
    last_g = last_slots(win.last.cpu().numpy(), win.ranges.cpu().numpy(), win.vals[:S["ninst"]].cpu().numpy(),
                        W, H, 16)
    flagged = 0
    for view in (0, 5, 11, 15):
        k = 1000
        pix = np.stack([np.zeros(k, int), rng.integers(0, W, k), rng.integers(0, H, k)], 1).astype(np.int32)
        ranges_o, vals_o = oracle_rect_lists(view)
        rec10, _, _ = rec_from_gpu(win.rec.view(-1, 12)[view * n:(view + 1) * n].reshape(-1))
        ref = O.render_pixels(rec10, ranges_o, vals_o, W, H, 16, pix, tol=1e-5)
        xx, yy = pix[:, 1], pix[:, 2]
        ok = ref["near"] == 0
        flagged += int((~ok).sum())
        err = np.abs(img[view][:, yy, xx].T - ref["img"]).max(1)
        assert err[ok].max() < PIX_TOL
        assert np.abs(tf[view, yy, xx] - ref["T"])[ok].max() < PIX_TOL
        dscale = max(1.0, np.abs(ref["depth"]).max())
        assert (np.abs(dep[view, yy, xx] - ref["depth"])[ok] / dscale).max() < PIX_TOL
        lo = ref["last"].astype(np.int64)
        tl = (yy // 16) * ((W + 15) // 16) + xx // 16
        slot_o = np.where(lo > 0, vals_o.astype(np.int64)[np.clip(ranges_o[tl, 0].astype(np.int64) + lo - 1, 0,
                                                                  len(vals_o) - 1)] + view * n, -1)
        assert np.array_equal(last_g[view, yy, xx][ok], slot_o[ok])
    assert flagged < 0.01 * 4000
    print(f"[fullsize fwd pixels] flagged {flagged} of 4000")


def sampled_tile_lists(S, per_view=16, views=(0, 5, 11, 15), seed=2):
    """Busy tiles sampled from some views: the window's culled ranges with every other tile
    emptied (device tensor), and the oracle's rect lists of the same tiles in the window's
    global slot and tile numbering, plus the oracle's near-threshold flags of their pixels."""
    torch = torch_cuda()
    sc, win = S["sc"], S["win"]
    n, W, H, Tv = sc.n, sc.width, sc.height, win.Tv
    Tx = (W + 15) // 16
    rg = win.ranges.view(-1, 2).clone()
    lens = (rg[:, 1] - rg[:, 0]).cpu().numpy()
    rng = np.random.default_rng(seed)
    pick = []
    for v in views:
        busy = np.nonzero(lens[v * Tv:(v + 1) * Tv] > 0)[0]
        pick += list(v * Tv + rng.choice(busy, per_view, replace=False))
    pick = np.sort(np.asarray(pick))
    keep = torch.zeros(rg.shape[0], dtype=torch.bool, device="cuda")
    keep[torch.from_numpy(pick).cuda()] = True
    rg[:, 1] = torch.where(keep, rg[:, 1], rg[:, 0])
    # the oracle's rect lists of the picked tiles
    o_ranges = np.zeros((win.Ttot, 2), np.uint32)
    o_vals, pos = [], 0
    pix = []
    pick_set = set(pick.tolist())
    for t in range(win.Ttot):
        o_ranges[t] = pos
        if t in pick_set:
            v, tl = divmod(int(t), Tv)
            rr, vv = oracle_rect_lists(v)
            lst = vv[rr[tl, 0]:rr[tl, 1]].astype(np.int64) + v * n
            o_vals.append(lst)
            pos += len(lst)
            o_ranges[t, 1] = pos
            tx, ty = tl % Tx, tl // Tx
            ys, xs = np.mgrid[ty * 16:min(ty * 16 + 16, H), tx * 16:min(tx * 16 + 16, W)]
            pix.append(np.stack([np.full(xs.size, v), xs.ravel(), ys.ravel()], 1))
    o_vals = np.concatenate(o_vals).astype(np.uint32)
    pix = np.concatenate(pix).astype(np.int32)
    rec10, _, _ = rec_from_gpu(win.rec)
    px = O.render_pixels(rec10, o_ranges, o_vals, W, H, 16, pix, tol=1e-5)
    tr = win.tgt_rgb.cpu().numpy()[pix[:, 0], :, pix[:, 2], pix[:, 1]]
    resid = (np.abs(px["img"] - tr) < 1e-5).any(axis=1)     # the L1 residual's sign, near 0
    fl = pix[(px["near"] != 0) | resid]
    near_tiles = np.unique(fl[:, 0] * Tv + (fl[:, 2] // 16) * Tx + fl[:, 1] // 16)
    near = np.zeros(sc.views * n, bool)
    for t in near_tiles:
        near[o_vals[o_ranges[t, 0]:o_ranges[t, 1]].astype(np.int64)] = True
    return rg, o_ranges, o_vals, rec10, near


def test_fullsize_raster_backward_sampled_tiles():
    """The raster backward launched on the whole window with every tile's list emptied but 64
    sampled ones (16 in each of four views): its slot gradients are those tiles' pixels'
    contributions, which the oracle computes from its rect lists of the same tiles."""
    torch = torch_cuda()
    N = native()
    S = window()
    sc, win = S["sc"], S["win"]
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    rg, o_ranges, o_vals, rec10, near = sampled_tile_lists(S)
    sg = torch.zeros_like(win.slot_grad)
    N.cgs_raster_bwd(win.rec, win.vals, rg.reshape(-1), win.order, V, win.cfg, win.view_weight, win.img, win.depth,
                     win.t_final, win.last, win.tgt_rgb, win.tgt_depth, win.depth_count, None, None, sg)
    torch.cuda.synchronize()
    g = sg_from_gpu(sg)
    ref, mag = O.render_bwd(rec10, o_ranges, o_vals, V, n, W, H, 16, sc.cams, win.img.cpu().numpy(),
                            win.depth.cpu().numpy(), win.tgt_rgb.cpu().numpy(), win.tgt_depth.cpu().numpy(),
                            win.depth_count.cpu().numpy().astype(np.int64), with_abs=True)
    touched = np.abs(ref).sum(1) > 0
    assert touched.sum() > 2000
    print(f"[fullsize bwd] touched slots {touched.sum()}, in tiles with a flagged pixel {near.sum()}")
    field_grad_check(g[touched], ref[touched], near[touched], "fullsize bwd", mag=mag[touched])
    assert np.all(g[~touched] == 0)
    S["sampled"] = (rg, o_ranges, o_vals, rec10, near, ref)


def test_fullsize_end_to_end_gradient_sampled_tiles():
    """Raster backward then preprocess backward on the GPU over the 64 sampled tiles; the
    oracle takes its own slot gradients of those tiles (from its rect lists) through its own
    float64 chain rule from the parameters.  Parameter gradients of every Gaussian they touch."""
    torch = torch_cuda()
    N = native()
    S = window()
    sc, win = S["sc"], S["win"]
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    if "sampled" not in S:
        test_fullsize_raster_backward_sampled_tiles()
    rg, o_ranges, o_vals, rec10, near, ref_sg = S["sampled"]
    sg = torch.zeros_like(win.slot_grad)
    N.cgs_raster_bwd(win.rec, win.vals, rg.reshape(-1), win.order, V, win.cfg, win.view_weight, win.img, win.depth,
                     win.t_final, win.last, win.tgt_rgb, win.tgt_depth, win.depth_count, None, None, sg)
    grads = torch.zeros_like(win.grads)
    N.cgs_preprocess_bwd(win.params, n, win.cams, V, win.cfg, win.rec, sg, grads, False, None, None, None)
    torch.cuda.synchronize()
    touched_slot = np.abs(ref_sg).sum(1) > 0
    idx = np.nonzero(touched_slot.reshape(V, n).any(0))[0]
    rows = slot_rows(idx, n, V)
    sub = subset_params(sc.params, n, 3, idx)
    pre = O.preprocess(sub, len(idx), 3, sc.cams, W, H, 16)
    ref = O.preprocess_bwd(sub, len(idx), 3, sc.cams, W, H, 16, ref_sg[rows])
    got = subset_params(grads.cpu().numpy().astype(np.float64), n, 3, idx)
    expl = gaussians_of_slots(near[rows] | (pre["fragile"] > 0), len(idx))
    print(f"[fullsize end to end] Gaussians {len(idx)}, near a threshold {expl.sum()}")
    param_grad_check(got, ref, len(idx), 3, expl, "fullsize e2e")


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
        grad_check(gg, rr, None, f"fullsize pre bwd {name}", l2=1e-4)
