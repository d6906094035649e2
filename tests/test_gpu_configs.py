"""Whole-image parity at the stated sizes of the single-view Replica-like workload (100k
Gaussians, SH degree 3, one 1200x680 view) and the TUM-like keyframe window (200k Gaussians,
SH degree 3, eight 640x480 views whose visible counts fall from about 150k to about 20k),
in the benchmark's launch configuration (tile 16, staged batch depths 128 / 64, all views in
one launch per stage).  Every stage against the float64 oracle, every pixel and every
gradient element:
  - projection: the oracle's own, from the parameters;
  - tile lists: the window's culled lists against the oracle's rect lists of the same float32
    records (ordered subsequences; every dropped pair below alpha 1/255 at every pixel centre);
  - forward: every pixel blended by the oracle from its rect lists;
  - raster backward: every slot gradient from the oracle's hand-derived backward;
  - preprocess backward: every parameter gradient from the oracle's chain rule applied to the
    oracle's own slot gradients.
Tolerances: pixels 1e-4 (decisions near a threshold excluded and counted), gradients 1e-3
relative L2 and the per-element bound of tests.gpu_util.grad_check."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import make_scene
from tests.gpu_util import (F32_COND, GRAD_REL_TOL, PIX_TOL, check_culled_lists, field_grad_check,
                            gaussians_of_slots, last_slots, native, param_grad_check, rec_from_gpu,
                            residual_sign_flags, sg_from_gpu, slots_in_flagged_tiles, torch_cuda)

pytestmark = pytest.mark.gpu


def gpu_window(sc, torch):
    from paper_2410_00486_gb300.window import MappingWindow
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    cams = torch.from_numpy(np.ascontiguousarray(sc.cams)).cuda()
    kw = dict(tile=16, batch_depth=128, batch_depth_bwd=64)
    tw = MappingWindow(torch.from_numpy(sc.params_target).cuda(), n, sc.sh_degree, W, H, V, **kw)
    tw.set_window(cams, torch.zeros(V, 3, H, W), None)
    tw.fit_capacity()
    tw.forward(with_loss=False)          # targets: the render of the perturbed copy
    tgt_rgb, tgt_d = tw.img.clone(), tw.depth.clone()
    del tw
    win = MappingWindow(torch.from_numpy(sc.params).cuda(), n, sc.sh_degree, W, H, V, **kw)
    win.set_window(cams, tgt_rgb, tgt_d)
    win.fit_capacity()
    win.forward()
    win.backward()
    torch.cuda.synchronize()
    assert win.read_status()[0] == 0
    return win


@pytest.mark.parametrize("config", [2, 4])
def test_config_stages_match_oracle_on_whole_images(config):
    torch = torch_cuda()
    native()
    sc = make_scene(config)
    V, n, W, H = sc.views, sc.n, sc.width, sc.height
    win = gpu_window(sc, torch)
    rec10, radius, _ = rec_from_gpu(win.rec)
    visible = (radius.reshape(V, n) > 0).sum(1)
    print(f"[config {config}] visible per view {visible.tolist()}, culled instances {int(win.n_inst.item())}")
    if config == 4:
        assert visible.min() < 25_000 and visible.max() > 145_000     # uneven: about 20k to 150k

    # projection, from the parameters
    pre = O.preprocess(sc.params, n, sc.sh_degree, sc.cams, W, H, 16)
    fr = pre["fragile"] > 0
    assert np.array_equal(radius[~fr], pre["radius"][~fr])
    both = (radius > 0) & (pre["radius"] > 0) & ~fr
    e = np.abs(rec10[both] - pre["rec"][both])
    r = pre["rec"][both]
    assert e[:, 0:2].max() < 2e-3 and (e[:, 2:5] / np.abs(r[:, 2:5]).max(1, keepdims=True)).max() < 1e-4
    assert e[:, 6:9].max() < 2e-5 and (e[:, 9] / r[:, 9]).max() < 1e-6

    # tile lists of the whole window
    ranges_o, vals_o = O.bin_lists(rec10[:, 0], rec10[:, 1], rec10[:, 9], radius, V, n, W, H, 16)
    gr = win.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    gv = win.vals[: int(win.n_inst.item())].cpu().numpy().view(np.uint32)
    tot, kept, dropped = check_culled_lists(win.rec.cpu().numpy().reshape(-1, 12), ranges_o, vals_o, gr, gv, W, H,
                                            16)
    print(f"[config {config}] lists: rect {tot} kept {kept} dropped {dropped}")

    # forward, every pixel
    tr, td = win.tgt_rgb.cpu().numpy().astype(np.float64), win.tgt_depth.cpu().numpy().astype(np.float64)
    fw = O.render_fwd(rec10, ranges_o, vals_o, V, W, H, 16, sc.cams, (0.0, 0.0, 0.0), tr, td, 0.1, tol=1e-5)
    ok = fw["near"] == 0
    img = win.img.cpu().numpy()
    err = np.abs(img - fw["img"]).max(1)
    dscale = max(1.0, np.abs(fw["depth"]).max())
    e_d = (np.abs(win.depth.cpu().numpy() - fw["depth"]) / dscale)[ok].max()
    e_T = np.abs(win.t_final.cpu().numpy() - fw["T"])[ok].max()
    print(f"[config {config}] pixels near a threshold {1 - ok.mean():.2e}, beyond {PIX_TOL:g} {(err > PIX_TOL).mean():.2e},"
          f" max|dimg| elsewhere {err[ok].max():.2e} |dT| {e_T:.2e} |ddepth|/scale {e_d:.2e}")
    assert err[ok].max() < PIX_TOL and e_T < PIX_TOL and e_d < PIX_TOL
    assert (err > PIX_TOL).mean() < 1e-4
    ls_g = last_slots(win.last.cpu().numpy(), gr, gv, W, H, 16)
    ls_o = last_slots(fw["last"], ranges_o, vals_o, W, H, 16)
    assert np.array_equal(ls_g[ok], ls_o[ok])
    np.testing.assert_allclose(win.loss_view.cpu().numpy(), fw["loss_view"], rtol=2e-5)

    # raster backward, every slot
    ref_sg, mag = O.render_bwd(rec10, ranges_o, vals_o, V, n, W, H, 16, sc.cams, img.astype(np.float64),
                               win.depth.cpu().numpy().astype(np.float64), tr, td,
                               win.depth_count.cpu().numpy().astype(np.int64), with_abs=True)
    flag = (fw["near"] != 0) | residual_sign_flags(fw["img"], tr, fw["depth"], td)
    near = slots_in_flagged_tiles(flag, ranges_o, vals_o, W, H, 16, V * n)
    sg = sg_from_gpu(win.slot_grad)
    touched = np.abs(ref_sg).sum(1) > 0
    print(f"[config {config}] slots with a gradient {touched.sum()}, in tiles with a flagged pixel {near.sum()}")
    field_grad_check(sg, ref_sg, near, f"config {config} slot", mag=mag)

    # preprocess backward: the oracle's chain rule on the oracle's own slot gradients
    ref = O.preprocess_bwd(sc.params, n, sc.sh_degree, sc.cams, W, H, 16, ref_sg)
    scale = np.abs(ref_sg).max(axis=0, keepdims=True)
    plain = GRAD_REL_TOL * (np.abs(ref_sg) + GRAD_REL_TOL * scale)
    dd = np.abs(sg - ref_sg)
    cond = ((dd > plain) & (dd <= plain + F32_COND * mag)).any(axis=1)
    expl = gaussians_of_slots(near | fr | cond, n)
    print(f"[config {config}] Gaussians near a threshold or float32-conditioned {expl.sum()} of {n}")
    param_grad_check(win.grads.cpu().numpy(), ref, n, sc.sh_degree, expl, f"config {config}")
