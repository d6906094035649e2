"""Pins of the oracle's hand-derived backward (Eqs. 2-4 plus the projection chain rule)
against central finite differences of the oracle's own forward, in float64, on tiny
scenes; plus the per-view sum identity, the opacity regulariser (Eqs. 10-11) and the
densification statistics (CPU only)."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import make_tiny_scene
from synth.scenes import param_layout

H_FD = 1e-4


def targets(sc, seed=11):
    """Target image/depth: the oracle's render of the perturbed copy, with depth noise and
    a band of invalid (zero) depth."""
    pre = O.preprocess(sc.params_target, sc.n, sc.sh_degree, sc.cams, sc.width, sc.height, sc.tile)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], sc.views, sc.n,
                               sc.width, sc.height, sc.tile)
    fw = O.render_fwd(rec, ranges, vals, sc.views, sc.width, sc.height, sc.tile, sc.cams)
    rng = np.random.default_rng(seed)
    tgt_rgb = fw["img"] + rng.normal(0, 0.02, fw["img"].shape)
    tgt_d = fw["depth"] + rng.normal(0, 0.05, fw["depth"].shape)
    tgt_d[:, : sc.height // 4] = 0.0
    return tgt_rgb, tgt_d


def evaluate(sc, params, tgt_rgb, tgt_d, cams=None, bg=(0.0, 0.0, 0.0)):
    cams = sc.cams if cams is None else cams
    V = cams.shape[0]
    pre = O.preprocess(params, sc.n, sc.sh_degree, cams, sc.width, sc.height, sc.tile)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], V, sc.n,
                               sc.width, sc.height, sc.tile)
    fw = O.render_fwd(rec, ranges, vals, V, sc.width, sc.height, sc.tile, cams, bg=bg,
                      tgt_rgb=tgt_rgb, tgt_depth=tgt_d, lambda_d=0.1, want_hash=True)
    sig = (fw["hash"], vals.tobytes(), ranges.tobytes(), pre["radius"].tobytes(),
           pre["clamp"].tobytes(), np.sign(fw["img"] - tgt_rgb).tobytes(),
           np.sign(fw["depth"] - tgt_d).tobytes())
    return float(fw["loss_view"].sum()), sig


FD_CASES = [(0, 1, 0.0, (0.0, 0.0, 0.0)), (1, 2, 0.0, (0.2, 0.5, 0.1)),
            (3, 3, 1.0, (0.0, 0.0, 0.0)), (1, 4, -1.0, (1.0, 0.3, 0.0))]


@pytest.mark.parametrize("deg,seed,opac,bg", FD_CASES)
def test_backward_matches_central_fd(deg, seed, opac, bg):
    sc = make_tiny_scene(seed=seed, n=24, sh_degree=deg, W=32, H=24, views=2, tile=8,
                         opacity_mean=opac)
    params = sc.params.astype(np.float64)
    tgt_rgb, tgt_d = targets(sc)
    it = O.iteration(params, sc.n, deg, sc.cams, sc.width, sc.height, sc.tile, tgt_rgb, tgt_d,
                     bg=bg)
    g = it["grads"]
    L0, sig0 = evaluate(sc, params, tgt_rgb, tgt_d, bg=bg)
    assert L0 == pytest.approx(it["loss"], rel=1e-14)
    checked = skipped = 0
    gmax = np.abs(g).max()
    for i in range(params.size):
        pp = params.copy()
        pp[i] += H_FD
        Lp, sp = evaluate(sc, pp, tgt_rgb, tgt_d, bg=bg)
        pm = params.copy()
        pm[i] -= H_FD
        Lm, sm = evaluate(sc, pm, tgt_rgb, tgt_d, bg=bg)
        if sp != sig0 or sm != sig0:
            skipped += 1               # a discrete decision changed inside [-h, h]
            continue
        fd = (Lp - Lm) / (2 * H_FD)
        assert abs(fd - g[i]) <= 1e-6 * gmax + 1e-4 * abs(g[i]), (i, fd, g[i])
        checked += 1
    assert checked > 0.9 * params.size, (checked, skipped)
    assert np.count_nonzero(g) > 0.5 * params.size


def test_window_gradient_is_sum_of_views():
    sc = make_tiny_scene(seed=5, n=30, sh_degree=1, W=32, H=24, views=3, tile=8)
    params = sc.params.astype(np.float64)
    tgt_rgb, tgt_d = targets(sc)
    full = O.iteration(params, sc.n, 1, sc.cams, sc.width, sc.height, sc.tile, tgt_rgb, tgt_d)
    acc = np.zeros_like(full["grads"])
    loss = 0.0
    for v in range(3):
        it = O.iteration(params, sc.n, 1, sc.cams[v:v + 1], sc.width, sc.height, sc.tile,
                         tgt_rgb[v:v + 1], tgt_d[v:v + 1])
        acc += it["grads"]
        loss += it["loss"]
    np.testing.assert_allclose(full["grads"], acc, rtol=1e-12, atol=1e-15)
    assert full["loss"] == pytest.approx(loss, rel=1e-13)


def test_loss_weight_scales_view():
    sc = make_tiny_scene(seed=6, n=20, sh_degree=0, W=16, H=16, views=1, tile=8)
    params = sc.params.astype(np.float64)
    tgt_rgb, tgt_d = targets(sc)
    it1 = O.iteration(params, sc.n, 0, sc.cams, 16, 16, 8, tgt_rgb, tgt_d)
    cams = sc.cams.copy()
    cams[:, 16] = 3.0
    it3 = O.iteration(params, sc.n, 0, cams, 16, 16, 8, tgt_rgb, tgt_d)
    np.testing.assert_allclose(it3["grads"], 3 * it1["grads"], rtol=1e-12, atol=1e-16)
    assert it3["loss"] == pytest.approx(3 * it1["loss"])


def test_opacity_regulariser_gradient():
    # L_o = lambda_o / N sum sigmoid(x_i) (Eqs. 10-11): d/dx_i = lambda_o o_i (1 - o_i) / N
    sc = make_tiny_scene(seed=2, n=10, sh_degree=0)
    p = sc.params.astype(np.float64)
    lo, g = O.opacity_reg(p, sc.n, 0.001)
    x = p[10 * sc.n: 11 * sc.n]
    assert lo == pytest.approx(0.001 * np.mean(1 / (1 + np.exp(-x))))
    for i in range(sc.n):
        pp = p.copy()
        pp[10 * sc.n + i] += 1e-5
        pm = p.copy()
        pm[10 * sc.n + i] -= 1e-5
        fd = (O.opacity_reg(pp, sc.n, 0.001)[0] - O.opacity_reg(pm, sc.n, 0.001)[0]) / 2e-5
        assert fd == pytest.approx(g[i], rel=1e-6)


def test_densify_stats_hand_example():
    # one Gaussian seen by two views (one culled in a third): accum is the sum of the
    # per-view NDC gradient norms, denom the number of views it was visible in
    n, V, W, H = 1, 3, 40, 20
    sg = np.zeros((V * n, 10))
    sg[0, :2] = (0.03, -0.04)      # (0.6, -0.4)  -> norm sqrt(0.52)
    sg[1, :2] = (0.0, 0.1)         # (0, 1.0)      -> 1.0
    sg[2, :2] = (5.0, 5.0)         # culled view: ignored
    radius = np.array([7, 3, 0], np.int32)
    acc, den, mx = O.densify_stats(sg, radius, V, n, W, H)
    assert acc[0] == pytest.approx(np.sqrt(0.6 ** 2 + 0.4 ** 2) + 1.0)
    assert den[0] == 2
    assert mx[0] == 7
    acc2, den2, mx2 = O.densify_stats(sg, radius, V, n, W, H, acc, den, mx)
    assert den2[0] == 4 and acc2[0] == pytest.approx(2 * acc[0]) and mx2[0] == 7


def test_params_layout_groups():
    lay = param_layout(5, 3)
    assert lay["total"] == 5 * 59
    assert lay["sh_rest"] - lay["sh_dc"] == 15


def test_operand_magnitudes_bound_the_gradient_terms():
    # grads_mag sums each term with its operands replaced by their magnitudes: never below
    # |grad| (triangle inequality); for the colour and depth fields, whose terms are single
    # products, equal to the sum of |terms|, i.e. |grad| where every term has one sign
    sc = make_tiny_scene(seed=2, n=40, sh_degree=1, W=32, H=24, views=2, tile=8)
    pre = O.preprocess(sc.params, sc.n, 1, sc.cams, sc.width, sc.height, sc.tile)
    rec = pre["rec"]
    ranges, vals = O.bin_records(rec, pre["radius"], 2, sc.n, sc.width, sc.height, sc.tile)
    fw = O.render_fwd(rec, ranges, vals, 2, sc.width, sc.height, sc.tile, sc.cams)
    tgt = fw["img"] + 0.05
    g, mag = O.render_bwd(rec, ranges, vals, 2, sc.n, sc.width, sc.height, sc.tile, sc.cams, fw["img"],
                          fw["depth"], tgt, None, fw["depth_count"], with_abs=True)
    g2 = O.render_bwd(rec, ranges, vals, 2, sc.n, sc.width, sc.height, sc.tile, sc.cams, fw["img"],
                      fw["depth"], tgt, None, fw["depth_count"])
    assert np.array_equal(g, g2)                       # the magnitudes do not touch the gradient
    assert np.all(mag >= np.abs(g) * (1 - 1e-12))
    np.testing.assert_allclose(mag[:, 6:9], np.abs(g[:, 6:9]), rtol=1e-12)   # img < tgt: one sign
    assert (mag[:, 0] > 1.5 * np.abs(g[:, 0])).any()  # du terms cancel somewhere
