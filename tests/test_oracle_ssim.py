"""Pins of the oracle's SSIM term (Eq. 9): brute-force windowed sums on a small image,
identity and symmetry, and central finite differences of the gradient (CPU only)."""
import numpy as np
import pytest

from oracle import oracle as O


def brute_ssim_map(x, y):
    """Per pixel, the 11x11 window sums written out (zero outside the image)."""
    g = O.ssim_window()
    w2 = np.outer(g, g)
    H, W = x.shape
    r = 5
    S = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = exx = eyy = exy = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < H and 0 <= jj < W:
                        wt = w2[a + r, b + r]
                        xv, yv = x[ii, jj], y[ii, jj]
                        mx += wt * xv
                        my += wt * yv
                        exx += wt * xv * xv
                        eyy += wt * yv * yv
                        exy += wt * xv * yv
            sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
            S[i, j] = ((2 * mx * my + O.SSIM_C1) * (2 * sxy + O.SSIM_C2)) / \
                ((mx * mx + my * my + O.SSIM_C1) * (sx + sy + O.SSIM_C2))
    return S


def test_window_is_normalised_gaussian():
    g = O.ssim_window()
    assert g.sum() == pytest.approx(1.0)
    assert g[5] == g.max() and g[0] == pytest.approx(g[10])
    assert g[6] / g[5] == pytest.approx(np.exp(-1 / (2 * 1.5 ** 2)))


def test_ssim_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (1, 3, 9, 13))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    loss, _ = O.ssim_loss(x, y)
    S = np.stack([brute_ssim_map(x[0, c], y[0, c]) for c in range(3)])
    assert loss[0] == pytest.approx(1.0 - S.mean(), rel=1e-12)


def test_identity_and_symmetry():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (2, 3, 12, 10))
    y = rng.uniform(0, 1, (2, 3, 12, 10))
    loss, grad = O.ssim_loss(x, x)
    np.testing.assert_allclose(loss, 0.0, atol=1e-12)
    np.testing.assert_allclose(grad, 0.0, atol=1e-12)      # a maximum of SSIM
    l1, _ = O.ssim_loss(x, y)
    l2, _ = O.ssim_loss(y, x)
    np.testing.assert_allclose(l1, l2, rtol=1e-12)


def test_gradient_central_fd():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (1, 3, 8, 9))
    y = rng.uniform(0, 1, (1, 3, 8, 9))
    _, grad = O.ssim_loss(x, y)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 3, 4), (0, 2, 7, 8), (0, 0, 4, 0), (0, 1, 0, 8), (0, 2, 5, 5)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (O.ssim_loss(xp, y)[0][0] - O.ssim_loss(xm, y)[0][0]) / (2 * h)
        assert fd == pytest.approx(grad[idx], rel=1e-6, abs=1e-10)


# ---------------------------------------------------------------- Eq. 9 in full

def _render(sc, params, cams=None):
    cams = sc.cams if cams is None else cams
    V = cams.shape[0]
    pre = O.preprocess(params, sc.n, sc.sh_degree, cams, sc.width, sc.height, sc.tile)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], V, sc.n,
                               sc.width, sc.height, sc.tile)
    return pre, ranges, vals


def test_photometric_loss_without_ssim_is_the_fused_l1():
    # lambda_ssim = 0: the numpy loss of Eq. 9 equals the C forward's fused L1 + depth loss,
    # and feeding its pixel gradients to the backward equals the fused backward
    from tests.test_oracle_grad import targets
    from synth import make_tiny_scene
    sc = make_tiny_scene(seed=4, n=30, sh_degree=1, W=32, H=24, views=2, tile=8)
    params = sc.params.astype(np.float64)
    tgt_rgb, tgt_d = targets(sc)
    cams = sc.cams.copy()
    cams[:, 16] = (1.0, 2.5)
    pre, ranges, vals = _render(sc, params, cams)
    rec = pre["rec"]
    fw = O.render_fwd(rec, ranges, vals, 2, sc.width, sc.height, sc.tile, cams, tgt_rgb=tgt_rgb,
                      tgt_depth=tgt_d, lambda_d=0.1)
    lv, gi, gd = O.photometric_loss(fw["img"], fw["depth"], tgt_rgb, tgt_d, cams[:, 16], 0.0, 0.1)
    np.testing.assert_allclose(lv, fw["loss_view"], rtol=1e-12)
    fused = O.render_bwd(rec, ranges, vals, 2, sc.n, sc.width, sc.height, sc.tile, cams, fw["img"],
                         fw["depth"], tgt_rgb, tgt_d, fw["depth_count"], lambda_d=0.1)
    given = O.render_bwd(rec, ranges, vals, 2, sc.n, sc.width, sc.height, sc.tile, cams, fw["img"],
                         fw["depth"], tgt_rgb, tgt_d, fw["depth_count"], lambda_d=0.1, dl_dimg=gi,
                         dl_ddepth=gd)
    assert np.count_nonzero(fused) > 0
    np.testing.assert_allclose(given, fused, rtol=1e-12, atol=1e-18)


def test_photometric_loss_depth_term_hand_example():
    # one view, 1x2 image: depth residuals +0.5 (valid) and -3 (invalid target 0)
    img = np.full((1, 3, 1, 2), 0.5)
    tgt = np.full((1, 3, 1, 2), 0.25)
    dep = np.array([[[2.5, 4.0]]])
    tgd = np.array([[[2.0, 0.0]]])
    lv, gi, gd = O.photometric_loss(img, dep, tgt, tgd, [2.0], 0.0, 0.1)
    assert lv[0] == pytest.approx(2.0 * (0.25 + 0.1 * 0.5))
    np.testing.assert_allclose(gi, 2.0 / 6.0)
    np.testing.assert_allclose(gd, [[[0.2, 0.0]]])


@pytest.mark.parametrize("deg,seed,lam", [(1, 7, 0.2), (0, 8, 0.8)])
def test_eq9_gradient_matches_central_fd(deg, seed, lam):
    # the whole chain (SSIM + L1 + depth -> blend backward with given pixel gradients ->
    # projection chain rule) against central differences of the forward loss
    from tests.test_oracle_grad import targets
    from synth import make_tiny_scene
    sc = make_tiny_scene(seed=seed, n=20, sh_degree=deg, W=24, H=16, views=2, tile=8)
    params = sc.params.astype(np.float64)
    tgt_rgb, tgt_d = targets(sc)
    it = O.iteration(params, sc.n, deg, sc.cams, sc.width, sc.height, sc.tile, tgt_rgb, tgt_d,
                     lambda_ssim=lam)
    g = it["grads"]

    def evaluate(p):
        pre, ranges, vals = _render(sc, p)
        fw = O.render_fwd(pre["rec"], ranges, vals, 2, sc.width, sc.height, sc.tile, sc.cams,
                          tgt_rgb=tgt_rgb, tgt_depth=tgt_d, lambda_d=0.1, want_hash=True)
        lv, _, _ = O.photometric_loss(fw["img"], fw["depth"], tgt_rgb, tgt_d, sc.cams[:, 16], lam, 0.1)
        sig = (fw["hash"], vals.tobytes(), ranges.tobytes(), pre["radius"].tobytes(),
               pre["clamp"].tobytes(), np.sign(fw["img"] - tgt_rgb).tobytes(),
               np.sign(fw["depth"] - tgt_d).tobytes())
        return float(lv.sum()), sig

    L0, sig0 = evaluate(params)
    assert L0 == pytest.approx(it["loss"], rel=1e-14)
    h = 1e-4
    gmax = np.abs(g).max()
    checked = 0
    for i in range(params.size):
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        Lp, sp = evaluate(pp)
        Lm, sm = evaluate(pm)
        if sp != sig0 or sm != sig0:
            continue
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * gmax + 1e-4 * abs(g[i]), (i, fd, g[i])
        checked += 1
    assert checked > 0.9 * params.size
    assert np.count_nonzero(g) > 0.5 * params.size
