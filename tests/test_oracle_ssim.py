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
