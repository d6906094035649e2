"""Pins of the oracle's adaptive density control (clone / split / prune with the paper's
thresholds, Sec. III-A.3 and IV-A): a hand-checked example, the output-count identity,
and the split children's spread against scipy's rotation (CPU only)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth.scenes import param_layout


def four_gaussians():
    n, deg = 4, 0
    lay = param_layout(n, deg)
    p = np.zeros(lay["total"], np.float32)
    p[0:12] = np.arange(12)                         # means
    ls = np.log([[0.01] * 3, [0.01] * 3, [0.5, 0.1, 0.1], [0.01] * 3])
    p[lay["log_scales"]: lay["log_scales"] + 12] = ls.reshape(-1)
    p[lay["quats"]: lay["quats"] + 16] = np.tile([1, 0, 0, 0], 4)
    p[lay["opacity"]: lay["opacity"] + 4] = [0.0, 0.0, 0.0, -5.0]    # sigmoid(-5) = 0.0067 < 0.02
    p[lay["sh_dc"]: lay["sh_dc"] + 12] = np.arange(12) * 0.1
    accum = np.array([0.0005, 0.004, 0.006, 0.01], np.float32)
    denom = np.array([1, 2, 2, 1], np.float32)                      # grads 0.0005, 0.002, 0.003, 0.01
    return p, n, deg, accum, denom


def test_hand_example():
    p, n, deg, accum, denom = four_gaussians()
    code, count = O.densify_plan(p, n, deg, accum, denom, tau_p=0.001, scale_thr=0.05, eps_alpha=0.02)
    # 0: low gradient -> keep; 1: high, small -> clone; 2: high, big -> split; 3: low opacity -> prune
    assert list(code) == [1, 2, 3, 0]
    assert list(count) == [1, 2, 2, 0]
    m = np.arange(p.size, dtype=np.float64) * 1e-3
    v = np.arange(p.size, dtype=np.float64) * 1e-4
    z = np.array([[[1.0, 0.0, 0.0], [0.0, -1.0, 0.0]]] * 4)
    P2, M2, V2, n2 = O.densify_apply(p, m, v, n, deg, code, z)
    assert n2 == 5
    means = P2[0:15].reshape(5, 3)
    np.testing.assert_allclose(means[0], [0, 1, 2])
    np.testing.assert_allclose(means[1], [3, 4, 5])
    np.testing.assert_allclose(means[2], [3, 4, 5])                  # the clone
    # split children of Gaussian 2 (identity rotation, scales 0.5, 0.1, 0.1): mean + s * z
    np.testing.assert_allclose(means[3], [6 + 0.5, 7, 8])
    np.testing.assert_allclose(means[4], [6, 7 - 0.1, 8])
    logs = P2[15:30].reshape(5, 3)
    np.testing.assert_allclose(np.exp(logs[3]), [0.5 / 1.6, 0.1 / 1.6, 0.1 / 1.6], rtol=1e-6)  # float32 input
    # Adam state: originals keep theirs, clone and children start at zero
    Mm = M2[0:15].reshape(5, 3)
    np.testing.assert_allclose(Mm[0], m[0:3])
    np.testing.assert_allclose(Mm[1], m[3:6])
    assert not Mm[2].any() and not Mm[3].any() and not Mm[4].any()
    # colours copied
    dc = P2[11 * 5: 14 * 5].reshape(5, 3)
    np.testing.assert_allclose(dc[2], dc[1])
    np.testing.assert_allclose(dc[3], p[param_layout(4, 0)["sh_dc"] + 6: param_layout(4, 0)["sh_dc"] + 9])


def test_count_identity_and_zero_denominator():
    rng = np.random.default_rng(0)
    n, deg = 500, 1
    lay = param_layout(n, deg)
    p = rng.normal(size=lay["total"]).astype(np.float32)
    p[lay["log_scales"]: lay["log_scales"] + 3 * n] = rng.normal(-3, 1, 3 * n)
    accum = rng.uniform(0, 0.01, n).astype(np.float32)
    denom = rng.integers(0, 4, n).astype(np.float32)                 # some never seen: grad 0
    code, count = O.densify_plan(p, n, deg, accum, denom, 0.001, 0.05, 0.02)
    assert np.all(code[denom == 0] <= 1)                             # unseen: never densified
    z = rng.normal(size=(n, 2, 3))
    P2, M2, V2, n2 = O.densify_apply(p, np.zeros(p.size), np.zeros(p.size), n, deg, code, z)
    assert n2 == count.sum() == (code == 1).sum() + 2 * (code == 2).sum() + 2 * (code == 3).sum()
    assert P2.size == param_layout(n2, deg)["total"]


def test_split_children_spread_matches_covariance():
    # for z ~ N(0, I), children mean + R (s * z) have covariance R diag(s^2) R^T (the
    # Gaussian's own covariance), with R from scipy's quaternion convention
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(3)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    s = np.array([0.3, 0.1, 0.05])
    n, deg = 1, 0
    lay = param_layout(n, deg)
    p = np.zeros(lay["total"])
    p[3:6] = np.log(s)
    p[6:10] = q
    code = np.array([3])
    samples = []
    for _ in range(4000):
        z = rng.normal(size=(1, 2, 3))
        P2, _, _, n2 = O.densify_apply(p, np.zeros(p.size), np.zeros(p.size), n, deg, code, z)
        samples.append(P2[0:6].reshape(2, 3))
    X = np.concatenate(samples)
    R = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sigma = R @ np.diag(s ** 2) @ R.T
    np.testing.assert_allclose(np.cov(X.T), Sigma, atol=4e-3)
