"""Pins of the oracle's projection / SH colour step against closed forms, scipy and
invariants (CPU only).  Paper: the "projected 2D Gaussian" and colour c_k of Eq. 1
(Sec. III-B); the projection itself is the 3DGS one the paper builds on."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth.scenes import param_layout, _camera_row, look_at


def one_gaussian(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, dc=(0, 0, 0), deg=0, rest=None):
    n = 1
    K = (deg + 1) ** 2
    lay = param_layout(n, deg)
    p = np.zeros(lay["total"])
    p[0:3] = mean
    p[3:6] = log_scale
    p[6:10] = quat
    p[10] = logit
    p[11:14] = dc
    if deg > 0:
        p[14:] = np.zeros(3 * (K - 1)) if rest is None else np.asarray(rest).reshape(-1)
    return p


def cam(f=150.0, cx=80.0, cy=60.0, R=np.eye(3), t=np.zeros(3)):
    return _camera_row(R, t, f, f, cx, cy)[None].astype(np.float64)


def test_isotropic_on_axis_closed_form():
    # isotropic scale s at depth z on the optical axis: Sigma' = (f s / z)^2 I + 0.3 I
    f, z, s = 150.0, 2.0, 0.05
    p = one_gaussian((0, 0, z), (math.log(s),) * 3)
    out = O.preprocess(p, 1, 0, cam(f), 160, 120, 16)
    rec = out["rec"][0]
    a = (f * s / z) ** 2 + 0.3
    assert rec[0] == pytest.approx(80.0, abs=1e-12)
    assert rec[1] == pytest.approx(60.0, abs=1e-12)
    np.testing.assert_allclose(rec[2:5], [1 / a, 0.0, 1 / a], rtol=1e-12, atol=1e-15)
    assert rec[5] == pytest.approx(0.5)          # sigmoid(0)
    assert rec[9] == pytest.approx(z)
    # mid^2 - det = 0 for an isotropic footprint, so lambda = a + sqrt(0.1) (floor 0.1)
    assert out["radius"][0] == math.ceil(3 * math.sqrt(a + math.sqrt(0.1)))


def test_worked_projection_point():
    # camera at the origin looking +z: point (1, 0.5, 2) lands at (80 + 150*0.5, 60 + 150*0.25)
    p = one_gaussian((1.0, 0.5, 2.0), (-3.0,) * 3)
    rec = O.preprocess(p, 1, 0, cam(), 160, 120, 16)["rec"][0]
    assert rec[0] == pytest.approx(155.0)
    assert rec[1] == pytest.approx(97.5)


def numeric_cov2(mean, Sigma, f, cx, cy, Rc, tc):
    """2D covariance from a central-difference Jacobian of the perspective map."""
    def proj(x):
        t = Rc @ x + tc
        return np.array([f * t[0] / t[2] + cx, f * t[1] / t[2] + cy])
    h = 1e-6
    Jw = np.zeros((2, 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        Jw[:, i] = (proj(mean + e) - proj(mean - e)) / (2 * h)
    return Jw @ Sigma @ Jw.T + 0.3 * np.eye(2)


@pytest.mark.parametrize("seed", range(6))
def test_ewa_covariance_matches_numeric_jacobian(seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    ls = rng.normal(-2.5, 0.5, 3)
    R, t = look_at((0.3, -0.2, -0.5), (0.1, 0.2, 3.0), world_up=(0, -1, 0))
    mean = rng.uniform([-0.8, -0.6, 2.0], [0.8, 0.6, 4.0])
    p = one_gaussian(mean, ls, q)
    C = _camera_row(R, t, 150, 150, 80, 60)[None].astype(np.float64)
    Rc = C[0, :9].reshape(3, 3)
    tc = C[0, 9:12]
    out = O.preprocess(p, 1, 0, C, 160, 120, 16)
    assert out["radius"][0] > 0
    A, B, Cc = out["rec"][0, 2:5]
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    Rq = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: scalar-last
    Sigma = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
    cov2 = numeric_cov2(mean, Sigma, 150, 80, 60, Rc, tc)
    np.testing.assert_allclose(np.linalg.inv(np.array([[A, B], [B, Cc]])), cov2, rtol=1e-6)


def test_rotation_about_z_swaps_axes():
    # q = (cos 45, 0, 0, sin 45) rotates x into y: world covariance diag(sy^2, sx^2, sz^2)
    sx, sy = 0.08, 0.02
    c = math.cos(math.pi / 4)
    z = 3.0
    p_rot = one_gaussian((0, 0, z), (math.log(sx), math.log(sy), math.log(0.01)), (c, 0, 0, c))
    p_ref = one_gaussian((0, 0, z), (math.log(sy), math.log(sx), math.log(0.01)))
    r1 = O.preprocess(p_rot, 1, 0, cam(), 160, 120, 16)["rec"][0]
    r2 = O.preprocess(p_ref, 1, 0, cam(), 160, 120, 16)["rec"][0]
    np.testing.assert_allclose(r1[2:5], r2[2:5], rtol=1e-10, atol=1e-14)


def test_quaternion_scale_invariance():
    # q and 3q describe the same rotation (normalised before use)
    q = np.array([0.3, -0.5, 0.7, 0.2])
    p1 = one_gaussian((0.2, 0.1, 2.5), (-2.5, -3.0, -2.8), q)
    p2 = one_gaussian((0.2, 0.1, 2.5), (-2.5, -3.0, -2.8), 3 * q)
    r1 = O.preprocess(p1, 1, 0, cam(), 160, 120, 16)["rec"][0]
    r2 = O.preprocess(p2, 1, 0, cam(), 160, 120, 16)["rec"][0]
    np.testing.assert_allclose(r1, r2, rtol=1e-12)


def test_guard_band_freezes_jacobian():
    # beyond 1.3 x half-FoV the Jacobian uses the clamped x: moving further out at a fixed
    # depth no longer changes the footprint (only the centre moves)
    z = 2.0
    lim = 1.3 * (160 / 2) / 150
    recs = []
    for x in (lim * z * 1.1, lim * z * 1.3):
        p = one_gaussian((x, 0.0, z), (math.log(0.9),) * 3)
        out = O.preprocess(p, 1, 0, cam(), 160, 120, 16)
        assert out["radius"][0] > 0
        recs.append(out["rec"][0])
    np.testing.assert_allclose(recs[0][2:5], recs[1][2:5], rtol=1e-12)
    assert recs[1][0] > recs[0][0]


def test_near_plane_cull():
    for z, vis in ((0.19, False), (0.21, True)):
        p = one_gaussian((0.0, 0.0, z), (-6.0,) * 3)
        out = O.preprocess(p, 1, 0, cam(), 160, 120, 16)
        assert (out["radius"][0] > 0) == vis


def test_offscreen_rect_is_culled():
    p = one_gaussian((5.0, 0.0, 2.0), (-5.0,) * 3)   # u = 455 px, far right of a 160 px image
    out = O.preprocess(p, 1, 0, cam(), 160, 120, 16)
    assert out["radius"][0] == 0


def test_rect_straddling_tile_corner():
    # centre exactly at pixel (32, 16) (a tile corner for B=16) and a known radius:
    # x tiles [floor((32-r)/16), floor((32+r+15)/16)), y tiles likewise from 16
    f, z, s = 150.0, 2.0, 0.02
    u, v = 32.0, 16.0
    p = one_gaussian(((u - 80) * z / f, (v - 60) * z / f, z), (math.log(s),) * 3)
    out = O.preprocess(p, 1, 0, cam(f), 160, 120, 16)
    r = out["radius"][0]
    assert out["rec"][0, 0] == pytest.approx(u) and out["rec"][0, 1] == pytest.approx(v)
    exp = [max(0, (32 - r) // 16), min(10, (32 + r + 15) // 16),
           max(0, (16 - r) // 16), min(8, (16 + r + 15) // 16)]
    assert list(out["rect"][0]) == exp


def scipy_real_sh(l, m, d):
    """Real SH with the Condon-Shortley phase kept: sqrt2 Im Y_l^|m| (m<0), Y_l^0, sqrt2 Re Y_l^m."""
    sp = pytest.importorskip("scipy.special")
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x) % (2 * math.pi)
    Y = sp.sph_harm_y(l, abs(m), theta, phi)
    if m < 0:
        return math.sqrt(2) * Y.imag
    if m == 0:
        return Y.real
    return math.sqrt(2) * Y.real


@pytest.mark.parametrize("seed", range(5))
def test_sh_basis_matches_scipy(seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    Y, _ = O.sh_basis(3, d)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            assert Y[k] == pytest.approx(scipy_real_sh(l, m, d), abs=1e-12), (l, m)
            k += 1


def test_sh_basis_gradient_fd():
    rng = np.random.default_rng(7)
    d = rng.normal(size=3)
    _, dY = O.sh_basis(3, d)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (O.sh_basis(3, d + e)[0] - O.sh_basis(3, d - e)[0]) / (2 * h)
        np.testing.assert_allclose(dY[:, i], fd, atol=1e-8)


def test_sh_degree0_colour_is_view_independent_and_clamped():
    Y0 = 0.5 / math.sqrt(math.pi)
    dc = np.array([0.2, -0.5, -3.0]) / Y0          # rgb = 0.7, 0.0, -2.5 -> clamped to 0
    recs = []
    for t in ((0, 0, 0), (0.3, -0.1, 0.2)):
        p = one_gaussian((0.1, 0.05, 2.0), (-3.0,) * 3, dc=dc)
        out = O.preprocess(p, 1, 0, cam(t=np.array(t, float)), 160, 120, 16)
        recs.append(out["rec"][0, 6:9])
        assert out["clamp"][0] == 0b100
    np.testing.assert_allclose(recs[0], [0.7, 0.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(recs[1], recs[0], atol=1e-12)


def test_sh_degree1_band_rotation():
    # the l = 1 band is a linear function of the direction: rgb - (Y0 dc + 1/2) = -c1 (y, -z, x).k
    c1 = math.sqrt(3 / (4 * math.pi))
    k = np.array([[0.1, 0.2, 0.3], [-0.2, 0.05, 0.1], [0.3, -0.1, 0.2]])  # rest[3][3]
    mean = np.array([0.4, -0.3, 2.0])
    p = one_gaussian(mean, (-3.0,) * 3, dc=(0, 0, 0), deg=1, rest=k)
    rec = O.preprocess(p, 1, 1, cam(), 160, 120, 16)["rec"][0]
    d = mean / np.linalg.norm(mean)
    basis = np.array([-c1 * d[1], c1 * d[2], -c1 * d[0]])
    np.testing.assert_allclose(rec[6:9], np.maximum(basis @ k + 0.5, 0.0), atol=1e-12)
