"""Pins of the oracle's geometric densification (a keyframe's coloured point cloud ->
initial Gaussians, Sec. III-A.3 / III-B with the 3DGS initialisation): the exact 3-nearest
neighbour distances against a hand example, a lattice closed form and scipy's k-d tree;
the initial attributes against the SH basis and the activations (CPU only)."""
import numpy as np
import pytest

from oracle import oracle as O
from synth import make_point_cloud
from synth.scenes import param_layout


def test_knn_hand_example():
    # points on a line at 0, 1, 3, 7: squared distances written out per point
    x = np.array([[0, 0, 0], [1, 0, 0], [3, 0, 0], [7, 0, 0]], float)
    expect = [(1 + 9 + 49) / 3, (1 + 4 + 36) / 3, (9 + 4 + 16) / 3, (49 + 36 + 16) / 3]
    np.testing.assert_allclose(O.knn_mean_d2(x), expect, rtol=1e-15)


def test_knn_lattice_closed_form():
    # a cubic lattice of spacing a: every point has (at least) three neighbours at distance a
    a = 0.37
    g = np.stack(np.meshgrid(np.arange(4), np.arange(3), np.arange(5), indexing="ij"), -1).reshape(-1, 3) * a
    np.testing.assert_allclose(O.knn_mean_d2(g), a * a, rtol=1e-13)


def test_knn_few_points():
    x = np.array([[0, 0, 0], [0, 2, 0], [0, 0, 3]], float)
    np.testing.assert_allclose(O.knn_mean_d2(x[:1]), [0.0])
    np.testing.assert_allclose(O.knn_mean_d2(x[:2]), [4.0, 4.0])
    np.testing.assert_allclose(O.knn_mean_d2(x), [(4 + 9) / 2, (4 + 13) / 2, (9 + 13) / 2])


def test_knn_matches_scipy_kdtree():
    from scipy.spatial import cKDTree
    xyz, _ = make_point_cloud(3, 1500, dup_frac=0.05)
    x = xyz.astype(np.float64)
    d, _ = cKDTree(x).query(x, k=4)          # includes the point itself at distance 0
    ref = (d[:, 1:] ** 2).mean(axis=1)
    got = O.knn_mean_d2(x)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    assert (d[:, 1] == 0).sum() > 0           # the cloud has exact duplicates (zero distances)


def test_gaussians_from_points_attributes():
    xyz, rgb = make_point_cloud(4, 300)
    for deg in (0, 1, 3):
        p = O.gaussians_from_points(xyz, rgb, deg)
        m = xyz.shape[0]
        lay = param_layout(m, deg)
        assert p.size == lay["total"]
        np.testing.assert_array_equal(p[: 3 * m].reshape(m, 3), xyz.astype(np.float64))
        logs = p[lay["log_scales"]: lay["quats"]].reshape(m, 3)
        d2 = np.maximum(O.knn_mean_d2(xyz), 1e-7)
        np.testing.assert_allclose(np.exp(2 * logs), np.repeat(d2[:, None], 3, 1), rtol=1e-12)
        q = p[lay["quats"]: lay["opacity"]].reshape(m, 4)
        assert np.all(q == [1, 0, 0, 0])
        o = 1.0 / (1.0 + np.exp(-p[lay["opacity"]: lay["sh_dc"]]))
        np.testing.assert_allclose(o, 0.1, rtol=1e-12)
        # the degree-0 colour (SH basis of the oracle, pinned against scipy) is the point's rgb
        Y, _ = O.sh_basis(0, (0.3, -0.2, 0.9))
        dc = p[lay["sh_dc"]: lay["sh_rest"]].reshape(m, 3)
        np.testing.assert_allclose(Y[0] * dc + 0.5, rgb, atol=1e-12)
        assert np.all(p[lay["sh_rest"]:] == 0)


def test_gaussians_from_points_floor_for_duplicates():
    xyz = np.array([[1, 2, 3]] * 5, np.float32)
    p = O.gaussians_from_points(xyz, np.zeros((5, 3)), 0)
    np.testing.assert_allclose(p[15:30], 0.5 * np.log(1e-7))
    with pytest.raises(ValueError):
        O.knn_mean_d2(xyz, k=0)


def test_sampled_knn_equals_full():
    xyz, _ = make_point_cloud(8, 800, dup_frac=0.05)
    idx = np.array([0, 5, 799, 400, 5])
    np.testing.assert_array_equal(O.knn_mean_d2_at(xyz, idx), O.knn_mean_d2(xyz)[idx])
    with pytest.raises(ValueError):
        O.knn_mean_d2_at(xyz, [800])
