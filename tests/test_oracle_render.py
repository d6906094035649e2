"""Pins of the oracle's binning, blending (Eq. 1) and L1 loss against closed forms,
invariants and a brute-force pure-Python renderer (CPU only)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth import make_scene, make_tiny_scene, make_records
from synth.scenes import param_layout, _camera_row

Y0 = 0.5 / math.sqrt(math.pi)


def stack_params(depths, logit, rgb, s=0.05, x=0.0, y=0.0):
    n = len(depths)
    lay = param_layout(n, 0)
    p = np.zeros(lay["total"])
    for g, z in enumerate(depths):
        p[3 * g: 3 * g + 3] = (x * z, y * z, z)          # all on the same ray
        p[lay["log_scales"] + 3 * g: lay["log_scales"] + 3 * g + 3] = math.log(s * z)
        p[lay["quats"] + 4 * g] = 1.0
        p[lay["opacity"] + g] = logit
        p[lay["sh_dc"] + 3 * g: lay["sh_dc"] + 3 * g + 3] = (np.asarray(rgb) - 0.5) / Y0
    return p, n


def render(p, n, deg=0, W=160, H=120, B=16, f=150.0, cx=80.0, cy=60.0, bg=(0, 0, 0)):
    cams = _camera_row(np.eye(3), np.zeros(3), f, f, cx, cy)[None]
    pre = O.preprocess(p, n, deg, cams, W, H, B)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], 1, n, W, H, B)
    return pre, ranges, vals, O.render_fwd(rec, ranges, vals, 1, W, H, B, cams, bg=bg)


def test_single_gaussian_at_pixel_centre():
    # o = sigmoid(0) = 0.5 at the centre pixel (80, 60): I = 0.5 c + 0.5 bg, D = 0.5 z, T = 0.5
    p, n = stack_params([2.0], 0.0, (0.6, 0.3, 0.9))
    _, _, _, fw = render(p, n, bg=(0.1, 0.2, 0.3))
    np.testing.assert_allclose(fw["img"][0, :, 60, 80], 0.5 * np.array([0.6, 0.3, 0.9])
                               + 0.5 * np.array([0.1, 0.2, 0.3]), atol=1e-12)
    assert fw["depth"][0, 60, 80] == pytest.approx(1.0)
    assert fw["T"][0, 60, 80] == pytest.approx(0.5)
    assert fw["last"][0, 60, 80] == 1


def test_stack_transmittance_and_early_stop():
    # identical alpha = 0.8 splats on one ray: T = 0.2^k; the 6th would take T below 1e-4,
    # so blending stops after 5 with T = 0.2^5 and I = c (1 - 0.2^5)
    logit = math.log(0.8 / 0.2)
    p, n = stack_params([1.0 + 0.1 * k for k in range(8)], logit, (1.0, 0.5, 0.25))
    _, _, _, fw = render(p, n)
    T = 0.2 ** 5
    assert fw["T"][0, 60, 80] == pytest.approx(T, rel=1e-12)
    assert fw["last"][0, 60, 80] == 5
    np.testing.assert_allclose(fw["img"][0, :, 60, 80], np.array([1.0, 0.5, 0.25]) * (1 - T),
                               rtol=1e-12)
    # depth = sum z_k alpha T_k
    zs = np.array([1.0 + 0.1 * k for k in range(5)])
    wts = 0.8 * 0.2 ** np.arange(5)
    assert fw["depth"][0, 60, 80] == pytest.approx((zs * wts).sum(), rel=1e-12)


def test_alpha_clamped_at_099():
    # logit 10 -> o = 0.99995 -> alpha = min(0.99, .) = 0.99 at the centre
    p, n = stack_params([2.0], 10.0, (1, 1, 1))
    _, _, _, fw = render(p, n)
    assert fw["T"][0, 60, 80] == pytest.approx(0.01, rel=1e-12)


def test_alpha_sum_invariant():
    # with every colour 1, depth-ordered blending gives I = sum alpha_k T_k = 1 - T_final
    sc = make_scene(1, n=600)
    p = sc.params.astype(np.float64).copy()
    lay = param_layout(sc.n, 0)
    p[lay["sh_dc"]: lay["sh_dc"] + 3 * sc.n] = 0.5 / Y0
    _, _, _, fw = render(p, sc.n)
    np.testing.assert_allclose(fw["img"][0], np.broadcast_to(1 - fw["T"][0], (3, 120, 160)),
                               atol=1e-12)


def brute_render(rec, radius, rect, n, W, H, B):
    """Pure-Python renderer: per pixel, every Gaussian whose tile rect covers the pixel's
    tile (rect taken from the C4 formula with a float floor of (u - r)/B), sorted by
    (depth, index), blended front to back with the same 3DGS rules."""
    Tx = (W + B - 1) // B
    Ty = (H + B - 1) // B
    img = np.zeros((3, H, W))
    Tf = np.ones((H, W))
    for y in range(H):
        for x in range(W):
            tx, ty = x // B, y // B
            cand = []
            for g in range(n):
                if radius[g] <= 0:
                    continue
                u, v, r = rec[g, 0], rec[g, 1], radius[g]
                x0 = min(max(math.floor((u - r) / B), 0), Tx)
                x1 = min(max(math.floor((u + r + B - 1) / B), 0), Tx)
                y0 = min(max(math.floor((v - r) / B), 0), Ty)
                y1 = min(max(math.floor((v + r + B - 1) / B), 0), Ty)
                if x0 <= tx < x1 and y0 <= ty < y1:
                    cand.append((rec[g, 9], g))
            cand.sort()
            T = 1.0
            C = np.zeros(3)
            for _, g in cand:
                u, v, A, Bc, Cc, o = rec[g, :6]
                dx, dy = u - x, v - y
                power = -0.5 * (A * dx * dx + Cc * dy * dy) - Bc * dx * dy
                if power > 0:
                    continue
                a = min(0.99, o * math.exp(power))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                C += rec[g, 6:9] * a * T
                T *= 1 - a
            img[:, y, x] = C
            Tf[y, x] = T
    return img, Tf


@pytest.mark.parametrize("seed", [3, 8])
def test_tiled_render_matches_brute_force(seed):
    # a tile's list holds every splat whose rect covers the tile, so the tiled render equals
    # the render over all Gaussians
    sc = make_tiny_scene(seed=seed, n=30, sh_degree=1, W=24, H=16, views=1, tile=8)
    cams = sc.cams
    pre = O.preprocess(sc.params, sc.n, 1, cams, sc.width, sc.height, sc.tile)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], 1, sc.n,
                               sc.width, sc.height, sc.tile)
    fw = O.render_fwd(rec, ranges, vals, 1, sc.width, sc.height, sc.tile, cams)
    img, Tf = brute_render(rec, pre["radius"], pre["rect"], sc.n, sc.width, sc.height, sc.tile)
    assert (pre["radius"] > 0).sum() > 10
    np.testing.assert_allclose(fw["img"][0], img, atol=1e-12)
    np.testing.assert_allclose(fw["T"][0], Tf, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_bin_lists_brute_force(seed):
    # every visible slot sits in exactly the tiles of its rect (float floor((u - r)/B)
    # formula), lists are ordered by depth then slot, ranges tile the list contiguously
    V, n, W, H, B = 2, 300, 96, 64, 16
    u, v, r, z = make_records(seed, V, n, W, H, max_radius=24)
    ranges, vals = O.bin_lists(u, v, z, r, V, n, W, H, B)
    Tx, Ty = (W + B - 1) // B, (H + B - 1) // B
    expect = {}
    for s in range(V * n):
        if r[s] <= 0:
            continue
        uu, vv, rr = float(u[s]), float(v[s]), int(r[s])
        x0 = min(max(math.floor((uu - rr) / B), 0), Tx)
        x1 = min(max(math.floor((uu + rr + B - 1) / B), 0), Tx)
        y0 = min(max(math.floor((vv - rr) / B), 0), Ty)
        y1 = min(max(math.floor((vv + rr + B - 1) / B), 0), Ty)
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                expect.setdefault((s // n) * Tx * Ty + ty * Tx + tx, []).append(s)
    pos = 0
    for t in range(V * Tx * Ty):
        st, en = ranges[t]
        lst = sorted(expect.get(t, []), key=lambda s: (float(z[s]), s))
        assert st == pos                     # ranges are the exclusive scan of the counts
        assert list(vals[st:en]) == lst
        pos = en
    assert pos == len(vals)


def test_l1_loss_closed_form():
    sc = make_tiny_scene(seed=1, n=20, W=16, H=16, views=2, tile=8)
    pre = O.preprocess(sc.params, sc.n, 1, sc.cams, 16, 16, 8)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], 2, sc.n, 16, 16, 8)
    fw0 = O.render_fwd(rec, ranges, vals, 2, 16, 16, 8, sc.cams)
    rng = np.random.default_rng(0)
    d_img = rng.normal(0, 0.1, fw0["img"].shape)
    tgt_d = fw0["depth"] + rng.normal(0, 0.2, fw0["depth"].shape)
    tgt_d[:, :4] = 0.0                       # invalid depth rows are masked out
    fw = O.render_fwd(rec, ranges, vals, 2, 16, 16, 8, sc.cams, tgt_rgb=fw0["img"] - d_img,
                      tgt_depth=tgt_d, lambda_d=0.1)
    for v in range(2):
        m = tgt_d[v] > 0
        exp = np.abs(d_img[v]).mean() + 0.1 * np.abs(fw0["depth"][v][m] - tgt_d[v][m]).mean()
        assert fw["loss_view"][v] == pytest.approx(exp, rel=1e-12)
        assert fw["depth_count"][v] == m.sum()


def test_render_pixels_matches_full_render():
    sc = make_scene(1, n=500)
    pre = O.preprocess(sc.params, sc.n, 0, sc.cams, 160, 120, 16)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], 1, sc.n, 160, 120, 16)
    fw = O.render_fwd(rec, ranges, vals, 1, 160, 120, 16, sc.cams, bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(0)
    pix = np.stack([np.zeros(50, int), rng.integers(0, 160, 50), rng.integers(0, 120, 50)], 1)
    px = O.render_pixels(rec, ranges, vals, 160, 120, 16, pix, bg=(0.1, 0.2, 0.3))
    np.testing.assert_array_equal(px["img"], fw["img"][0][:, pix[:, 2], pix[:, 1]].T)
    np.testing.assert_array_equal(px["T"], fw["T"][0][pix[:, 2], pix[:, 1]])
    np.testing.assert_array_equal(px["last"], fw["last"][0][pix[:, 2], pix[:, 1]])


def test_oracle_results_do_not_depend_on_thread_count():
    # the C oracle's parallel loops write disjoint outputs and add per-row sums in order
    sc = make_tiny_scene(seed=5, n=200, sh_degree=3, W=61, H=45, views=3, tile=8)
    pre = O.preprocess(sc.params_target, sc.n, 3, sc.cams, sc.width, sc.height, sc.tile)
    ranges, vals = O.bin_records(pre["rec"], pre["radius"], 3, sc.n, sc.width, sc.height, sc.tile)
    tgt = O.render_fwd(pre["rec"], ranges, vals, 3, sc.width, sc.height, sc.tile, sc.cams)
    saved = O.get_threads()
    runs = []
    try:
        for k in (1, 4):
            O.set_threads(k)
            runs.append(O.iteration(sc.params, sc.n, 3, sc.cams, sc.width, sc.height, sc.tile, tgt["img"],
                                    tgt["depth"], tol=1e-5))
    finally:
        O.set_threads(saved)
    a, b = runs
    assert np.array_equal(a["vals"], b["vals"]) and np.array_equal(a["ranges"], b["ranges"])
    for k in ("img", "depth", "T", "last", "loss_view", "near"):
        assert np.array_equal(a["fwd"][k], b["fwd"][k]), k
    assert np.array_equal(a["slot_grads"], b["slot_grads"]) and np.array_equal(a["grads"], b["grads"])
