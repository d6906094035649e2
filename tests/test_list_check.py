"""The list and gradient checkers the GPU parity tests rely on, pinned on the CPU: the
float64 alpha brute force against a pure-Python loop, and planted mistakes in a culled list
(a dropped pair that blends, two entries swapped, an entry outside the rect) each caught."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synth import make_conics, make_records
from tests.gpu_util import check_culled_lists, entry_tiles, grad_check, last_slots, max_alpha_over_tiles


def records(seed=3, V=2, n=400, W=90, H=70, B=16):
    u, v, r, z = make_records(seed, V, n, W, H, max_radius=30)
    conic, opac = make_conics(seed + 1, r)
    rec12 = np.zeros((V * n, 12), np.float32)
    rec12[:, 0], rec12[:, 1], rec12[:, 2:5], rec12[:, 5], rec12[:, 6] = u, v, conic, opac, z
    ranges, vals = O.bin_lists(rec12[:, 0], rec12[:, 1], rec12[:, 6], r, V, n, W, H, B)
    return rec12, ranges, vals, (V, n, W, H, B)


def test_max_alpha_matches_python_loop():
    rec12, ranges, vals, (V, n, W, H, B) = records()
    tiles = entry_tiles(ranges)
    pick = np.random.default_rng(0).choice(len(vals), 60, replace=False)
    got = max_alpha_over_tiles(rec12, vals[pick], tiles[pick], W, H, B)
    Tx, Ty = (W + B - 1) // B, (H + B - 1) // B
    for k, i in enumerate(pick):
        u, v, A, Bc, C, o = (float(x) for x in rec12[vals[i], :6])
        t = int(tiles[i]) % (Tx * Ty)
        best = 0.0
        for y in range((t // Tx) * B, min((t // Tx) * B + B, H)):
            for x in range((t % Tx) * B, min((t % Tx) * B + B, W)):
                dx, dy = u - x, v - y
                p = -0.5 * (A * dx * dx + C * dy * dy) - Bc * dx * dy
                if p <= 0.0:
                    best = max(best, min(0.99, o * math.exp(p)))
        assert got[k] == pytest.approx(best, rel=1e-12, abs=0)


def valid_culled(rec12, ranges, vals, W, H, B):
    """Drop exactly the rect entries that reach alpha >= 1/255 nowhere in their tile."""
    tiles = entry_tiles(ranges)
    keep = max_alpha_over_tiles(rec12, vals, tiles, W, H, B) >= 1.0 / 255.0
    counts = np.bincount(tiles[keep], minlength=len(ranges))
    ends = np.cumsum(counts)
    return np.stack([ends - counts, ends], 1).astype(np.uint32), vals[keep], keep


def test_culled_list_checker_accepts_a_valid_cull_and_catches_planted_mistakes():
    rec12, ranges, vals, (V, n, W, H, B) = records()
    rc, vc, keep = valid_culled(rec12, ranges, vals, W, H, B)
    tot, kept, dropped = check_culled_lists(rec12, ranges, vals, rc, vc, W, H, B)
    assert dropped == (~keep).sum() > 0 and kept == keep.sum()
    # a pair that does blend somewhere in its tile, left out
    i = np.nonzero(keep)[0][10]
    keep2 = keep.copy()
    keep2[i] = False
    tiles = entry_tiles(ranges)
    counts = np.bincount(tiles[keep2], minlength=len(ranges))
    ends = np.cumsum(counts)
    with pytest.raises(AssertionError):
        check_culled_lists(rec12, ranges, vals, np.stack([ends - counts, ends], 1), vals[keep2], W, H, B)
    # two entries of one tile swapped
    lens = rc[:, 1] - rc[:, 0]
    t = int(np.nonzero(lens >= 2)[0][0])
    bad = vc.copy()
    bad[rc[t, 0]], bad[rc[t, 0] + 1] = bad[rc[t, 0] + 1], bad[rc[t, 0]]
    with pytest.raises(AssertionError):
        check_culled_lists(rec12, ranges, vals, rc, bad, W, H, B)
    # an entry whose slot is not in that tile's rect list
    bad = vc.copy()
    others = np.setdiff1d(np.arange(V * n), vals[ranges[t, 0]:ranges[t, 1]])
    bad[rc[t, 0]] = others[0]
    with pytest.raises(AssertionError):
        check_culled_lists(rec12, ranges, vals, rc, bad, W, H, B)


def test_last_slots_maps_positions_through_lists():
    W = H = B = 2                         # one 2x2 tile per view, two views
    ranges = np.array([[0, 3], [3, 5]], np.uint32)
    vals = np.array([7, 4, 9, 2, 8], np.uint32)
    last = np.array([[[0, 1], [3, 2]], [[2, 1], [0, 0]]], np.uint32)
    got = last_slots(last, ranges, vals, W, H, B)
    assert np.array_equal(got, [[[-1, 7], [9, 4]], [[8, 2], [-1, -1]]])


def test_grad_check_counts_explained_rows_and_fails_on_others():
    rng = np.random.default_rng(1)
    ref = rng.normal(size=(500, 3))
    got = ref * (1 + 1e-6 * rng.normal(size=ref.shape))
    got[17, 1] += 0.1                        # one element far off, in row 17
    expl = np.zeros(500, bool)
    expl[17] = True
    _, nbad, nexpl = grad_check(got, ref, expl, "planted", l2=1.0)
    assert nbad == nexpl == 1
    with pytest.raises(AssertionError):
        grad_check(got, ref, None, "planted", l2=1.0)
