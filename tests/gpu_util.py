"""Helpers for the GPU parity tests: layout conversion between the oracle's float64
records and the library's 12-float records, scene set-up and comparisons."""
import numpy as np
import pytest

from oracle import oracle as O

# oracle record field k (u, v, A, B, C, o, r, g, b, z) -> library record index
GPU_IDX = [0, 1, 2, 3, 4, 5, 8, 9, 10, 6]

# Tolerances (stated by the task's target: max abs pixel error 1e-4, gradient
# relative error 1e-3 against the FP64 oracle).
PIX_TOL = 1e-4
GRAD_REL_TOL = 1e-3
# Rounding allowance of a float32 evaluation, per unit of a term's operand magnitude (the
# oracle's grads_mag): 2^11 roundings of 2^-24, the transmittance and colour-behind
# recursions of a pixel over up to 2048 blended splats with one rounding each.  Where the
# blend's derivative cancels (a splat's colour close to the colour behind it), the exact
# value is small but float32 rounds against the operands' size.
F32_COND = 2.0 ** -13


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


_built = False


def native():
    global _built
    torch_cuda()
    from paper_2410_00486_gb300 import build as B
    if not _built:
        B.build()
        _built = True
    from paper_2410_00486_gb300 import _native as N
    N.lib()
    return N


def rec_to_gpu(rec10, radius, tau=None):
    """Library records (12 floats: u, v, A, B | C, o, z, radius | r, g, b, tau) from oracle
    records; tau = -ln(255 o) rounded to float32 (O.tau32) unless given."""
    import torch
    m = rec10.shape[0]
    a = np.zeros((m, 12), np.float32)
    a[:, GPU_IDX] = rec10.astype(np.float32)
    a[:, 7] = np.ascontiguousarray(radius, np.int32).view(np.float32)
    a[:, 11] = O.tau32(a[:, 5]) if tau is None else np.asarray(tau, np.float32)
    return torch.from_numpy(a.reshape(-1)).cuda()


def rec_from_gpu(t):
    """(oracle-order records [m, 10] in float64, radius int32 [m], tau float32 [m])."""
    a = t.detach().cpu().numpy().reshape(-1, 12)
    rec10 = a[:, GPU_IDX].astype(np.float64)
    radius = np.ascontiguousarray(a[:, 7]).view(np.int32).copy()
    return rec10, radius, a[:, 11].copy()


def sg_from_gpu(t):
    a = t.detach().cpu().numpy().reshape(-1, 12)
    return a[:, GPU_IDX].astype(np.float64)


def sg_to_gpu(sg10):
    import torch
    a = np.zeros((sg10.shape[0], 12), np.float32)
    a[:, GPU_IDX] = sg10.astype(np.float32)
    return torch.from_numpy(a.reshape(-1)).cuda()


def round32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def oracle_targets(sc, noise_rgb=0.02, noise_d=0.05, seed=11):
    """Targets rendered by the oracle from the perturbed copy, plus noise; the top
    eighth of each depth map is invalid (zero)."""
    pre = O.preprocess(sc.params_target, sc.n, sc.sh_degree, sc.cams, sc.width, sc.height, sc.tile)
    rec = pre["rec"]
    ranges, vals = O.bin_lists(rec[:, 0], rec[:, 1], rec[:, 9], pre["radius"], sc.views, sc.n,
                               sc.width, sc.height, sc.tile)
    fw = O.render_fwd(rec, ranges, vals, sc.views, sc.width, sc.height, sc.tile, sc.cams)
    rng = np.random.default_rng(seed)
    tgt_rgb = (fw["img"] + rng.normal(0, noise_rgb, fw["img"].shape)).astype(np.float32)
    tgt_d = (fw["depth"] + rng.normal(0, noise_d, fw["depth"].shape)).astype(np.float32)
    tgt_d[:, : max(1, sc.height // 8)] = 0.0
    return tgt_rgb, tgt_d


def rel_l2(a, b):
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    nb = np.linalg.norm(np.asarray(b))
    return d / nb if nb > 0 else d


def group_slices(n, deg):
    K = (deg + 1) ** 2
    sizes = [("means", 3 * n), ("log_scales", 3 * n), ("quats", 4 * n), ("opacity", n),
             ("sh_dc", 3 * n), ("sh_rest", 3 * (K - 1) * n)]
    out, o = {}, 0
    for name, s in sizes:
        if s:
            out[name] = slice(o, o + s)
        o += s
    return out


# ------------------------------------------------- tile lists: culled vs rect

def entry_tiles(ranges):
    """Global tile of every list entry, for contiguous ranges [T, 2] (entry 0 at ranges[0, 0])."""
    rg = np.asarray(ranges, np.int64).reshape(-1, 2)
    return np.repeat(np.arange(rg.shape[0], dtype=np.int64), rg[:, 1] - rg[:, 0])


def max_alpha_over_tiles(rec12, slots, tiles, W, H, B, chunk=32768):
    """For each (slot, tile) pair the largest alpha = min(0.99, o exp(power)) over the tile's
    pixel centres (pixels outside the image excluded; power > 0 counts as skipped, alpha 0),
    in float64 from the pair's float32 record (u, v, A, B, C, o): the blend's definition
    evaluated at every pixel, nothing else."""
    Tx = (W + B - 1) // B
    Tv = Tx * ((H + B - 1) // B)
    out = np.zeros(len(slots))
    off = np.arange(B, dtype=np.float64)
    for a in range(0, len(slots), chunk):
        s = np.asarray(slots[a:a + chunk], np.int64)
        t = np.asarray(tiles[a:a + chunk], np.int64) % Tv
        r = rec12[s].astype(np.float64)
        u, v, A, Bc, C, o = (r[:, k] for k in range(6))
        px = (t % Tx)[:, None] * B + off[None, :]                 # [m, B]
        py = (t // Tx)[:, None] * B + off[None, :]
        dx = u[:, None] - px
        dy = v[:, None] - py
        power = (-0.5 * (A[:, None, None] * (dx * dx)[:, None, :] + C[:, None, None] * (dy * dy)[:, :, None])
                 - Bc[:, None, None] * dy[:, :, None] * dx[:, None, :])          # [m, y, x]
        alpha = np.minimum(0.99, o[:, None, None] * np.exp(np.minimum(power, 0.0)))
        inside = (py < H)[:, :, None] & (px < W)[:, None, :] & (power <= 0.0)
        out[a:a + chunk] = np.where(inside, alpha, 0.0).max(axis=(1, 2))
    return out


def check_culled_lists(rec12, ranges_rect, vals_rect, ranges_cull, vals_cull, W, H, B, slot_base=0):
    """The culled lists against the rect lists of the same records: (i) each tile's culled
    list is an ordered subsequence of its rect list (same (depth, slot) order); (ii) every
    (slot, tile) pair the culling dropped has alpha < 1/255 at every pixel centre of the
    tile, evaluated in float64 by brute force, so no pixel would have blended it.  The
    ranges cover the same tiles; slot_base is subtracted from the culled ids (a view's ids
    when the culled lists come from a whole window).  Returns (rect, kept, dropped) counts."""
    rr = np.asarray(ranges_rect, np.int64).reshape(-1, 2)
    rc = np.asarray(ranges_cull, np.int64).reshape(-1, 2)
    assert rr.shape == rc.shape
    rc = rc - rc[0, 0]
    rr = rr - rr[0, 0]
    vr = np.asarray(vals_rect, np.int64)
    vc = np.asarray(vals_cull, np.int64) - slot_base
    assert len(vr) == rr[-1, 1] and len(vc) == rc[-1, 1]
    S = int(max(vr.max(initial=0), vc.max(initial=0))) + 1
    key_r = entry_tiles(rr) * S + vr
    key_c = entry_tiles(rc) * S + vc
    order = np.argsort(key_r, kind="stable")
    srt = key_r[order]
    idx = np.minimum(np.searchsorted(srt, key_c), max(len(srt) - 1, 0))
    assert len(key_c) == 0 or np.all(srt[idx] == key_c), "a culled entry is not in its tile's rect list"
    pos = order[idx]
    assert np.all(np.diff(pos) > 0), "culled lists are not ordered subsequences of the rect lists"
    dropped = np.ones(len(vr), bool)
    dropped[pos] = False
    amax = max_alpha_over_tiles(rec12, vr[dropped], entry_tiles(rr)[dropped], W, H, B)
    bad = amax >= 1.0 / 255.0
    assert not bad.any(), f"{bad.sum()} dropped pairs reach alpha >= 1/255 (max {amax.max():.6g})"
    return len(vr), len(vc), int(dropped.sum())


def last_slots(last, ranges, vals, W, H, B):
    """The slot of each pixel's last blended splat (-1 where none): the list position `last`
    (1-based) mapped through the pixel's tile list, which identifies the splat whatever the
    list's other entries."""
    last = np.asarray(last).view(np.uint32).astype(np.int64)
    V = last.shape[0]
    Tx, Ty = (W + B - 1) // B, (H + B - 1) // B
    ys, xs = np.mgrid[0:H, 0:W]
    tile = (np.arange(V)[:, None, None] * (Tx * Ty) + (ys // B) * Tx + xs // B)
    rg = np.asarray(ranges, np.int64).reshape(-1, 2)
    vals = np.asarray(vals, np.int64)
    pos = rg[tile, 0] + last - 1
    return np.where(last > 0, vals[np.clip(pos, 0, max(len(vals) - 1, 0))], -1)


# ------------------------------------------------------- gradient comparisons

def grad_check(got, ref, explained=None, name="", rel=GRAD_REL_TOL, l2=None, mag=None):
    """Gradient parity: relative L2 error <= rel over the whole array, and per element
    |got - ref| <= rel (|ref| + rel max|ref|) [+ F32_COND mag, when the oracle's operand
    magnitudes `mag` of each element are given].  Rows (slots or Gaussians) in `explained`
    (bool per row) are where the oracle found a decision input near its threshold, so float32
    and float64 may take a different branch there: elements of those rows may exceed the
    per-element bound and are counted; any other element beyond it fails.  Returns
    (relative L2 error, elements beyond the bound, of which explained).  l2 (default rel)
    is the bound on the relative L2 error."""
    g = np.asarray(got, np.float64)
    r = np.asarray(ref, np.float64)
    e = rel_l2(g, r)
    scale = np.abs(r).max() if r.size else 0.0
    bound = rel * (np.abs(r) + rel * scale)
    if mag is not None:
        bound = bound + F32_COND * np.asarray(mag, np.float64).reshape(bound.shape)
    bad = np.abs(g - r) > bound
    if bad.ndim == 1:
        bad = bad[:, None]
    rows = bad.any(axis=1)
    expl = rows & explained if explained is not None else np.zeros_like(rows)
    unexpl = rows & ~expl
    print(f"    [{name}] rel L2 {e:.1e}  elements beyond the per-element bound: {int(bad.sum())} "
          f"({int(bad[expl].sum())} in rows near a threshold)")
    g2, r2 = g.reshape(bad.shape), r.reshape(bad.shape)
    for i, j in list(zip(*np.nonzero(bad & unexpl[:, None])))[:6]:
        b2 = np.asarray(bound).reshape(bad.shape)
        extra = f" mag {np.asarray(mag).reshape(bad.shape)[i, j]:.2e}" if mag is not None else ""
        print(f"      row {i} col {j}: got {g2[i, j]:.6e} ref {r2[i, j]:.6e} |d| {abs(g2[i, j] - r2[i, j]):.2e} "
              f"bound {b2[i, j]:.2e} max|ref| {scale:.2e}{extra}")
    assert e < (rel if l2 is None else l2), (name, e)
    assert not unexpl.any(), (name, f"{int(bad[unexpl].sum())} elements beyond the per-element bound, "
                                    f"e.g. rows {np.nonzero(unexpl)[0][:5]}")
    return e, int(bad.sum()), int(bad[expl].sum())


def residual_sign_flags(img, tgt_rgb, depth=None, tgt_depth=None, eps=1e-5):
    """Pixels whose L1 residual in some channel (or in depth, where the target depth is valid)
    lies within eps of 0: the sign the loss's derivative takes there is a decision that a
    rounding-sized difference in the render can flip."""
    f = (np.abs(np.asarray(img) - np.asarray(tgt_rgb)) < eps).any(axis=1)
    if depth is not None and tgt_depth is not None:
        td = np.asarray(tgt_depth)
        dscale = max(1.0, float(np.abs(td).max()))
        f |= (td > 0) & (np.abs(np.asarray(depth) - td) < eps * dscale)
    return f


def slots_in_flagged_tiles(near, ranges, vals, W, H, B, m, reach_px=0):
    """bool[m]: slots listed in a tile that holds a pixel the oracle flagged as near a
    decision threshold (their gradients may take the other branch in float32), or a pixel
    within reach_px of one (a loss that couples neighbouring pixels, like SSIM's window)."""
    near = np.asarray(near) != 0
    if reach_px > 0:
        from scipy.ndimage import maximum_filter
        near = maximum_filter(near, size=(1, 2 * reach_px + 1, 2 * reach_px + 1))
    V = near.shape[0]
    Tx, Ty = (W + B - 1) // B, (H + B - 1) // B
    vv, ys, xs = np.nonzero(near)
    tiles = np.unique(vv * (Tx * Ty) + (ys // B) * Tx + xs // B)
    rg = np.asarray(ranges, np.int64).reshape(-1, 2)
    out = np.zeros(m, bool)
    for t in tiles:
        out[np.asarray(vals[rg[t, 0]:rg[t, 1]], np.int64)] = True
    return out


def param_grad_check(got, ref, n, deg, explained=None, tag="", rel=GRAD_REL_TOL, l2=None, checks=None):
    """grad_check per parameter group of the flat parameter vector, rows = Gaussians
    (explained: bool per Gaussian)."""
    out = {}
    for name, sl in group_slices(n, deg).items():
        w = (sl.stop - sl.start) // n
        try:
            out[name] = grad_check(np.asarray(got)[sl].reshape(n, w), np.asarray(ref)[sl].reshape(n, w), explained,
                                   f"{tag} {name}", rel, l2)
        except AssertionError as err:
            if checks is None:
                raise
            checks.append(err)
    return out


def field_grad_check(got, ref, explained=None, tag="", mag=None, rel=GRAD_REL_TOL, l2=None):
    """grad_check on each of the ten slot-gradient fields (columns); every field is checked
    (and printed) before the first failure is raised."""
    errs = []
    for k, f in enumerate(["u", "v", "A", "B", "C", "o", "r", "g", "b", "z"]):
        try:
            grad_check(got[:, k], ref[:, k], explained, f"{tag} {f}", rel, l2,
                       None if mag is None else mag[:, k])
        except AssertionError as err:
            errs.append(err)
    if errs:
        raise errs[0]


def gaussians_of_slots(slot_mask, n):
    """bool per Gaussian: any of its slots (v n + g) set."""
    m = np.asarray(slot_mask, bool)
    return m.reshape(-1, n).any(axis=0)


def from_params_explained(sc, it, gpu_img, gpu_slot_grad, reach_px=0, tol=1e-3):
    """Gaussians whose gradients a float32 iteration from the same parameters may legitimately
    take elsewhere than the float64 oracle's iteration `it`:
      - a slot listed in a tile holding a pixel whose decision inputs lie within a relative
        `tol` of a threshold (1e-3: the float32 projection upstream moves the records by about
        that much more than the blend's own rounding), or a pixel whose value differs by more
        than the pixel tolerance, or within reach_px of one;
      - a slot whose projection is fragile (its tile rectangle or visibility may differ);
      - a slot whose gradient differs from the oracle's by more than the per-element bound
        but within the float32 rounding allowance of its terms (F32_COND x operand
        magnitudes from the oracle), which the chain rule then carries to the parameters.
    Returns (bool per Gaussian, dict of counts)."""
    V, n, W, H, B = sc.views, sc.n, sc.width, sc.height, sc.tile
    rec, ranges, vals = it["pre"]["rec"], it["ranges"], it["vals"]
    fw = O.render_fwd(rec, ranges, vals, V, W, H, B, sc.cams, tol=tol)
    flag = (fw["near"] != 0) | (np.abs(np.asarray(gpu_img) - it["fwd"]["img"]).max(1) > PIX_TOL)
    if it["dl_dimg"] is None:        # the L1 loss: the residual's sign is a decision
        flag |= residual_sign_flags(it["fwd"]["img"], it["tgt_rgb"], it["fwd"]["depth"], it["tgt_depth"])
    near = slots_in_flagged_tiles(flag, ranges, vals, W, H, B, V * n, reach_px)
    _, mag = O.render_bwd(rec, ranges, vals, V, n, W, H, B, sc.cams, it["fwd"]["img"], it["fwd"]["depth"],
                          it["tgt_rgb"], it["tgt_depth"], it["fwd"]["depth_count"], dl_dimg=it["dl_dimg"],
                          dl_ddepth=it["dl_ddepth"], with_abs=True)
    sg = np.asarray(gpu_slot_grad, np.float64)
    ref = it["slot_grads"]
    scale = np.abs(ref).max(axis=0, keepdims=True)
    plain = GRAD_REL_TOL * (np.abs(ref) + GRAD_REL_TOL * scale)
    d = np.abs(sg - ref)
    cond = ((d > plain) & (d <= plain + F32_COND * mag)).any(axis=1)
    fragile = it["pre"]["fragile"] > 0
    expl = gaussians_of_slots(near | fragile | cond, n)
    counts = {"flagged_px": float(flag.mean()), "near_slots": int(near.sum()), "fragile_slots": int(fragile.sum()),
              "conditioned_slots": int(cond.sum()), "gaussians": int(expl.sum())}
    return expl, counts


def check_iteration_against_oracle(sc, win, it, tag, reach_px=0, grads=None):
    """A GPU window iteration from the same parameters as the oracle's iteration `it`: pixels
    within PIX_TOL except where a decision input lies within a relative 1e-3 of its
    threshold (those are counted, and fewer than 1e-4 of all pixels may actually differ by
    more), per-view losses within 1e-4, parameter gradients by param_grad_check with the rows
    from_params_explained gives.  `grads` overrides the window's gradient (autograd)."""
    img = win.img.cpu().numpy()
    expl, counts = from_params_explained(sc, it, img, sg_from_gpu(win.slot_grad), reach_px)
    err = np.abs(img - it["fwd"]["img"]).max(1)
    ok = ~(O.render_fwd(it["pre"]["rec"], it["ranges"], it["vals"], sc.views, sc.width, sc.height, sc.tile,
                        sc.cams, tol=1e-3)["near"] != 0)
    dscale = max(1.0, np.abs(it["fwd"]["depth"]).max())
    e_d = (np.abs(win.depth.cpu().numpy() - it["fwd"]["depth"])[ok] / dscale).max()
    print(f"[{tag}] pixels near a threshold {1 - ok.mean():.2e}, beyond {PIX_TOL:g}: {(err > PIX_TOL).mean():.2e}, "
          f"max|dimg| elsewhere {err[ok].max():.2e}, |ddepth|/scale {e_d:.2e}; explained Gaussians {counts}")
    assert err[ok].max() < PIX_TOL and e_d < PIX_TOL
    assert (err > PIX_TOL).mean() < 1e-4
    np.testing.assert_allclose(win.loss_view.cpu().numpy(), it["loss_view"], rtol=1e-4)
    g = (win.grads if grads is None else grads).detach().cpu().numpy().astype(np.float64)
    return param_grad_check(g, it["grads"], sc.n, sc.sh_degree, expl, tag)
