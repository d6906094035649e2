"""Python face of the FP64 CPU oracle (CaRtGS, arXiv 2410.00486).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only users.  The library path never imports this module.

The render, gradient and statistics steps call the plain C implementation in
cgs_oracle.c (double precision, one pixel / one Gaussian at a time).  Adam, the
opacity regulariser and the adaptive keyframe scheduler are written here in
numpy / plain Python, step by step from the paper:

  * opacity regularisation, Eqs. 10-11 (Sec. III-C.3)
  * Adam with the 3DGS hyper-parameters the paper keeps (Sec. IV-A)
  * adaptive optimisation scheduler, Eqs. 5-8 (Sec. III-C.2)
  * adaptive density control (clone / split / prune, Sec. III-A.3, IV-A)
  * the SSIM term and the full loss of Eq. 9 (Sec. III-C.3)
  * geometric densification: point cloud -> initial Gaussians (Sec. III-A.3, III-B),
    with the exact k-nearest-neighbour distances computed in C by brute force

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, invariants, finite differences, scipy's spherical harmonics,
torch.optim.Adam, brute-force enumeration); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "cgs_oracle.c"
_SO = _HERE / "_build" / "liboracle.so"

NREC = 10
NCAM = 17
REC_FIELDS = ("u", "v", "conA", "conB", "conC", "opacity", "r", "g", "b", "depth")

_lib = None


def build(force: bool = False) -> Path:
    """Compile the C oracle with gcc (no FMA contraction, so each formula rounds as written)."""
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        _SO.parent.mkdir(parents=True, exist_ok=True)
        tmp = _SO.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                        "-o", str(tmp), str(_SRC), "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_SO))
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.orc_preprocess.argtypes = [P, i64, i32, P, i32, i32, i32, i32, f64, f64, P, P, P, P, P]
        lib.orc_set_threads.argtypes = [i32]
        lib.orc_set_threads.restype = None
        lib.orc_get_threads.restype = i32
        lib.orc_bin.argtypes = [P, P, P, P, i32, i64, i32, i32, i32, i64, P, P]
        lib.orc_bin.restype = i64
        lib.orc_render_fwd.argtypes = [P, P, P, i32, i32, i32, i32, P, P, P, P, f64, f64,
                                       P, P, P, P, P, P, P, P]
        lib.orc_render_bwd.argtypes = [P, P, P, i32, i64, i32, i32, i32, P, P, P, P, P, P, P,
                                       f64, P, P, P, P]
        lib.orc_preprocess_bwd.argtypes = [P, i64, i32, P, i32, i32, i32, i32, f64, P, P]
        lib.orc_densify_stats.argtypes = [P, P, i32, i64, i32, i32, P, P, P]
        lib.orc_sh_basis.argtypes = [i32, f64, f64, f64, P, P]
        lib.orc_knn_mean_d2.argtypes = [P, i64, i32, P]
        lib.orc_knn_mean_d2_at.argtypes = [P, i64, i32, P, i64, P]
        lib.orc_render_pixels.argtypes = [P, P, P, i32, i32, i32, P, P, i64, f64, P, P, P, P, P]
        _lib = lib
    return _lib


def set_threads(k: int) -> int:
    """Threads of the C oracle's parallel loops (results do not depend on it); returns the
    count now in effect."""
    lib = _load()
    lib.orc_set_threads(int(k))
    return int(lib.orc_get_threads())


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def cams_to_oracle(cams: np.ndarray) -> np.ndarray:
    """float32[V][20] camera rows -> double[V][17] (R, t, fx, fy, cx, cy, weight)."""
    cams = np.asarray(cams)
    return _f64(cams[:, :17])


def sh_basis(deg: int, d) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib.orc_sh_basis(deg, float(d[0]), float(d[1]), float(d[2]), _p(Y), _p(dY))
    return Y, dY.reshape(16, 3)


def preprocess(params, n, deg, cams, W, H, B, near=0.2, tol_px=5e-4) -> dict:
    lib = _load()
    P = _f64(params)
    C = cams_to_oracle(cams)
    V = C.shape[0]
    m = V * n
    out = dict(rec=np.zeros((m, NREC)), radius=np.zeros(m, np.int32),
               rect=np.zeros((m, 4), np.int32), clamp=np.zeros(m, np.int32),
               fragile=np.zeros(m, np.int32))
    lib.orc_preprocess(_p(P), n, deg, _p(C), V, W, H, B, near, tol_px, _p(out["rec"]),
                       _p(out["radius"]), _p(out["rect"]), _p(out["clamp"]), _p(out["fragile"]))
    return out


def tiles(W, H, B):
    return (W + B - 1) // B, (H + B - 1) // B


def tau32(opacity) -> np.ndarray:
    """tau = -ln(255 o) of each splat, rounded to float32: the field of the library's
    12-float record that the tests fill when they hand oracle records to the kernels."""
    with np.errstate(divide="ignore"):
        return (-np.log(255.0 * np.asarray(opacity, np.float64))).astype(np.float32)


def bin_lists(u, v, z, radius, V, n, W, H, B):
    """Tile lists: every visible slot in every tile of its rect, ordered by (tile, depth,
    slot): returns (ranges[Ttot, 2], vals[count])."""
    lib = _load()
    Tx, Ty = tiles(W, H, B)
    Ttot = V * Tx * Ty
    u, v, z = _f64(u), _f64(v), _f64(z)
    radius = np.ascontiguousarray(radius, np.int32)
    ranges = np.zeros((Ttot, 2), np.uint32)
    args = (_p(u), _p(v), _p(z), _p(radius))
    cnt = lib.orc_bin(*args, V, n, W, H, B, 0, _p(ranges), None)
    vals = np.zeros(max(1, cnt), np.uint32)
    cnt2 = lib.orc_bin(*args, V, n, W, H, B, vals.size, _p(ranges), _p(vals))
    assert cnt2 == cnt
    return ranges, vals[:cnt]


def bin_records(rec, radius, V, n, W, H, B):
    """bin_lists for oracle records [m, 10] (u, v, A, B, C, o, r, g, b, z)."""
    r = np.asarray(rec, np.float64)
    return bin_lists(r[:, 0], r[:, 1], r[:, 9], radius, V, n, W, H, B)


def render_fwd(rec, ranges, vals, V, W, H, B, cams, bg=(0.0, 0.0, 0.0), tgt_rgb=None,
               tgt_depth=None, lambda_d=0.1, tol=0.0, want_hash=False) -> dict:
    lib = _load()
    rec = _f64(rec)
    C = cams_to_oracle(cams)
    bgv = _f64(bg)
    HW = H * W
    out = dict(img=np.zeros((V, 3, H, W)), depth=np.zeros((V, H, W)), T=np.zeros((V, H, W)),
               last=np.zeros((V, H, W), np.uint32), loss_view=np.zeros(V),
               depth_count=np.zeros(V, np.int64), near=np.zeros((V, H, W), np.int32))
    h = np.zeros(1, np.uint64)
    tr = _f64(tgt_rgb) if tgt_rgb is not None else None
    td = _f64(tgt_depth) if tgt_depth is not None else None
    lib.orc_render_fwd(_p(rec), _p(np.ascontiguousarray(ranges, np.uint32)),
                       _p(np.ascontiguousarray(vals, np.uint32)), V, W, H, B, _p(bgv), _p(C),
                       _p(tr) if tr is not None else None, _p(td) if td is not None else None,
                       lambda_d, tol, _p(out["img"]), _p(out["depth"]), _p(out["T"]),
                       _p(out["last"]), _p(out["loss_view"]), _p(out["depth_count"]),
                       _p(out["near"]), _p(h) if want_hash else None)
    del HW
    if want_hash:
        out["hash"] = int(h[0])
    return out


def render_pixels(rec, ranges, vals, W, H, B, pix, bg=(0.0, 0.0, 0.0), tol=0.0) -> dict:
    """Forward blend of selected pixels only; pix is int[k][3] = (view, x, y)."""
    lib = _load()
    pix = np.ascontiguousarray(pix, np.int32)
    k = pix.shape[0]
    out = dict(img=np.zeros((k, 3)), depth=np.zeros(k), T=np.zeros(k), last=np.zeros(k, np.uint32),
               near=np.zeros(k, np.int32))
    lib.orc_render_pixels(_p(_f64(rec)), _p(np.ascontiguousarray(ranges, np.uint32)),
                          _p(np.ascontiguousarray(vals, np.uint32)), W, H, B, _p(_f64(bg)), _p(pix), k, tol,
                          _p(out["img"]), _p(out["depth"]), _p(out["T"]), _p(out["last"]), _p(out["near"]))
    return out


def render_bwd(rec, ranges, vals, V, n, W, H, B, cams, img, depth, tgt_rgb, tgt_depth,
               depth_count, bg=(0.0, 0.0, 0.0), lambda_d=0.1, dl_dimg=None, dl_ddepth=None,
               with_abs=False):
    """Slot gradients [V*n][10]; pixel gradients from the fused L1 loss, or dl_dimg
    [V,3,H,W] / dl_ddepth [V,H,W] (None: zero) when dl_dimg is given.  with_abs: also the
    per-field sums of the terms evaluated on their operands' magnitudes (the rounding scale
    of a float32 evaluation), returned as (grads, magnitudes)."""
    lib = _load()
    grads = np.zeros((V * n, NREC))
    gabs = np.zeros((V * n, NREC)) if with_abs else None
    td = _f64(tgt_depth) if tgt_depth is not None else None
    gi = _f64(dl_dimg) if dl_dimg is not None else None
    gd = _f64(dl_ddepth) if dl_ddepth is not None else None
    lib.orc_render_bwd(_p(_f64(rec)), _p(np.ascontiguousarray(ranges, np.uint32)),
                       _p(np.ascontiguousarray(vals, np.uint32)), V, n, W, H, B, _p(_f64(bg)),
                       _p(cams_to_oracle(cams)), _p(_f64(img)), _p(_f64(depth)), _p(_f64(tgt_rgb)),
                       _p(td) if td is not None else None,
                       _p(np.ascontiguousarray(depth_count, np.int64)), lambda_d,
                       _p(gi) if gi is not None else None, _p(gd) if gd is not None else None, _p(grads),
                       _p(gabs) if with_abs else None)
    return (grads, gabs) if with_abs else grads


def preprocess_bwd(params, n, deg, cams, W, H, B, slot_grads, near=0.2) -> np.ndarray:
    lib = _load()
    P = _f64(params)
    out = np.zeros_like(P)
    C = cams_to_oracle(cams)
    lib.orc_preprocess_bwd(_p(P), n, deg, _p(C), C.shape[0], W, H, B, near,
                           _p(_f64(slot_grads)), _p(out))
    return out


def densify_stats(slot_grads, radius, V, n, W, H, accum=None, denom=None, max_r2d=None):
    lib = _load()
    accum = np.zeros(n) if accum is None else _f64(accum).copy()
    denom = np.zeros(n) if denom is None else _f64(denom).copy()
    max_r2d = np.zeros(n) if max_r2d is None else _f64(max_r2d).copy()
    lib.orc_densify_stats(_p(_f64(slot_grads)), _p(np.ascontiguousarray(radius, np.int32)), V, n,
                          W, H, _p(accum), _p(denom), _p(max_r2d))
    return accum, denom, max_r2d


# --------------------------------------------------------------- loss pieces

def opacity_reg(params, n, lambda_o):
    """L_o = (1/N) sum_i |o_i| with o_i = sigmoid(opacity logit) > 0 (Eq. 10), weighted by
    lambda_o (Eq. 11).  Returns (lambda_o * L_o, gradient w.r.t. the logits)."""
    x = _f64(params)[10 * n: 11 * n]
    o = 1.0 / (1.0 + np.exp(-x))
    return lambda_o * o.sum() / n, lambda_o * o * (1.0 - o) / n


def adam(theta, grad, m, v, step, lr_per_elem, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step with bias correction (t starts at 1); every element is updated,
    including those with zero gradient (reading).  Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr_per_elem * mhat / (np.sqrt(vhat) + eps), m, v


def lr_per_element(n, deg, lr6):
    """Expand the six per-group learning rates to the flat parameter layout."""
    K = (deg + 1) ** 2
    sizes = [3 * n, 3 * n, 4 * n, n, 3 * n, 3 * (K - 1) * n]
    return np.concatenate([np.full(s, float(l)) for s, l in zip(sizes, lr6)])


def iteration(params, n, deg, cams, W, H, B, tgt_rgb, tgt_depth, bg=(0.0, 0.0, 0.0),
              lambda_d=0.1, lambda_o=0.0, near=0.2, tol=0.0, lambda_ssim=0.0) -> dict:
    """Loss and parameter gradient of one window iteration, plus every intermediate.
    lambda_ssim > 0 adds the SSIM term of Eq. 9 (photometric_loss); 0 keeps the L1 form."""
    V = np.asarray(cams).shape[0]
    pre = preprocess(params, n, deg, cams, W, H, B, near)
    rec = pre["rec"]
    ranges, vals = bin_records(rec, pre["radius"], V, n, W, H, B)
    fw = render_fwd(rec, ranges, vals, V, W, H, B, cams, bg, tgt_rgb, tgt_depth, lambda_d, tol)
    loss_view = fw["loss_view"]
    gi = gd = None
    if lambda_ssim > 0.0:
        loss_view, gi, gd = photometric_loss(fw["img"], fw["depth"], tgt_rgb, tgt_depth,
                                             np.asarray(cams)[:, 16], lambda_ssim, lambda_d)
    sg = render_bwd(rec, ranges, vals, V, n, W, H, B, cams, fw["img"], fw["depth"], tgt_rgb,
                    tgt_depth, fw["depth_count"], bg, lambda_d, gi, gd)
    grads = preprocess_bwd(params, n, deg, cams, W, H, B, sg, near)
    lo, glo = opacity_reg(params, n, lambda_o)
    grads[10 * n: 11 * n] += glo
    return dict(pre=pre, ranges=ranges, vals=vals, fwd=fw, slot_grads=sg, grads=grads, tgt_rgb=tgt_rgb,
                tgt_depth=tgt_depth, dl_dimg=gi, dl_ddepth=gd,
                loss_view=loss_view, loss=float(loss_view.sum() + lo), loss_o=lo)


# ------------------------------------------------------ adaptive scheduler

class Scheduler:
    """Adaptive keyframe selection, Eqs. 5-8 (Sec. III-C.2), step by step.

    Readings: a new keyframe's loss starts at +inf (it is never read before the
    keyframe is trained once, since r0 >= 1); d_k = max(1, floor(k / d)); ties in the
    top-d_k selection go to the lower index; a draw picks uniformly among keyframes
    with r_i > 0 using a caller-supplied uniform 32-bit integer (index = u mod count
    into the ascending list of eligible keyframes).
    """

    def __init__(self, d: int = 4):
        self.d = d
        self.K: list[int] = []       # keyframe ids (Eq. 5)
        self.R: list[int] = []       # remaining iterations (Eq. 6)
        self.L: list[float] = []     # last loss (Eq. 7)

    def add(self, keyframe_id: int, r0: int):
        self.K.append(keyframe_id)
        self.R.append(int(r0))
        self.L.append(float("inf"))

    def _refill(self):
        """Eq. 8: r_i = 2 for the d_k largest losses, 1 otherwise."""
        k = len(self.K)
        dk = max(1, k // self.d)
        order = sorted(range(k), key=lambda i: (-self.L[i], i))
        top = set(order[:dk])
        self.R = [2 if i in top else 1 for i in range(k)]

    def draw(self, rand_u32: int) -> int:
        """Pick a pool index with r > 0 (refilling first if none is left); r -= 1."""
        if not self.K:
            raise ValueError("empty keyframe pool")
        elig = [i for i, r in enumerate(self.R) if r > 0]
        if not elig:
            self._refill()
            elig = [i for i, r in enumerate(self.R) if r > 0]
        i = elig[int(rand_u32) % len(elig)]
        self.R[i] -= 1
        return i

    def report(self, index: int, loss: float):
        self.L[index] = float(loss)


# ------------------------------------------------------------ densification

SPLIT_CHILDREN = 2
SPLIT_SCALE_DIV = 1.6          # children's scale = parent's / (0.8 * 2), as in 3DGS


def densify_thresholds(tau_p, scale_thr, eps_alpha):
    """Float32 decision thresholds, computed in double and rounded once: the gradient
    threshold, log(scale threshold) and logit(eps_alpha)."""
    return (np.float32(tau_p), np.float32(np.log(scale_thr)), np.float32(np.log(eps_alpha / (1.0 - eps_alpha))))


def densify_plan(params, n, deg, accum, denom, tau_p, scale_thr, eps_alpha):
    """Adaptive density control of 3DGS with the paper's thresholds (Sec. III-A.3, IV-A:
    densify with positional-gradient threshold tau_p, remove Gaussians with opacity below
    eps_alpha).  Decisions are taken in float32 (the kernel's precision):
      grad = accum / denom (0 where denom = 0); high = grad >= tau_p;
      small = max_i log s_i <= log(scale_thr);  prune = opacity logit < logit(eps_alpha)
      clone = high & small & ~prune;  split = high & ~small & ~prune;  keep = ~prune & ~split
    Returns (code, count) with code 0 prune, 1 keep, 2 keep + clone, 3 split; count =
    outputs per Gaussian (0, 1, 2, 2)."""
    t_grad, t_logs, t_logit = densify_thresholds(tau_p, scale_thr, eps_alpha)
    P = np.asarray(params, np.float32)
    acc = np.asarray(accum, np.float32)
    den = np.asarray(denom, np.float32)
    with np.errstate(divide="ignore", invalid="ignore"):
        grad = np.where(den > 0, acc / np.where(den > 0, den, np.float32(1)), np.float32(0)).astype(np.float32)
    high = grad >= t_grad
    logs = P[3 * n: 6 * n].reshape(n, 3)
    small = logs.max(axis=1) <= t_logs
    prune = P[10 * n: 11 * n] < t_logit
    split = high & ~small & ~prune
    clone = high & small & ~prune
    code = np.where(prune, 0, np.where(split, 3, np.where(clone, 2, 1))).astype(np.int32)
    count = np.array([0, 1, 2, 2], np.int64)[code]
    return code, count


def densify_apply(params, m, v, n, deg, code, normals):
    """New parameter vector and Adam state after clone / split / prune, Gaussian by
    Gaussian in order (reading: each Gaussian's outputs are consecutive):
      keep  -> the Gaussian (with its Adam state)
      clone -> the Gaussian (with its state), then a copy (zero state)
      split -> two children: mean + R(q) (s * z_c) with z_c = normals[g, c] ~ N(0, I),
               scale s / 1.6, other attributes copied, zero state
      prune -> nothing.
    Returns (params_out, m_out, v_out, n_out) in the flat layout for n_out Gaussians."""
    K = (deg + 1) ** 2
    widths = [3, 3, 4, 1, 3, 3 * (K - 1)]
    offs = np.cumsum([0] + [w * n for w in widths])

    def groups(a, nn):
        o = np.cumsum([0] + [w * nn for w in widths])
        return [np.asarray(a[o[i]:o[i + 1]]).reshape(nn, widths[i]) for i in range(6)]

    Pg, Mg, Vg = groups(np.asarray(params, np.float64), n), groups(np.asarray(m, np.float64), n), \
        groups(np.asarray(v, np.float64), n)
    outP = [[] for _ in range(6)]
    outM = [[] for _ in range(6)]
    outV = [[] for _ in range(6)]
    zero = [np.zeros(w) for w in widths]
    for g in range(n):
        c = code[g]
        rows = []
        if c in (1, 2):
            rows.append(([Pg[i][g] for i in range(6)], [Mg[i][g] for i in range(6)], [Vg[i][g] for i in range(6)]))
        if c == 2:
            rows.append(([Pg[i][g] for i in range(6)], zero, zero))
        if c == 3:
            q = Pg[2][g] / np.linalg.norm(Pg[2][g])
            w_, x, y, z = q
            R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w_ * z), 2 * (x * z + w_ * y)],
                          [2 * (x * y + w_ * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w_ * x)],
                          [2 * (x * z - w_ * y), 2 * (y * z + w_ * x), 1 - 2 * (x * x + y * y)]])
            s = np.exp(Pg[1][g])
            for ci in range(SPLIT_CHILDREN):
                mean = Pg[0][g] + R @ (s * np.asarray(normals[g, ci], np.float64))
                logs = Pg[1][g] - np.log(SPLIT_SCALE_DIV)
                rows.append(([mean, logs] + [Pg[i][g] for i in range(2, 6)], zero, zero))
        for rp, rm, rv in rows:
            for i in range(6):
                outP[i].append(rp[i])
                outM[i].append(rm[i])
                outV[i].append(rv[i])
    n_out = len(outP[0])
    flat = lambda parts: np.concatenate([np.asarray(parts[i]).reshape(-1) for i in range(6)]) if n_out else \
        np.zeros(0)
    del offs
    return flat(outP), flat(outM), flat(outV), n_out


# ----------------------------------------------------------------- SSIM term

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_WIN = 11
SSIM_SIGMA = 1.5


def ssim_window():
    """Normalised 11-tap Gaussian (sigma 1.5); the 2-D window is its outer product."""
    x = np.arange(SSIM_WIN) - SSIM_WIN // 2
    g = np.exp(-(x * x) / (2.0 * SSIM_SIGMA ** 2))
    return g / g.sum()


def _blur(img):
    """Zero-padded 'same' correlation of each [H, W] plane with the 2-D window."""
    g = ssim_window()
    r = SSIM_WIN // 2
    H, W = img.shape[-2:]
    pad = np.zeros(img.shape[:-2] + (H + 2 * r, W + 2 * r))
    pad[..., r:r + H, r:r + W] = img
    tmp = np.zeros(img.shape[:-2] + (H + 2 * r, W))
    for k in range(SSIM_WIN):
        tmp += g[k] * pad[..., :, k:k + W]
    out = np.zeros(img.shape)
    for k in range(SSIM_WIN):
        out += g[k] * tmp[..., k:k + H, :]
    return out


def ssim_loss(img, tgt):
    """Structural-similarity term of Eq. 9 per view: L_ssim = 1 - mean over channels and pixels
    of SSIM, with mu, sigma^2, sigma_xy from the 11x11 Gaussian window (sigma 1.5, zero
    padding), C1 = 0.01^2, C2 = 0.03^2 (reading: the 3DGS loss the paper keeps).
    img, tgt: [V, 3, H, W].  Returns (loss[V], dloss/dimg [V, 3, H, W])."""
    x = np.asarray(img, np.float64)
    y = np.asarray(tgt, np.float64)
    mx, my = _blur(x), _blur(y)
    exx, eyy, exy = _blur(x * x), _blur(y * y), _blur(x * y)
    sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2
    B1, B2 = mx * mx + my * my + SSIM_C1, sx + sy + SSIM_C2
    S = (A1 * A2) / (B1 * B2)
    M = x.shape[1] * x.shape[2] * x.shape[3]
    loss = 1.0 - S.reshape(S.shape[0], -1).mean(axis=1)
    # dS/d(mx), dS/d(E[x^2]), dS/d(E[xy]) per pixel (E = window mean), then back through the
    # window: dL/dx = -(1/M) [ blur(a) + 2 x blur(b) + y blur(c) ]
    dS_dA1 = A2 / (B1 * B2)
    dS_dA2 = A1 / (B1 * B2)
    dS_dB1 = -S / B1
    dS_dB2 = -S / B2
    # A1 = 2 mx my + C1, A2 = 2 (exy - mx my) + C2, B1 = mx^2 + my^2 + C1, B2 = exx - mx^2 + eyy - my^2 + C2
    a = dS_dA1 * 2 * my + dS_dA2 * (-2 * my) + dS_dB1 * 2 * mx + dS_dB2 * (-2 * mx)
    b = dS_dB2
    c = dS_dA2 * 2
    grad = -(_blur(a) + 2 * x * _blur(b) + y * _blur(c)) / M
    return loss, grad


def photometric_loss(img, depth, tgt_rgb, tgt_depth, weight, lambda_ssim, lambda_d=0.1):
    """Per-view loss of Eq. 9 with the depth term: L_v = w_v [ (1 - l) L1 + l L_ssim +
    lambda_d mean over {tgt_depth > 0} of |D - D*| ], l = lambda_ssim, L1 the mean over
    channels and pixels of |img - tgt| (sign(0) = 0).  tgt_depth may be None (no depth
    term).  Returns (loss[V], dL/dimg [V,3,H,W], dL/ddepth [V,H,W])."""
    x = np.asarray(img, np.float64)
    y = np.asarray(tgt_rgb, np.float64)
    V = x.shape[0]
    w = np.asarray(weight, np.float64).reshape(V)
    M = x.shape[1] * x.shape[2] * x.shape[3]
    l1 = np.abs(x - y).reshape(V, -1).mean(axis=1)
    ls, gs = ssim_loss(x, y)
    loss = (1.0 - lambda_ssim) * l1 + lambda_ssim * ls
    g_img = (1.0 - lambda_ssim) * np.sign(x - y) / M + lambda_ssim * gs
    g_dep = np.zeros(x.shape[:1] + x.shape[2:])
    if tgt_depth is not None:
        D = np.asarray(depth, np.float64)
        Dt = np.asarray(tgt_depth, np.float64)
        mask = Dt > 0.0
        cnt = mask.reshape(V, -1).sum(axis=1)
        r = np.where(mask, D - Dt, 0.0)
        for v in range(V):
            if cnt[v] > 0:
                loss[v] += lambda_d * np.abs(r[v]).sum() / cnt[v]
                g_dep[v] = lambda_d * np.sign(r[v]) / cnt[v]
    return w * loss, w[:, None, None, None] * g_img, w[:, None, None] * g_dep


# ------------------------------------------------------- geometric densification

SH_C0 = 0.28209479177387814      # Y_0^0 = 1 / (2 sqrt(pi))
KNN_K = 3
KNN_FLOOR = 1e-7
INIT_OPACITY = 0.1


def knn_mean_d2(xyz, k=KNN_K) -> np.ndarray:
    """Mean squared distance of every point to its k nearest other points (brute force, C)."""
    lib = _load()
    x = _f64(xyz).reshape(-1, 3)
    out = np.zeros(x.shape[0])
    if lib.orc_knn_mean_d2(_p(x), x.shape[0], k, _p(out)) != 0:
        raise ValueError("k out of range")
    return out


def knn_mean_d2_at(xyz, idx, k=KNN_K) -> np.ndarray:
    """knn_mean_d2 for the listed point indices only (brute force over the whole cloud)."""
    lib = _load()
    x = _f64(xyz).reshape(-1, 3)
    ii = np.ascontiguousarray(idx, np.int64)
    out = np.zeros(ii.size)
    if lib.orc_knn_mean_d2_at(_p(x), x.shape[0], k, _p(ii), ii.size, _p(out)) != 0:
        raise ValueError("k or an index out of range")
    return out


def gaussians_from_points(xyz, rgb, deg, init_opacity=INIT_OPACITY, k=KNN_K, floor=KNN_FLOOR) -> np.ndarray:
    """Geometric densification (Sec. III-A.3, III-B): one Gaussian per point of a keyframe's
    coloured point cloud, initialised as 3DGS does (the renderer the paper keeps):
      mean = the point; log-scale = log sqrt(max(d2, floor)) on all three axes, d2 the mean
      squared distance to the k = 3 nearest other points (exact here; reading);
      rotation = identity (1, 0, 0, 0); opacity logit = logit(init_opacity);
      SH DC = (rgb - 1/2) / Y_0^0 (so the degree-0 colour is rgb); higher bands 0.
    Returns the flat parameter vector (float64) of the m new Gaussians."""
    x = _f64(xyz).reshape(-1, 3)
    c = _f64(rgb).reshape(-1, 3)
    m = x.shape[0]
    K = (deg + 1) ** 2
    d2 = np.maximum(knn_mean_d2(x, k), floor)
    logs = np.repeat(0.5 * np.log(d2)[:, None], 3, axis=1)
    quats = np.zeros((m, 4))
    quats[:, 0] = 1.0
    opac = np.full(m, np.log(init_opacity / (1.0 - init_opacity)))
    dc = (c - 0.5) / SH_C0
    rest = np.zeros((m, K - 1, 3))
    return np.concatenate([x.ravel(), logs.ravel(), quats.ravel(), opac, dc.ravel(), rest.ravel()])
