"""ctypes binding of libcgs (include/cgs.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls and takes torch
tensors (or None) where the C function takes a pointer.  Device-pointer arguments
must be CUDA tensors; a CPU tensor raises before anything is launched.  There is
no fallback: if libcgs.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_float, c_int32, c_int64, c_size_t, c_uint32, c_void_p
from pathlib import Path

import numpy as np
import torch

LIB_PATH = Path(__file__).resolve().parent / "_build" / "libcgs.so"

REC_FLOATS = 12
CAM_FLOATS = 20

CGS_OK = 0
CGS_ERR_ARG = -1
CGS_ERR_WORKSPACE = -2
CGS_ERR_CUDA = -3
CGS_ERR_CAPACITY = -4
CGS_ERR_NONFINITE = -5
CGS_ERR_TIMEOUT = -6


class cgs_camera(ctypes.Structure):
    _fields_ = [("R", c_float * 9), ("t", c_float * 3), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("loss_weight", c_float), ("pad", c_float * 3)]


class cgs_config(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("tile", c_int32), ("batch_depth", c_int32),
                ("sh_degree", c_int32), ("near_z", c_float), ("bg", c_float * 3),
                ("lambda_depth", c_float), ("batch_depth_bwd", c_int32), ("count_work", c_int32),
                ("rect_lists", c_int32)]


def make_config(width, height, tile=16, batch_depth=64, sh_degree=3, near_z=0.2,
                bg=(0.0, 0.0, 0.0), lambda_depth=0.1, batch_depth_bwd=0, count_work=False,
                rect_lists=False) -> cgs_config:
    c = cgs_config()
    c.width, c.height, c.tile, c.batch_depth, c.sh_degree = width, height, tile, batch_depth, sh_degree
    c.near_z = near_z
    c.bg = (c_float * 3)(*bg)
    c.lambda_depth = lambda_depth
    c.batch_depth_bwd = batch_depth_bwd
    c.count_work = 1 if count_work else 0
    c.rect_lists = 1 if rect_lists else 0
    return c


_P = c_void_p
_SIGS = {
    "cgs_param_count": (c_int64, [c_int64, c_int32]),
    "cgs_tiles_per_view": (c_int64, [_P]),
    "cgs_preprocess": (c_int32, [_P, c_int64, _P, c_int32, _P, _P, _P, _P, _P]),
    "cgs_bin_sort_workspace": (c_size_t, [c_int64, c_int64, c_int32, _P]),
    "cgs_bin_sort": (c_int32, [_P, c_int64, c_int32, _P, _P, c_size_t, c_int64, _P, _P, _P, _P, _P, _P]),
    "cgs_render_fwd_workspace": (c_size_t, [c_int32, _P]),
    "cgs_render_fwd": (c_int32, [_P, _P, _P, _P, c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                 c_size_t, _P, _P]),
    "cgs_render_fwd_noalloc": (c_int32, [_P, _P, _P, _P, c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                         _P, _P]),
    "cgs_ckpt_bytes": (c_size_t, [c_int64, _P]),
    "cgs_render_fwd_ckpt": (c_int32, [_P, _P, _P, _P, c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                      c_size_t, _P, c_int64, _P, _P, _P]),
    "cgs_raster_bwd_splat": (c_int32, [_P, _P, _P, _P, c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                       _P, c_int64, _P, _P, _P, _P]),
    "cgs_raster_bwd": (c_int32, [_P, _P, _P, _P, c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                 _P, _P, _P, _P]),
    "cgs_preprocess_bwd": (c_int32, [_P, c_int64, _P, c_int32, _P, _P, _P, _P, c_int32, _P, _P, _P,
                                     _P, _P]),
    "cgs_render_bwd": (c_int32, [_P, c_int64, _P, c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                 _P, _P, _P, _P, _P, _P, c_int32, _P, _P, _P, _P, _P, _P]),
    "cgs_densify_stats": (c_int32, [_P, _P, c_int64, c_int32, _P, _P, _P, _P, _P]),
    "cgs_adam": (c_int32, [_P, _P, _P, _P, c_int64, c_int32, _P, c_float, c_float, c_float, c_int32,
                           _P, c_float, _P, _P]),
    "cgs_densify_workspace": (c_size_t, [c_int64]),
    "cgs_densify_plan": (c_int32, [_P, c_int64, c_int32, _P, _P, c_double, c_double, c_double, _P, c_size_t, _P,
                                   _P]),
    "cgs_densify_apply": (c_int32, [_P, _P, _P, c_int64, c_int32, _P, c_size_t, _P, c_int64, _P, _P, _P, _P]),
    "cgs_points_workspace": (c_size_t, [c_int64]),
    "cgs_points_to_gaussians": (c_int32, [_P, _P, _P, c_int64, c_int32, _P, _P, c_int64, c_float, _P, c_size_t, _P,
                                          _P, _P, _P, _P]),
    "cgs_ssim_workspace": (c_size_t, [c_int32, _P]),
    "cgs_ssim_loss": (c_int32, [_P, _P, _P, _P, _P, c_int32, _P, _P, c_float, _P, _P, _P, _P, c_size_t, _P,
                                _P]),
    "cgs_sched_create": (_P, [c_int32]),
    "cgs_sched_destroy": (None, [_P]),
    "cgs_sched_add": (c_int32, [_P, c_int32, c_int32]),
    "cgs_sched_draw": (c_int32, [_P, c_uint32]),
    "cgs_sched_report": (c_int32, [_P, c_int32, c_double]),
    "cgs_sched_draw_n": (c_int32, [_P, _P, c_int32, _P]),
    "cgs_sched_report_n": (c_int32, [_P, _P, _P, c_int32]),
    "cgs_sched_state": (c_int32, [_P, POINTER(c_int32), POINTER(c_int32), POINTER(c_double), c_int32]),
    "cgs_status_string": (ctypes.c_char_p, [c_int32]),
}
EXPORTS = tuple(_SIGS)

_lib = None


class CgsError(RuntimeError):
    def __init__(self, name: str, status: int):
        self.status = status
        super().__init__(f"{name}: {status_string(status)} (status {status})")


def lib() -> ctypes.CDLL:
    """Load libcgs.so (built in-tree by paper_2410_00486_gb300.build)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_00486_gb300.build.build()")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().cgs_status_string(int(status)).decode()


def _dev(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("a device-pointer argument must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor arguments must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _check(name, rc):
    if rc != CGS_OK:
        raise CgsError(name, rc)


def cgs_param_count(n: int, sh_degree: int) -> int:
    return lib().cgs_param_count(n, sh_degree)


def cgs_tiles_per_view(cfg: cgs_config) -> int:
    return lib().cgs_tiles_per_view(byref(cfg))


def cgs_preprocess(params, n, cams, V, cfg, rec, slot_grad=None, status=None, stream=None):
    _check("cgs_preprocess", lib().cgs_preprocess(_dev(params), n, _dev(cams), V, byref(cfg), _dev(rec),
                                                  _dev(slot_grad), _dev(status), _stream(stream)))


def cgs_bin_sort_workspace(capacity, n, V, cfg) -> int:
    return lib().cgs_bin_sort_workspace(capacity, n, V, byref(cfg))


def cgs_bin_sort(rec, n, V, cfg, workspace, capacity, vals, ranges, tile_order, n_inst, status=None,
                 stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check("cgs_bin_sort", lib().cgs_bin_sort(_dev(rec), n, V, byref(cfg), _dev(workspace), nbytes, capacity,
                                              _dev(vals), _dev(ranges), _dev(tile_order), _dev(n_inst),
                                              _dev(status), _stream(stream)))


def cgs_render_fwd_workspace(V, cfg) -> int:
    return lib().cgs_render_fwd_workspace(V, byref(cfg))


def cgs_render_fwd(rec, vals, ranges, tile_order, V, cfg, view_weight, tgt_rgb, tgt_depth, img, depth,
                   t_final, last, loss_view, depth_count, workspace, status=None, stream=None):
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check("cgs_render_fwd", lib().cgs_render_fwd(
        _dev(rec), _dev(vals), _dev(ranges), _dev(tile_order), V, byref(cfg), _dev(view_weight),
        _dev(tgt_rgb), _dev(tgt_depth), _dev(img), _dev(depth), _dev(t_final), _dev(last),
        _dev(loss_view), _dev(depth_count), _dev(workspace), nbytes, _dev(status), _stream(stream)))


def cgs_render_fwd_noalloc(rec, vals, ranges, tile_order, V, cfg, view_weight, tgt_rgb, tgt_depth, img, depth,
                           t_final, last, loss_view, depth_count, status=None, stream=None):
    """cgs_render_fwd with the library's built-in scratch (no workspace argument); for
    callers that cannot allocate.  Windows above 65536 tiles are refused."""
    _check("cgs_render_fwd_noalloc", lib().cgs_render_fwd_noalloc(
        _dev(rec), _dev(vals), _dev(ranges), _dev(tile_order), V, byref(cfg), _dev(view_weight),
        _dev(tgt_rgb), _dev(tgt_depth), _dev(img), _dev(depth), _dev(t_final), _dev(last),
        _dev(loss_view), _dev(depth_count), _dev(status), _stream(stream)))


def cgs_ckpt_bytes(max_buckets, cfg) -> int:
    return lib().cgs_ckpt_bytes(max_buckets, byref(cfg))


def cgs_render_fwd_ckpt(rec, vals, ranges, tile_order, V, cfg, view_weight, tgt_rgb, tgt_depth, img, depth,
                        t_final, last, loss_view, depth_count, workspace, ckpt, max_buckets, bucket_start,
                        status=None, stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check("cgs_render_fwd_ckpt", lib().cgs_render_fwd_ckpt(
        _dev(rec), _dev(vals), _dev(ranges), _dev(tile_order), V, byref(cfg), _dev(view_weight),
        _dev(tgt_rgb), _dev(tgt_depth), _dev(img), _dev(depth), _dev(t_final), _dev(last),
        _dev(loss_view), _dev(depth_count), _dev(workspace), nbytes, _dev(ckpt), max_buckets,
        _dev(bucket_start), _dev(status), _stream(stream)))


def cgs_raster_bwd_splat(rec, vals, ranges, tile_order, V, cfg, view_weight, img, depth, t_final, last,
                         tgt_rgb, tgt_depth, depth_count, dl_dimg, dl_ddepth, ckpt, max_buckets, bucket_start,
                         slot_grad, status=None, stream=None):
    _check("cgs_raster_bwd_splat", lib().cgs_raster_bwd_splat(
        _dev(rec), _dev(vals), _dev(ranges), _dev(tile_order), V, byref(cfg), _dev(view_weight), _dev(img),
        _dev(depth), _dev(t_final), _dev(last), _dev(tgt_rgb), _dev(tgt_depth), _dev(depth_count),
        _dev(dl_dimg), _dev(dl_ddepth), _dev(ckpt), max_buckets, _dev(bucket_start), _dev(slot_grad),
        _dev(status), _stream(stream)))


def cgs_raster_bwd(rec, vals, ranges, tile_order, V, cfg, view_weight, img, depth, t_final, last, tgt_rgb,
                   tgt_depth, depth_count, dl_dimg, dl_ddepth, slot_grad, status=None, stream=None, work=None):
    _check("cgs_raster_bwd", lib().cgs_raster_bwd(
        _dev(rec), _dev(vals), _dev(ranges), _dev(tile_order), V, byref(cfg), _dev(view_weight), _dev(img),
        _dev(depth), _dev(t_final), _dev(last), _dev(tgt_rgb), _dev(tgt_depth), _dev(depth_count),
        _dev(dl_dimg), _dev(dl_ddepth), _dev(slot_grad), _dev(work), _dev(status), _stream(stream)))


def cgs_preprocess_bwd(params, n, cams, V, cfg, rec, slot_grad, param_grad, accumulate=False, accum=None,
                       denom=None, max_r2d=None, status=None, stream=None):
    _check("cgs_preprocess_bwd", lib().cgs_preprocess_bwd(
        _dev(params), n, _dev(cams), V, byref(cfg), _dev(rec), _dev(slot_grad), _dev(param_grad),
        int(bool(accumulate)), _dev(accum), _dev(denom), _dev(max_r2d), _dev(status), _stream(stream)))


def cgs_render_bwd(params, n, cams, V, cfg, rec, vals, ranges, tile_order, view_weight, img, depth, t_final,
                   last, tgt_rgb, tgt_depth, depth_count, dl_dimg, dl_ddepth, slot_grad, param_grad,
                   accumulate=False, accum=None, denom=None, max_r2d=None, status=None, stream=None, work=None):
    _check("cgs_render_bwd", lib().cgs_render_bwd(
        _dev(params), n, _dev(cams), V, byref(cfg), _dev(rec), _dev(vals), _dev(ranges), _dev(tile_order),
        _dev(view_weight), _dev(img), _dev(depth), _dev(t_final), _dev(last), _dev(tgt_rgb), _dev(tgt_depth),
        _dev(depth_count), _dev(dl_dimg), _dev(dl_ddepth), _dev(slot_grad), _dev(param_grad),
        int(bool(accumulate)), _dev(accum), _dev(denom), _dev(max_r2d), _dev(work), _dev(status),
        _stream(stream)))


def cgs_densify_stats(rec, slot_grad, n, V, cfg, accum, denom, max_r2d, stream=None):
    _check("cgs_densify_stats", lib().cgs_densify_stats(_dev(rec), _dev(slot_grad), n, V, byref(cfg),
                                                        _dev(accum), _dev(denom), _dev(max_r2d),
                                                        _stream(stream)))


def cgs_adam(params, grads, m, v, n, sh_degree, lr, beta1, beta2, eps, step, lambda_o, loss_o=None,
             step_dev=None, stream=None):
    lr6 = (c_float * 6)(*[float(x) for x in lr])
    _check("cgs_adam", lib().cgs_adam(_dev(params), _dev(grads), _dev(m), _dev(v), n, sh_degree,
                                      ctypes.cast(lr6, c_void_p), beta1, beta2, eps, step, _dev(step_dev),
                                      lambda_o, _dev(loss_o), _stream(stream)))


def cgs_densify_workspace(n) -> int:
    return lib().cgs_densify_workspace(n)


def cgs_densify_plan(params, n, sh_degree, accum, denom, tau_p, scale_thr, eps_alpha, workspace, n_out,
                     stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check("cgs_densify_plan", lib().cgs_densify_plan(_dev(params), n, sh_degree, _dev(accum), _dev(denom),
                                                      float(tau_p), float(scale_thr), float(eps_alpha),
                                                      _dev(workspace), nbytes, _dev(n_out), _stream(stream)))


def cgs_densify_apply(params, m, v, n, sh_degree, workspace, normals, n_out, params_out, m_out, v_out,
                      stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check("cgs_densify_apply", lib().cgs_densify_apply(_dev(params), _dev(m), _dev(v), n, sh_degree,
                                                        _dev(workspace), nbytes, _dev(normals), n_out,
                                                        _dev(params_out), _dev(m_out), _dev(v_out),
                                                        _stream(stream)))


def cgs_points_workspace(n_points) -> int:
    return lib().cgs_points_workspace(n_points)


def cgs_points_to_gaussians(params, m, v, n, sh_degree, xyz, rgb, n_points, init_opacity, workspace, params_out,
                            m_out, v_out, status=None, stream=None):
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("cgs_points_to_gaussians", lib().cgs_points_to_gaussians(
        _dev(params), _dev(m), _dev(v), n, sh_degree, _dev(xyz), _dev(rgb), n_points, float(init_opacity),
        _dev(workspace), nbytes, _dev(params_out), _dev(m_out), _dev(v_out), _dev(status), _stream(stream)))


def cgs_ssim_workspace(V, cfg) -> int:
    return lib().cgs_ssim_workspace(V, byref(cfg))


def cgs_ssim_loss(img, tgt_rgb, depth, tgt_depth, depth_count, V, cfg, view_weight, lambda_ssim, loss_view,
                  dl_dimg, dl_ddepth, workspace, status=None, stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check("cgs_ssim_loss", lib().cgs_ssim_loss(_dev(img), _dev(tgt_rgb), _dev(depth), _dev(tgt_depth),
                                                _dev(depth_count), V, byref(cfg), _dev(view_weight),
                                                float(lambda_ssim), _dev(loss_view), _dev(dl_dimg),
                                                _dev(dl_ddepth), _dev(workspace), nbytes, _dev(status),
                                                _stream(stream)))


class Scheduler:
    """Host-side adaptive keyframe scheduler of libcgs (Eqs. 5-8); see cgs.h."""

    def __init__(self, d: int = 4):
        self._h = lib().cgs_sched_create(d)
        if not self._h:
            raise CgsError("cgs_sched_create", CGS_ERR_ARG)

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.cgs_sched_destroy(h)

    def add(self, keyframe_id: int, r0: int) -> int:
        rc = lib().cgs_sched_add(self._h, keyframe_id, r0)
        if rc < 0:
            raise CgsError("cgs_sched_add", rc)
        return rc

    def draw(self, rand_u32: int) -> int:
        rc = lib().cgs_sched_draw(self._h, int(rand_u32) & 0xFFFFFFFF)
        if rc < 0:
            raise CgsError("cgs_sched_draw", rc)
        return rc

    def report(self, index: int, loss: float):
        _check("cgs_sched_report", lib().cgs_sched_report(self._h, index, float(loss)))

    def draw_n(self, rand_u32) -> np.ndarray:
        """len(rand_u32) draws in one call; returns the pool indices (int32)."""
        r = np.ascontiguousarray(rand_u32, dtype=np.uint32)
        out = np.empty(r.size, dtype=np.int32)
        _check("cgs_sched_draw_n", lib().cgs_sched_draw_n(self._h, r.ctypes.data, r.size, out.ctypes.data))
        return out

    def report_n(self, index, loss):
        """Reports loss[i] for pool index index[i], in one call."""
        idx = np.ascontiguousarray(index, dtype=np.int32)
        ls = np.ascontiguousarray(loss, dtype=np.float64)
        if idx.size != ls.size:
            raise ValueError("index and loss differ in length")
        _check("cgs_sched_report_n", lib().cgs_sched_report_n(self._h, idx.ctypes.data, ls.ctypes.data, idx.size))

    def state(self):
        k = lib().cgs_sched_state(self._h, None, None, None, 0)
        ids = (c_int32 * max(k, 1))()
        r = (c_int32 * max(k, 1))()
        l = (c_double * max(k, 1))()
        lib().cgs_sched_state(self._h, ids, r, l, k)
        return list(ids)[:k], list(r)[:k], list(l)[:k]
