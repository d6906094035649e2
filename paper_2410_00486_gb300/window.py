"""One CaRtGS mapping iteration over a window of keyframes, on the GPU.

`MappingWindow` owns the device-resident state of the photorealistic mapping
back-end (Sec. III-B): the Gaussian parameters, their Adam moments, the
densification statistics, and every buffer the iteration writes.  One window
iteration is preprocess -> bin_sort -> render_fwd (+ L1 loss) -> render_bwd
(+ densify statistics) -> Adam, each step a libcgs call.  PyTorch only allocates
memory and supplies the stream.

Two forms of the same iteration:
  * batched  (`step`): every view of the window in one launch per stage, the
    parameters read once per window, one shared tile sort;
  * per-view (`step_per_view`): the same math one view at a time (V launches of
    each raster stage), gradients accumulated, one Adam step.
Both give the same gradients (up to float summation order).

`capture()` records one batched iteration into a CUDA graph; `replay()` runs it.
The Adam step counter lives on the device, so replays advance it.
"""
from __future__ import annotations

import math

import torch

from . import _native as N

# Per-group learning rates: means, log_scales, quats, opacity, sh_dc, sh_rest.
LR_DEFAULT = (1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 2.5e-3 / 20.0)


def _u32(n, device):
    """uint32 storage (torch has no general uint32 arithmetic; int32 holds the bits)."""
    return torch.empty(n, dtype=torch.int32, device=device)


class MappingWindow:
    def __init__(self, params: torch.Tensor, n: int, sh_degree: int, width: int, height: int, views: int,
                 tile: int = 16, batch_depth: int = 64, lr=LR_DEFAULT, lambda_o: float = 0.0,
                 lambda_depth: float = 0.1, bg=(0.0, 0.0, 0.0), near_z: float = 0.2,
                 betas=(0.9, 0.999), eps: float = 1e-15, capacity: int | None = None,
                 densify_stats: bool = True, tile_order: bool = True, backward: str = "pixel",
                 lambda_ssim: float = 0.0, batch_depth_bwd: int = 0, persistent_bwd: bool = True):
        if not params.is_cuda or params.dtype != torch.float32:
            raise ValueError("params must be a float32 CUDA tensor")
        dev = params.device
        self.device = dev
        self.n, self.V, self.sh_degree = int(n), int(views), int(sh_degree)
        self.W, self.H = int(width), int(height)
        self.cfg = N.make_config(width, height, tile, batch_depth, sh_degree, near_z, bg, lambda_depth,
                                 batch_depth_bwd)
        P = N.cgs_param_count(n, sh_degree)
        if params.numel() != P:
            raise ValueError(f"params has {params.numel()} floats, expected {P}")
        self.P = P
        self.lr = tuple(float(x) for x in lr)
        self.lambda_o = float(lambda_o)
        self.betas = (float(betas[0]), float(betas[1]))
        self.eps = float(eps)
        self.track_stats = densify_stats
        if backward not in ("pixel", "splat"):
            raise ValueError("backward must be 'pixel' or 'splat'")
        self.backward_kind = backward
        if not 0.0 <= lambda_ssim <= 1.0:
            raise ValueError("lambda_ssim must lie in [0, 1]")
        self.lambda_ssim = float(lambda_ssim)
        f32 = dict(dtype=torch.float32, device=dev)

        self.params = params.contiguous()
        self.grads = torch.zeros(P, **f32)
        self.m = torch.zeros(P, **f32)
        self.v = torch.zeros(P, **f32)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)

        V, H, W = self.V, self.H, self.W
        self.cams = torch.zeros(V, N.CAM_FLOATS, **f32)
        self.view_weight = torch.ones(V, **f32)
        self.tgt_rgb = torch.zeros(V, 3, H, W, **f32)
        self.tgt_depth = torch.zeros(V, H, W, **f32)

        slots = V * self.n
        self.rec = torch.zeros(slots * N.REC_FLOATS, **f32)
        self.slot_grad = torch.zeros(slots * N.REC_FLOATS, **f32)
        self.Tv = N.cgs_tiles_per_view(self.cfg)
        self.Ttot = self.Tv * V
        self.ranges = _u32(2 * self.Ttot, dev)
        self.order = _u32(self.Ttot, dev) if tile_order else None
        self.n_inst = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        # work counter of the persistent raster backward (None: one block per tile)
        self.work = _u32(1, dev) if persistent_bwd else None

        self.img = torch.zeros(V, 3, H, W, **f32)
        self.depth = torch.zeros(V, H, W, **f32)
        self.t_final = torch.zeros(V, H, W, **f32)
        self.last = torch.zeros(V, H, W, dtype=torch.int32, device=dev)
        self.loss_view = torch.zeros(V, **f32)
        self.depth_count = torch.zeros(V, dtype=torch.int32, device=dev)
        self.loss_o = torch.zeros(1, **f32)
        self.fwd_ws = torch.empty(max(256, N.cgs_render_fwd_workspace(V, self.cfg)), dtype=torch.uint8,
                                  device=dev)
        if self.lambda_ssim > 0.0:
            # Eq. 9 with its SSIM term: the loss kernel writes the pixel gradients
            self.dl_dimg = torch.zeros(V, 3, H, W, **f32)
            self.dl_ddepth = torch.zeros(V, H, W, **f32)
            self.ssim_ws = torch.empty(N.cgs_ssim_workspace(V, self.cfg), dtype=torch.uint8, device=dev)
        self.accum = torch.zeros(self.n, **f32)
        self.denom = torch.zeros(self.n, **f32)
        self.max_r2d = torch.zeros(self.n, **f32)
        self._pv = None
        self._graphs = {}
        self._set = 0   # which of the two input sets (staging swaps them) is current
        self._alloc_capacity(capacity if capacity else max(1 << 20, 16 * slots))

    # ------------------------------------------------------------ buffers
    def _alloc_capacity(self, cap: int):
        self.capacity = int(cap)
        self.vals = _u32(max(1, self.capacity), self.device)
        ws = N.cgs_bin_sort_workspace(self.capacity, self.n, self.V, self.cfg)
        self.bin_ws = torch.empty(ws, dtype=torch.uint8, device=self.device)
        if self.backward_kind == "splat":
            # checkpoints of the splat-wise backward: at most capacity / 32 + tiles buckets
            self.max_buckets = self.capacity // 32 + self.Ttot
            nb = N.cgs_ckpt_bytes(self.max_buckets, self.cfg)
            self.ckpt = torch.empty(nb // 4, dtype=torch.float32, device=self.device)
            self.bucket_start = _u32(self.Ttot + 1, self.device)
        self._pv = None
        self._graphs = {}

    def set_window(self, cams, tgt_rgb, tgt_depth=None, view_weight=None, non_blocking=True):
        """Copy the window's cameras (float32[V][20]), targets and view weights into the
        resident buffers (host tensors should be pinned for an asynchronous copy)."""
        self.cams.copy_(torch.as_tensor(cams).reshape(self.V, N.CAM_FLOATS), non_blocking=non_blocking)
        self.tgt_rgb.copy_(torch.as_tensor(tgt_rgb).reshape(self.tgt_rgb.shape), non_blocking=non_blocking)
        if tgt_depth is not None:
            self.tgt_depth.copy_(torch.as_tensor(tgt_depth).reshape(self.tgt_depth.shape),
                                 non_blocking=non_blocking)
        else:
            self.tgt_depth.zero_()
        if view_weight is not None:
            self.view_weight.copy_(torch.as_tensor(view_weight, dtype=torch.float32), non_blocking=non_blocking)

    def set_view_weight(self, view_weight, non_blocking=True):
        self.view_weight.copy_(torch.as_tensor(view_weight, dtype=torch.float32), non_blocking=non_blocking)

    # ------------------------------------------------- pipelined input copies
    def stage_window(self, cams, tgt_rgb, tgt_depth=None):
        """Start copying the next window's cameras and targets from (pinned) host memory into
        device staging buffers on the window's copy stream, so the copy overlaps an iteration
        still running on the compute stream.  `commit_window()` makes them current."""
        if not hasattr(self, "_stage"):
            self._copy_stream = torch.cuda.Stream(device=self.device)
            self._stage = (torch.empty_like(self.cams), torch.empty_like(self.tgt_rgb),
                           torch.empty_like(self.tgt_depth))
            self._staged = torch.cuda.Event()
            self._consumed = torch.cuda.Event()
            self._consumed.record(torch.cuda.current_stream(self.device))
        c, r, d = self._stage
        with torch.cuda.stream(self._copy_stream):
            self._copy_stream.wait_event(self._consumed)       # the previous staging was committed
            c.copy_(torch.as_tensor(cams).reshape(c.shape), non_blocking=True)
            r.copy_(torch.as_tensor(tgt_rgb).reshape(r.shape), non_blocking=True)
            if tgt_depth is not None:
                d.copy_(torch.as_tensor(tgt_depth).reshape(d.shape), non_blocking=True)
            else:
                d.zero_()
            self._staged.record(self._copy_stream)
        self._pending = True

    def commit_window(self):
        """Make the staged inputs current: the compute stream waits for the staging copy and
        the staging buffers become the window's inputs (no copy); the buffers they replace
        take the next staging once the iterations already queued have read them.  Each of the
        two input sets has its own captured graph (`replay`)."""
        if not getattr(self, "_pending", False):
            # nothing staged since the last commit: swapping again would bring back the
            # previous window's inputs
            raise RuntimeError("stage_window() first: no inputs staged since the last commit_window()")
        self._pending = False
        cur = torch.cuda.current_stream(self.device)
        cur.wait_event(self._staged)
        (self.cams, self.tgt_rgb, self.tgt_depth), self._stage = self._stage, (self.cams, self.tgt_rgb,
                                                                              self.tgt_depth)
        self._set ^= 1
        self._consumed.record(cur)

    # ---------------------------------------------------------- iteration
    def forward(self, with_loss: bool = True, params: torch.Tensor | None = None):
        """Preprocess, bin and render every view of the window (loss fused if with_loss;
        with lambda_ssim > 0 the loss of Eq. 9 and its pixel gradients follow the render).
        `params` overrides the window's own parameter vector (same layout)."""
        c = self.cfg
        p = self.params if params is None else params
        N.cgs_preprocess(p, self.n, self.cams, self.V, c, self.rec, self.slot_grad, self.status)
        N.cgs_bin_sort(self.rec, self.n, self.V, c, self.bin_ws, self.capacity, self.vals, self.ranges,
                       self.order, self.n_inst, self.status)
        if self.backward_kind == "splat":
            N.cgs_render_fwd_ckpt(self.rec, self.vals, self.ranges, self.order, self.V, c, self.view_weight,
                                  self.tgt_rgb if with_loss else None, self.tgt_depth if with_loss else None,
                                  self.img, self.depth, self.t_final, self.last, self.loss_view,
                                  self.depth_count, self.fwd_ws, self.ckpt, self.max_buckets,
                                  self.bucket_start, self.status)
        else:
            N.cgs_render_fwd(self.rec, self.vals, self.ranges, self.order, self.V, c, self.view_weight,
                             self.tgt_rgb if with_loss else None, self.tgt_depth if with_loss else None,
                             self.img, self.depth, self.t_final, self.last, self.loss_view, self.depth_count,
                             self.fwd_ws, self.status)
        if with_loss and self.lambda_ssim > 0.0:
            N.cgs_ssim_loss(self.img, self.tgt_rgb, self.depth, self.tgt_depth, self.depth_count, self.V, c,
                            self.view_weight, self.lambda_ssim, self.loss_view, self.dl_dimg, self.dl_ddepth,
                            self.ssim_ws, self.status)

    def backward(self, dl_dimg=None, dl_ddepth=None, params: torch.Tensor | None = None,
                 grads_out: torch.Tensor | None = None):
        """Raster backward + chain rule to the parameters; overwrites self.grads (or
        grads_out).  Pixel gradients come from the fused L1 loss unless dl_dimg is given
        (or the window has an SSIM term, whose gradients the forward wrote)."""
        d = self.track_stats
        if dl_dimg is None and self.lambda_ssim > 0.0:
            dl_dimg, dl_ddepth = self.dl_dimg, self.dl_ddepth
        p = self.params if params is None else params
        g = self.grads if grads_out is None else grads_out
        if self.backward_kind == "splat":
            N.cgs_raster_bwd_splat(self.rec, self.vals, self.ranges, self.order, self.V, self.cfg,
                                   self.view_weight, self.img, self.depth, self.t_final, self.last, self.tgt_rgb,
                                   self.tgt_depth, self.depth_count, dl_dimg, dl_ddepth, self.ckpt,
                                   self.max_buckets, self.bucket_start, self.slot_grad, self.status)
            N.cgs_preprocess_bwd(p, self.n, self.cams, self.V, self.cfg, self.rec, self.slot_grad, g, False,
                                 self.accum if d else None, self.denom if d else None,
                                 self.max_r2d if d else None, self.status)
            return
        N.cgs_render_bwd(p, self.n, self.cams, self.V, self.cfg, self.rec, self.vals, self.ranges,
                         self.order, self.view_weight, self.img, self.depth, self.t_final, self.last,
                         self.tgt_rgb, self.tgt_depth, self.depth_count, dl_dimg, dl_ddepth, self.slot_grad,
                         g, False, self.accum if d else None, self.denom if d else None,
                         self.max_r2d if d else None, self.status, work=self.work)

    def optimizer_step(self):
        N.cgs_adam(self.params, self.grads, self.m, self.v, self.n, self.sh_degree, self.lr, self.betas[0],
                   self.betas[1], self.eps, 0, self.lambda_o, self.loss_o, step_dev=self.step_dev)

    def step(self):
        """One batched window iteration: fwd + loss + bwd + densify stats + Adam."""
        self.forward()
        self.backward()
        self.optimizer_step()

    # ------------------------------------------------------ densification
    def densify(self, tau_p: float = 0.001, eps_alpha: float = 0.02, percent_dense: float = 0.01,
                extent: float = 1.0, normals: torch.Tensor | None = None, seed: int = 0) -> dict:
        """Adaptive density control with the paper's thresholds (Sec. III-A.3, IV-A): clone
        small high-gradient Gaussians, split large ones in two, prune those with opacity below
        eps_alpha.  The gradient statistics are the accumulated view-space norms / counts of
        the iterations since the last call; they restart at zero.  Changes the number of
        Gaussians, so every per-Gaussian buffer is reallocated and a captured graph dropped.
        `normals` (float32 [n, 2, 3], standard normal) are the split samples; drawn from a
        seeded generator if not given."""
        n, deg = self.n, self.sh_degree
        ws = torch.empty(max(256, N.cgs_densify_workspace(n)), dtype=torch.uint8, device=self.device)
        n_out_dev = torch.zeros(1, dtype=torch.int64, device=self.device)
        N.cgs_densify_plan(self.params, n, deg, self.accum, self.denom, tau_p, percent_dense * extent, eps_alpha,
                           ws, n_out_dev)
        n_out = int(n_out_dev.item())
        if normals is None:
            gen = torch.Generator(device=self.device)
            gen.manual_seed(seed)
            normals = torch.randn(n, 2, 3, generator=gen, device=self.device)
        P2 = N.cgs_param_count(max(n_out, 1), deg)
        f32 = dict(dtype=torch.float32, device=self.device)
        p2, m2, v2 = torch.zeros(P2, **f32), torch.zeros(P2, **f32), torch.zeros(P2, **f32)
        N.cgs_densify_apply(self.params, self.m, self.v, n, deg, ws, normals.contiguous(), n_out, p2, m2, v2)
        code = ws[: 4 * n].view(torch.int32)
        counts = torch.bincount(code.long(), minlength=4).cpu().tolist()
        if n_out == 0:
            raise RuntimeError("densification pruned every Gaussian")
        self._resize(n_out, p2, m2, v2)
        return {"pruned": counts[0], "kept": counts[1], "cloned": counts[2], "split": counts[3], "n": n_out}

    def add_points(self, xyz: torch.Tensor, rgb: torch.Tensor, init_opacity: float = 0.1) -> int:
        """Geometric densification (Sec. III-A.3, III-B): append one Gaussian per point of a new
        keyframe's coloured point cloud (xyz, rgb: float32 [m, 3] on the device), initialised
        from the exact 3-nearest-neighbour distances; existing Gaussians keep their Adam state.
        Reallocates every per-Gaussian buffer (a captured graph is dropped).  Returns the new
        Gaussian count."""
        xyz = xyz.to(self.device, torch.float32).contiguous()
        rgb = rgb.to(self.device, torch.float32).contiguous()
        mpts = int(xyz.shape[0])
        if xyz.shape != (mpts, 3) or rgb.shape != (mpts, 3):
            raise ValueError("xyz and rgb must be [m, 3]")
        if mpts == 0:
            return self.n
        n_out = self.n + mpts
        P2 = N.cgs_param_count(n_out, self.sh_degree)
        f32 = dict(dtype=torch.float32, device=self.device)
        p2, m2, v2 = torch.empty(P2, **f32), torch.empty(P2, **f32), torch.empty(P2, **f32)
        ws = torch.empty(N.cgs_points_workspace(mpts), dtype=torch.uint8, device=self.device)
        N.cgs_points_to_gaussians(self.params, self.m, self.v, self.n, self.sh_degree, xyz, rgb, mpts, init_opacity,
                                  ws, p2, m2, v2, self.status)
        self._resize(n_out, p2, m2, v2)
        return n_out

    def _resize(self, n: int, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor):
        f32 = dict(dtype=torch.float32, device=self.device)
        self.n = int(n)
        self.P = N.cgs_param_count(self.n, self.sh_degree)
        self.params, self.m, self.v = params, m, v
        self.grads = torch.zeros(self.P, **f32)
        slots = self.V * self.n
        self.rec = torch.zeros(slots * N.REC_FLOATS, **f32)
        self.slot_grad = torch.zeros(slots * N.REC_FLOATS, **f32)
        self.accum = torch.zeros(self.n, **f32)
        self.denom = torch.zeros(self.n, **f32)
        self.max_r2d = torch.zeros(self.n, **f32)
        self._alloc_capacity(self.capacity)    # the binning workspace depends on n
        self._pv = None
        self._graphs = {}

    # ------------------------------------------------------- per-view form
    def _per_view_buffers(self):
        if self._pv is None:
            dev, n = self.device, self.n
            pv = {}
            pv["rec"] = torch.zeros(n * N.REC_FLOATS, dtype=torch.float32, device=dev)
            pv["slot_grad"] = torch.zeros(n * N.REC_FLOATS, dtype=torch.float32, device=dev)
            pv["ranges"] = _u32(2 * self.Tv, dev)
            pv["order"] = _u32(self.Tv, dev) if self.order is not None else None
            pv["ws"] = torch.empty(N.cgs_bin_sort_workspace(self.capacity, n, 1, self.cfg), dtype=torch.uint8,
                                   device=dev)
            pv["fwd_ws"] = torch.empty(max(256, N.cgs_render_fwd_workspace(1, self.cfg)), dtype=torch.uint8,
                                       device=dev)
            if self.lambda_ssim > 0.0:
                pv["ssim_ws"] = torch.empty(N.cgs_ssim_workspace(1, self.cfg), dtype=torch.uint8, device=dev)
            self._pv = pv
        return self._pv

    def step_per_view(self, adam_every_view: bool = False):
        """The same iteration, one view at a time (gradients accumulated, one Adam step).
        adam_every_view: the paper's sequential mapping loop instead (Sec. III-C.2), one
        optimiser step after every view, so each view renders the parameters the previous
        view's step left (V iterations of one keyframe each)."""
        pv = self._per_view_buffers()
        c = self.cfg
        d = self.track_stats
        for v in range(self.V):
            cam = self.cams[v:v + 1]
            N.cgs_preprocess(self.params, self.n, cam, 1, c, pv["rec"], pv["slot_grad"], self.status)
            N.cgs_bin_sort(pv["rec"], self.n, 1, c, pv["ws"], self.capacity, self.vals, pv["ranges"], pv["order"],
                           self.n_inst, self.status)
            img, dep, tf, la = self.img[v:v + 1], self.depth[v:v + 1], self.t_final[v:v + 1], self.last[v:v + 1]
            tr, td = self.tgt_rgb[v:v + 1], self.tgt_depth[v:v + 1]
            w, lv, dc = self.view_weight[v:v + 1], self.loss_view[v:v + 1], self.depth_count[v:v + 1]
            N.cgs_render_fwd(pv["rec"], self.vals, pv["ranges"], pv["order"], 1, c, w, tr, td, img, dep, tf, la,
                             lv, dc, pv["fwd_ws"], self.status)
            gi = gd = None
            if self.lambda_ssim > 0.0:
                gi, gd = self.dl_dimg[v:v + 1], self.dl_ddepth[v:v + 1]
                N.cgs_ssim_loss(img, tr, dep, td, dc, 1, c, w, self.lambda_ssim, lv, gi, gd, pv["ssim_ws"],
                                self.status)
            N.cgs_render_bwd(self.params, self.n, cam, 1, c, pv["rec"], self.vals, pv["ranges"], pv["order"], w,
                             img, dep, tf, la, tr, td, dc, gi, gd, pv["slot_grad"], self.grads,
                             v > 0 and not adam_every_view, self.accum if d else None,
                             self.denom if d else None, self.max_r2d if d else None, self.status, work=self.work)
            if adam_every_view:
                self.optimizer_step()
        if not adam_every_view:
            self.optimizer_step()

    # --------------------------------------------------------- CUDA graph
    def capture(self, warmup: int = 0):
        """Record one batched iteration (`step`) into a CUDA graph for the current input
        buffers (the graph of the other input set, after `commit_window`, is recorded at its
        first `replay`)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream(self.device).wait_stream(s)
        self._graphs = {}
        return self._capture_current()

    def _capture_current(self):
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self._graphs[self._set] = g
        return g

    @property
    def graph(self):
        """The captured iteration for the current input buffers (None if not captured)."""
        return self._graphs.get(self._set)

    def replay(self):
        g = self._graphs.get(self._set)
        if g is None:
            if not self._graphs:
                raise RuntimeError("capture() first")
            g = self._capture_current()   # first replay on the other input set
        g.replay()

    # ------------------------------------------------------------- status
    def read_status(self) -> tuple[int, int]:
        """(device status, instance count) -- synchronises."""
        return int(self.status.item()), int(self.n_inst.item())

    def ensure_capacity(self, headroom: float = 1.25) -> bool:
        """Check the device status after an iteration; on a capacity overflow, grow the
        instance buffers (dropping any captured graph) and return False so the caller
        re-runs the iteration."""
        st, ninst = self.read_status()
        if st == N.CGS_ERR_CAPACITY:
            self.status.zero_()
            self._alloc_capacity(int(math.ceil(ninst * headroom)))
            return False
        if st != 0:
            raise N.CgsError("device status", st)
        return True

    def fit_capacity(self, headroom: float = 1.25):
        """Run the forward once and size the instance buffers to headroom x the count."""
        self.forward(with_loss=False)
        ok = self.ensure_capacity(headroom)
        if not ok:
            self.forward(with_loss=False)
            self.ensure_capacity(headroom)
        ninst = int(self.n_inst.item())
        want = int(math.ceil(max(ninst, 1) * headroom))
        if want < self.capacity // 2 or want > self.capacity:
            self._alloc_capacity(want)
        return ninst
