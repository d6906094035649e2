/*
 * cgs.h -- C ABI of libcgs: one differentiable 3D Gaussian Splatting mapping
 * iteration over a window of keyframes, as used by the photorealistic mapping
 * back-end of CaRtGS (arXiv 2410.00486, Sec. III-B / III-C), for NVIDIA GB300
 * (sm_103a).
 *
 * Problem statement (Sec. III-B): Gaussians G = {p, q, s, sigma, SH} and a window
 * of keyframes (pose, observed RGB image, optional depth) are given; render each
 * keyframe by alpha blending (Eq. 1), measure the L1 photometric + depth loss
 * (the L1 part of Eq. 9, the opacity term of Eqs. 10-11) and take one optimiser
 * step on G.  The adaptive keyframe schedule (Eqs. 5-8) runs on the host.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All pointers marked "device" are CUDA device pointers owned by the caller.
 *    The library never allocates, frees or synchronises device memory; it only
 *    enqueues kernels and memsets on `stream` (a cudaStream_t, NULL = legacy
 *    default stream).  Nothing is allocated inside the calls, so the whole
 *    iteration can be captured into a CUDA graph by the caller.
 *  - Return value: synchronous argument validation and launch status
 *    (CGS_OK, CGS_ERR_ARG, CGS_ERR_WORKSPACE, CGS_ERR_CUDA).  Conditions found
 *    on the device are written to `*status_dev` (device int32, caller clears
 *    it to 0; first error wins) and read by the caller after synchronising:
 *    CGS_ERR_CAPACITY, CGS_ERR_NONFINITE.  No kernel traps or asserts.
 *  - A "slot" is one (view v, Gaussian g) pair, index v*n + g, 0 <= v < V.
 *  - All floating-point data is float32.
 *
 * Parameter vector (device float[cgs_param_count(n, sh_degree)]), groups in order:
 *    means[n][3] | log_scales[n][3] | quats[n][4] (w, x, y, z, unnormalised) |
 *    opacity_logits[n] | sh_dc[n][3] | sh_rest[n][K-1][3],   K = (sh_degree+1)^2
 *  Activations (Sec. III-B parameters p, q, s, sigma): s = exp(log_scale),
 *  q normalised, opacity = sigmoid(logit), colour = SH(dir) + 0.5 clamped below 0.
 *
 * Projected record of a slot (device float[V*n][CGS_REC_FLOATS], 16-byte aligned):
 *    [0] u  [1] v      projected centre, pixel (x, y) centred on integer (x, y)
 *    [2] A  [3] B  [4] C   conic (inverse 2-D covariance): power = -(A dx^2 + C dy^2)/2 - B dx dy
 *    [5] opacity  [6] depth (camera z)  [7] radius as int32 bits (0 = culled)
 *    [8] r  [9] g  [10] b  [11] tau = -ln(255 opacity): alpha >= 1/255 exactly when power >= tau
 * Slot gradient (device float[V*n][CGS_REC_FLOATS]): dL/d(field) at the same
 * index for fields 0-6 and 8-10; entries 7 and 11 are unused (kept zero).
 */
#ifndef CGS_H
#define CGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CGS_REC_FLOATS 12

enum cgs_status {
    CGS_OK = 0,
    CGS_ERR_ARG = -1,        /* invalid argument (null pointer, size, alignment, unsupported option) */
    CGS_ERR_WORKSPACE = -2,  /* workspace smaller than the matching *_workspace() query */
    CGS_ERR_CUDA = -3,       /* a CUDA launch or memset returned an error */
    CGS_ERR_CAPACITY = -4,   /* device: tile instances exceeded the capacity; lists were truncated */
    CGS_ERR_NONFINITE = -5,  /* device: the loss of a view was NaN or infinite */
    CGS_ERR_TIMEOUT = -6     /* reserved: a bounded device-side wait gave up (no call waits today) */
};

/* One keyframe's pinhole camera: world -> camera x_c = R x_w + t, camera axes x right,
 * y down, z forward; pixel = (fx x_c/z_c + cx, fy y_c/z_c + cy).  80 bytes. */
typedef struct {
    float R[9];          /* row-major rotation */
    float t[3];          /* translation */
    float fx, fy, cx, cy;
    float loss_weight;   /* not read by the kernels: view weights are passed as view_weight */
    float pad[3];
} cgs_camera;

/* Settings shared by every view of a window (host struct, read at call time). */
typedef struct {
    int32_t width, height;   /* image size in pixels, identical for all views */
    int32_t tile;            /* tile edge B: 8, 16 or 32 */
    int32_t batch_depth;     /* splats staged per shared-memory batch in the raster kernels:
                                32, 64, 128 or 256 */
    int32_t sh_degree;       /* 0..3 */
    float near_z;            /* near-plane cull: camera z must exceed this (0.2) */
    float bg[3];             /* background colour added with the final transmittance */
    float lambda_depth;      /* weight of the masked depth L1 term (0.1) */
    int32_t batch_depth_bwd; /* splats per batch in the pixel-wise raster backward: 0 (same as
                                batch_depth), 32, 64, 128 or 256 */
    int32_t count_work;      /* nonzero: cgs_render_fwd also counts the (splat, pixel) pairs it
                                blends (per-tile partial 4; a per-pair counter, about 5% of the
                                blend's time); 0: that partial is written as 0 */
    int32_t rect_lists;      /* nonzero: cgs_bin_sort lists every visible slot in every tile of
                                its rectangle (the plain 3DGS binning); 0: only in the tiles its
                                alpha >= 1/255 ellipse reaches (same renders, about half the
                                instances) */
} cgs_config;

/* Number of floats in the parameter vector: (14 + 3 (K-1)) n. */
int64_t cgs_param_count(int64_t n, int32_t sh_degree);

/* Number of tiles per view and for the whole window: ceil(W/B) ceil(H/B) (* V). */
int64_t cgs_tiles_per_view(const cgs_config *cfg);

/*
 * cgs_preprocess -- projection of every Gaussian into every view of the window
 * (the "projected 2D Gaussian" and colour c_k of Eq. 1, Sec. III-B; 3DGS EWA
 * projection): per slot, camera-space mean, near-plane cull, 3-D covariance
 * R diag(s^2) R^T, Jacobian of the perspective map (guard band 1.3 x half
 * field of view), 2-D covariance + 0.3 I, conic, radius ceil(3 sqrt(lambda_max))
 * (lambda_max = mid + sqrt(max(0.1, mid^2 - det))), tile rectangle (a slot with
 * an empty rectangle is culled), SH colour at the view direction (+0.5, clamped
 * at 0) and sigmoid opacity.  Each Gaussian's parameters are read once for all
 * V views.
 *   params    device, parameter vector (layout above), n Gaussians
 *   cams      device, cgs_camera[V]
 *   rec       device out, float[V*n][12] records (every slot's record is written; a
 *             culled slot's is all zero, radius 0)
 *   slot_grad device out, float[V*n][12]; zeroed for every slot so the backward
 *             can accumulate into it (may be NULL to skip)
 * Errors: CGS_ERR_ARG for null/unaligned pointers, n < 1, V < 1, V*n >= 2^32,
 * unsupported tile / sh_degree / sizes.
 */
int cgs_preprocess(const float *params, int64_t n, const cgs_camera *cams, int32_t V,
                   const cgs_config *cfg, float *rec, float *slot_grad, int32_t *status_dev,
                   void *stream);

/*
 * cgs_bin_sort -- tile binning: every visible slot is listed in each tile of its
 * rectangle that its alpha >= 1/255 ellipse can reach at a pixel centre (a splat left out
 * of a tile is one every pixel of the tile skips: the render is unchanged; with
 * cfg->rect_lists, in every tile of the rectangle), and each
 * tile's list is sorted by (depth, slot) ascending; tiles are
 * numbered view-major (global tile = v*Tx*Ty + ty*Tx + tx), so the whole window
 * shares one sort.  The order is the blending order of Eq. 1 (front to back);
 * equal depths keep the Gaussian order.  Rectangle of a slot with centre (u, v)
 * and radius r, in tile units, hi exclusive:
 *   [clamp(floor((u-r)/B), 0, Tx), clamp(floor((u+r+B-1)/B), 0, Tx)) and likewise in y,
 * evaluated exactly (u enters only through floor(u)).  Reach of a splat in the tile's
 * pixel-centre box [bx0, bx1] x [by0, by1], from the record's conic and tau in float32,
 * every operation one IEEE rounding: none if tau > 1e-4; all if A C - B B <= 0;
 * otherwise, with q = A dx^2 + 2 B dx dy + C dy^2 and t2 = (-2 tau) 1.001 + 1e-3, the
 * ellipse's bounding box (half-extents sqrt(t2 C / det) + 0.01, sqrt(t2 A / det) + 0.01)
 * must meet the box and, unless the centre is inside it, the minimum of q over the box
 * (on an edge: the parabola's clamped vertex) must be at most t2.
 * Method: a counting pass over tiles (the most significant radix digit, one per
 * tile), a scatter into per-tile buckets, then a per-tile sort of the unique
 * 64-bit keys (depth bits << 32 | slot) in shared memory.
 *   rec        device, records from cgs_preprocess (u, v, conic, depth, radius, tau are read)
 *   workspace  device scratch of at least cgs_bin_sort_workspace(capacity, n, V, cfg) bytes,
 *              256-byte aligned
 *   capacity   number of entries `vals` can hold
 *   vals       device out, uint32[capacity]: slot ids, tile after tile
 *   ranges     device out, uint32[2 * V * tiles_per_view]: [start, end) of each tile, the
 *              exclusive scan of the per-tile counts (an empty tile is [start, start))
 *   tile_order device out (may be NULL), uint32[V * tiles_per_view]: tiles ordered
 *              by decreasing list length (work order for the raster kernels)
 *   n_inst_dev device out, int64: total number of tile instances (also when it
 *              exceeds capacity; then lists are truncated and CGS_ERR_CAPACITY set)
 */
size_t cgs_bin_sort_workspace(int64_t capacity, int64_t n, int32_t V, const cgs_config *cfg);
int cgs_bin_sort(const float *rec, int64_t n, int32_t V, const cgs_config *cfg, void *workspace,
                 size_t workspace_bytes, int64_t capacity, uint32_t *vals, uint32_t *ranges,
                 uint32_t *tile_order, int64_t *n_inst_dev, int32_t *status_dev, void *stream);

/*
 * cgs_render_fwd -- alpha blending of Eq. 1 (Sec. III-B; read with (1 - alpha_j)
 * inside the product), front to back per pixel over its tile's list:
 *   power = -(A dx^2 + C dy^2)/2 - B dx dy, (dx, dy) = (u - x, v - y); skip if power > 0;
 *   alpha = min(0.99, opacity exp(power)); skip if alpha < 1/255;
 *   stop before a splat that would take T (1 - alpha) below 1e-4;
 *   img = sum c alpha T + T_final bg, depth = sum z alpha T.
 * With targets, the L1 loss of Eq. 9 (lambda_ssim = 0) plus the depth term is fused:
 *   L_v = w_v [ mean |img - tgt_rgb| + lambda_depth mean_{tgt_depth > 0} |depth - tgt_depth| ].
 *   vals, ranges  from cgs_bin_sort;  tile_order may be NULL (natural order)
 *   view_weight   device float[V] (w_v), may be NULL (all 1)
 *   tgt_rgb       device float[V][3][H][W] or NULL (no loss);  tgt_depth float[V][H][W] or NULL
 *   img float[V][3][H][W], depth float[V][H][W], t_final float[V][H][W],
 *   last uint32[V][H][W] (1-based list position of the last blended splat, 0 = none)
 *   loss_view     device float[V] out (only with targets)
 *   depth_count   device int32[V] out: |{tgt_depth > 0}| per view (only with targets)
 *   workspace     device scratch of cgs_render_fwd_workspace(V, cfg) bytes (required); on
 *                 return it holds float[V * tiles_per_view][5] per-tile partial sums: sum |r_rgb|,
 *                 sum |r_depth| over valid depth pixels, valid depth count, (splat, pixel)
 *                 pairs evaluated, pairs blended (the last two are the blend's work counts;
 *                 pairs blended only with cfg->count_work, else 0)
 */
size_t cgs_render_fwd_workspace(int32_t V, const cgs_config *cfg);
int cgs_render_fwd(const float *rec, const uint32_t *vals, const uint32_t *ranges,
                   const uint32_t *tile_order, int32_t V, const cgs_config *cfg,
                   const float *view_weight, const float *tgt_rgb, const float *tgt_depth,
                   float *img, float *depth, float *t_final, uint32_t *last, float *loss_view,
                   int32_t *depth_count, void *workspace, size_t workspace_bytes,
                   int32_t *status_dev, void *stream);

/*
 * cgs_render_fwd_noalloc -- cgs_render_fwd for callers that cannot allocate device
 * memory or pass a workspace: for instance a real-time mapping loop that must not
 * allocate once running (an allocation can block in the CUDA driver and miss the frame
 * budget), or glue code that only receives another framework's input and output
 * buffers.  The paper has no counterpart; it is an interface convenience.
 * Same arguments and results as cgs_render_fwd without the workspace.  The per-tile
 * partial sums live in one library-resident device array for at most 65536 tiles
 * (V * tiles_per_view; larger windows return CGS_ERR_WORKSPACE and launch nothing),
 * held on every GPU that loads the library until the process exits.
 *  - The first call on a device looks up that array's device address (with the device
 *    current) and caches it; make that first call before any stream capture.
 *  - The call allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *  - All calls share the one array, which keeps the last call's contents; each call
 *    writes every entry it reads, so nothing needs clearing, but calls that overlap
 *    on the GPU (different streams, or different host threads) race on it.
 */
int cgs_render_fwd_noalloc(const float *rec, const uint32_t *vals, const uint32_t *ranges,
                           const uint32_t *tile_order, int32_t V, const cgs_config *cfg,
                           const float *view_weight, const float *tgt_rgb, const float *tgt_depth,
                           float *img, float *depth, float *t_final, uint32_t *last, float *loss_view,
                           int32_t *depth_count, int32_t *status_dev, void *stream);

/*
 * cgs_raster_bwd -- backward of the blend (Eqs. 2-4, Sec. III-C.1), pixel-parallel,
 * back to front from `last`, with the transmittance recomputed from the stored
 * final T (T_j = T_{j+1} / (1 - alpha_j)) instead of stored per-pixel lists.  Per
 * blended (splat, pixel) pair, dL/d(u, v, A, B, C, opacity, rgb, depth); the pixels
 * of a warp are summed (in registers per thread, then across the warp through shared
 * memory) before one set of atomic adds per splat into slot_grad, or added by each
 * contributing lane directly when few lanes contribute.  dL/dalpha is zero where alpha
 * was clamped at 0.99.
 * Pixel gradients come either from the fused L1 loss (dl_dimg == NULL: sign of the
 * residual, 0 at 0, times w_v / (3 H W) and w_v lambda_depth / depth_count) or
 * from the caller (dl_dimg float[V][3][H][W], dl_ddepth float[V][H][W] or NULL).
 *   slot_grad  device in/out: accumulated (+=); zeroed by cgs_preprocess
 *   work       device uint32[1] or NULL.  Given, the launch is persistent: as many blocks as
 *              the GPU holds resident take the (view, tile) items, in tile_order, from this
 *              counter (the call sets it to 0 first and leaves the number of items taken plus
 *              the blocks in it).  NULL: one block per item.  Results are the same either way
 *              up to float summation order; calls that share a counter must not overlap.
 */
int cgs_raster_bwd(const float *rec, const uint32_t *vals, const uint32_t *ranges,
                   const uint32_t *tile_order, int32_t V, const cgs_config *cfg,
                   const float *view_weight, const float *img, const float *depth,
                   const float *t_final, const uint32_t *last, const float *tgt_rgb,
                   const float *tgt_depth, const int32_t *depth_count, const float *dl_dimg,
                   const float *dl_ddepth, float *slot_grad, uint32_t *work, int32_t *status_dev,
                   void *stream);

/*
 * Splat-wise backward (Sec. III-C.1 and Fig. 4a: the paper's backward).  The forward
 * saves every pixel's state (transmittance, accumulated colour, accumulated depth)
 * before list positions 32, 64, ... of its tile; the backward gives each warp a bucket
 * of 32 consecutive splats (one per lane), passes pixel states from lane to lane with
 * shuffles, and adds each splat's gradient once per tile (no per-pixel reduction).
 * Results equal cgs_raster_bwd's up to float summation order.
 *   cgs_ckpt_bytes(max_buckets, cfg) = max_buckets * tile^2 * 20 bytes of checkpoints;
 *     a window needs sum over tiles of ceil(len / 32) buckets <= n_inst / 32 + tiles.
 *   cgs_render_fwd_ckpt: cgs_render_fwd plus the checkpoints (its workspace's count of
 *     blended pairs is written as 0 whatever cfg->count_work says).
 *     ckpt          device out, 16-byte aligned, cgs_ckpt_bytes(max_buckets, cfg) bytes
 *     bucket_start  device out, uint32[V * tiles_per_view + 1]: first bucket of each tile
 *     more buckets than max_buckets set CGS_ERR_CAPACITY (checkpoints past it are dropped)
 *   cgs_raster_bwd_splat: cgs_raster_bwd reading those checkpoints (tile 8 or 16).
 */
size_t cgs_ckpt_bytes(int64_t max_buckets, const cgs_config *cfg);
int cgs_render_fwd_ckpt(const float *rec, const uint32_t *vals, const uint32_t *ranges,
                        const uint32_t *tile_order, int32_t V, const cgs_config *cfg,
                        const float *view_weight, const float *tgt_rgb, const float *tgt_depth,
                        float *img, float *depth, float *t_final, uint32_t *last, float *loss_view,
                        int32_t *depth_count, void *workspace, size_t workspace_bytes, float *ckpt,
                        int64_t max_buckets, uint32_t *bucket_start, int32_t *status_dev, void *stream);
int cgs_raster_bwd_splat(const float *rec, const uint32_t *vals, const uint32_t *ranges,
                         const uint32_t *tile_order, int32_t V, const cgs_config *cfg,
                         const float *view_weight, const float *img, const float *depth,
                         const float *t_final, const uint32_t *last, const float *tgt_rgb,
                         const float *tgt_depth, const int32_t *depth_count, const float *dl_dimg,
                         const float *dl_ddepth, const float *ckpt, int64_t max_buckets,
                         const uint32_t *bucket_start, float *slot_grad, int32_t *status_dev,
                         void *stream);

/*
 * cgs_preprocess_bwd -- chain rule from the slot gradients of every visible slot
 * back to the parameters (position, log-scale, quaternion, opacity logit, SH),
 * summed over the V views; the derivative of a guard-band-clamped Jacobian entry
 * and of a clamped colour channel is 0.  When accum/denom/max_r2d are non-NULL
 * the densification statistics of cgs_densify_stats are accumulated in the same
 * pass.
 *   param_grad device float[cgs_param_count]: overwritten (accumulate == 0) or added to
 */
int cgs_preprocess_bwd(const float *params, int64_t n, const cgs_camera *cams, int32_t V,
                       const cgs_config *cfg, const float *rec, const float *slot_grad,
                       float *param_grad, int32_t accumulate, float *accum, float *denom,
                       float *max_r2d, int32_t *status_dev, void *stream);

/* cgs_render_bwd -- cgs_raster_bwd followed by cgs_preprocess_bwd (same arguments). */
int cgs_render_bwd(const float *params, int64_t n, const cgs_camera *cams, int32_t V,
                   const cgs_config *cfg, const float *rec, const uint32_t *vals,
                   const uint32_t *ranges, const uint32_t *tile_order, const float *view_weight,
                   const float *img, const float *depth, const float *t_final,
                   const uint32_t *last, const float *tgt_rgb, const float *tgt_depth,
                   const int32_t *depth_count, const float *dl_dimg, const float *dl_ddepth,
                   float *slot_grad, float *param_grad, int32_t accumulate, float *accum,
                   float *denom, float *max_r2d, uint32_t *work, int32_t *status_dev, void *stream);

/*
 * cgs_densify_stats -- per-Gaussian statistics that guide adaptive densification
 * (Sec. III-A.3 "guided by gradients and the size"; Sec. IV-A densify every 500
 * iterations with tau_p = 0.001): for every visible slot of view v,
 *   accum[g] += || (dL_v/du * W/2, dL_v/dv * H/2) ||   (view-space, NDC units),
 *   denom[g] += 1,  max_r2d[g] = max(max_r2d[g], radius).
 * Uses per-view gradients (slot_grad), never their sum over views.  Accumulates.
 */
int cgs_densify_stats(const float *rec, const float *slot_grad, int64_t n, int32_t V,
                      const cgs_config *cfg, float *accum, float *denom, float *max_r2d,
                      void *stream);

/*
 * cgs_adam -- fused optimiser step on the whole parameter vector (Adam with bias
 * correction, the optimiser of the 3DGS training the paper keeps, Sec. IV-A), with
 * the opacity regulariser of Eqs. 10-11 folded into the gradient:
 *   g <- grad + lambda_o o (1 - o) / n on opacity logits (o = sigmoid(logit)),
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   p <- p - lr_group (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Every element is updated (zero-gradient elements move by momentum).
 *   lr        host float[6]: means, log_scales, quats, opacity, sh_dc, sh_rest
 *   step      >= 1, the step number t used for bias correction, unless step_dev is given
 *   step_dev  device int32 (may be NULL): when given, it is incremented on the device
 *             and its new value is the step t (so a captured CUDA graph advances t at
 *             every replay); `step` is then ignored
 *   loss_o    device float (may be NULL): overwritten with lambda_o * mean(o) of the
 *             parameters before the step (summed with float atomics: the last bits
 *             depend on scheduling)
 * params, grads, m, v: device float[cgs_param_count(n, sh_degree)].
 */
int cgs_adam(float *params, const float *grads, float *m, float *v, int64_t n,
             int32_t sh_degree, const float *lr, float beta1, float beta2, float eps,
             int32_t step, int32_t *step_dev, float lambda_o, float *loss_o, void *stream);

/*
 * Adaptive density control (Sec. III-A.3: cloning and splitting "guided by gradients and
 * the size", pruning transparent Gaussians; Sec. IV-A: tau_p = 0.001, eps_alpha = 0.02,
 * every 500 iterations).  Two calls, so the caller can size the new buffers:
 *   cgs_densify_plan: per Gaussian, in float32, grad = accum / denom (0 where denom = 0),
 *     prune if opacity logit < logit(eps_alpha); otherwise split if grad >= tau_p and the
 *     largest log-scale > log(scale_thr), clone if grad >= tau_p and it is <= log(scale_thr),
 *     else keep.  Thresholds are rounded to float once from the double arguments.  Writes
 *     the plan to the workspace (cgs_densify_workspace(n) bytes, 256-byte aligned) and the
 *     new Gaussian count to *n_out_dev (device int64).
 *   cgs_densify_apply: writes the new parameter vector and Adam moments for n_out
 *     Gaussians, each input Gaussian's outputs consecutive: keep -> itself (its moments);
 *     clone -> itself then a copy (zero moments); split -> two children at
 *     mean + R(q) (s * z_c) with scale s / 1.6, other attributes copied, zero moments;
 *     prune -> nothing.  normals: device float[n][2][3] standard normal samples z_c
 *     (random numbers are inputs).  Outputs must not alias inputs.  The densification
 *     statistics are the caller's to reset (zero) for the new Gaussians.
 */
size_t cgs_densify_workspace(int64_t n);
int cgs_densify_plan(const float *params, int64_t n, int32_t sh_degree, const float *accum,
                     const float *denom, double tau_p, double scale_thr, double eps_alpha,
                     void *workspace, size_t workspace_bytes, int64_t *n_out_dev, void *stream);
int cgs_densify_apply(const float *params, const float *m, const float *v, int64_t n,
                      int32_t sh_degree, const void *workspace, size_t workspace_bytes,
                      const float *normals, int64_t n_out, float *params_out, float *m_out,
                      float *v_out, void *stream);

/*
 * Geometric densification (Sec. III-A.3, III-B): the coloured point cloud of a new keyframe
 * becomes initial Gaussians, initialised as in 3D Gaussian Splatting (the renderer the paper
 * keeps): mean = the point; log-scale = log sqrt(max(d2, 1e-7)) on all three axes, d2 the
 * mean squared distance to the 3 nearest other points (exact; min(3, n_points - 1) of them,
 * none when n_points = 1); rotation (1, 0, 0, 0); opacity logit(init_opacity); SH DC
 * (rgb - 1/2) / Y_0^0; higher bands 0.
 * cgs_points_to_gaussians writes n + n_points Gaussians to params_out / m_out / v_out
 * (layout of cgs_param_count(n + n_points, sh_degree)): Gaussians 0..n-1 copied from
 * params / m / v (NULL allowed when n = 0), then point i as Gaussian n + i with zero Adam
 * moments.  xyz, rgb: device float[n_points][3].  The workspace (cgs_points_workspace(n_points)
 * bytes, 256-byte aligned) holds a uniform grid of the points' bounding box (about one cell
 * per point of its volume, at most 128 cells per axis) and the point ids sorted by cell.
 * Outputs must not alias inputs.  A non-finite coordinate sets CGS_ERR_NONFINITE in
 * *status_dev (that point's outputs are then unspecified).
 */
size_t cgs_points_workspace(int64_t n_points);
int cgs_points_to_gaussians(const float *params, const float *m, const float *v, int64_t n,
                            int32_t sh_degree, const float *xyz, const float *rgb, int64_t n_points,
                            float init_opacity, void *workspace, size_t workspace_bytes,
                            float *params_out, float *m_out, float *v_out, int32_t *status_dev,
                            void *stream);

/*
 * cgs_ssim_loss -- the photometric loss of Eq. 9 with its SSIM term (Sec. III-C.3), plus the
 * depth term, and its pixel gradients for the blend backward (cgs_render_bwd /
 * cgs_raster_bwd / cgs_raster_bwd_splat with dl_dimg, dl_ddepth non-NULL):
 *   loss_view[v] = w_v [ (1 - l) mean|img - tgt| + l (1 - mean SSIM) + lambda_depth
 *                   mean over {tgt_depth > 0} |depth - tgt_depth| ],  l = lambda_ssim in [0, 1]
 * SSIM per pixel and channel from 11x11 Gaussian-window (sigma 1.5) moments with zero
 * padding, C1 = 0.01^2, C2 = 0.03^2 (the 3D Gaussian Splatting loss the paper keeps).
 * img, tgt_rgb: device float[V][3][H][W]; depth, tgt_depth: float[V][H][W] (tgt_depth
 * NULL: no depth term; then depth, depth_count, dl_ddepth are not read or written);
 * depth_count: int32[V] = |{tgt_depth > 0}| per view (cgs_render_fwd writes it);
 * view_weight: float[V] or NULL (all 1).  Writes loss_view float[V] (overwritten),
 * dl_dimg float[V][3][H][W] and dl_ddepth float[V][H][W] (all overwritten).  The
 * workspace (cgs_ssim_workspace(V, cfg) bytes, 256-byte aligned) holds three per-pixel
 * partial-derivative maps and the per-view sums.  Reads only cfg->width, height and
 * lambda_depth.  A non-finite loss sets CGS_ERR_NONFINITE in *status_dev.
 */
size_t cgs_ssim_workspace(int32_t V, const cgs_config *cfg);
int cgs_ssim_loss(const float *img, const float *tgt_rgb, const float *depth,
                  const float *tgt_depth, const int32_t *depth_count, int32_t V,
                  const cgs_config *cfg, const float *view_weight, float lambda_ssim,
                  float *loss_view, float *dl_dimg, float *dl_ddepth, void *workspace,
                  size_t workspace_bytes, int32_t *status_dev, void *stream);

/*
 * Adaptive keyframe scheduler (Eqs. 5-8, Sec. III-C.2), host only.  A pool of
 * keyframes with remaining iteration counts r_i and last losses l_i; a draw picks
 * uniformly (index = rand_u32 mod count, in pool order) among keyframes with
 * r_i > 0 and decrements it; when none is left, r_i = 2 for the d_k = max(1, floor(k/d))
 * largest losses (ties to the lower index) and 1 for the rest.  A new keyframe's
 * loss starts at +infinity.  create/destroy manage host memory only.
 */
typedef struct cgs_scheduler cgs_scheduler;
cgs_scheduler *cgs_sched_create(int32_t d);
void cgs_sched_destroy(cgs_scheduler *s);
int cgs_sched_add(cgs_scheduler *s, int32_t keyframe_id, int32_t r0);  /* returns pool index */
int cgs_sched_draw(cgs_scheduler *s, uint32_t rand_u32);             /* returns pool index */
int cgs_sched_report(cgs_scheduler *s, int32_t index, double loss);
/* n draws in a row, exactly as n calls of cgs_sched_draw with rand_u32[0..n-1]: out[i]
 * receives the i-th pool index.  Returns CGS_OK, or the first error (out is then filled
 * up to that draw).  One call per window instead of one per view keeps the host's share of
 * a training step small. */
int cgs_sched_draw_n(cgs_scheduler *s, const uint32_t *rand_u32, int32_t n, int32_t *out);
/* n reports, exactly as n calls of cgs_sched_report(s, index[i], loss[i]). */
int cgs_sched_report_n(cgs_scheduler *s, const int32_t *index, const double *loss, int32_t n);
/* copies keyframe ids, r and l of the first `cap` pool entries; returns the pool size */
int cgs_sched_state(const cgs_scheduler *s, int32_t *ids, int32_t *r, double *l, int32_t cap);

const char *cgs_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* CGS_H */
