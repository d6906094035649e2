// C ABI of libcgs (declared in include/cgs.h): argument validation and launches.
#include <math.h>
#include <stdio.h>

#include "raster.cuh"

namespace cgs {
cudaError_t preprocess_fwd(const float *P, int64_t n, int deg, const cgs_camera *cams, int V, const Grid &g,
                           float near_z, float *rec, float *sgrad, cudaStream_t s);
cudaError_t preprocess_bwd(const float *P, int64_t n, int deg, const cgs_camera *cams, int V, const Grid &g,
                           float near_z, const float *rec, const float *sgrad, float *pgrad, int accumulate,
                           float *accum, float *denom, float *maxr, cudaStream_t s);
size_t bin_ws_bytes(int64_t capacity, int64_t n, int64_t V, int64_t Tv, int num_sms);
cudaError_t bin_sort(const float *rec, int64_t n, int V, const Grid &g, void *ws, int64_t capacity, uint32_t *vals,
                     uint32_t *ranges, uint32_t *order, int64_t *n_inst, int32_t *status, int num_sms,
                     cudaStream_t s);
cudaError_t loss_reduce(const float *partials, const Grid &g, int V, const float *weight, float lambda_d,
                        float *loss_view, int32_t *depth_count, int32_t *status, cudaStream_t s);
cudaError_t adam(float *p, const float *g, float *m, float *v, int64_t n, int deg, const float *lr, float b1,
                 float b2, float eps, int step, int32_t *step_dev, float lambda_o, float *loss_o, int num_sms,
                 cudaStream_t s);
cudaError_t densify_stats(const float *rec, const float *sgrad, int64_t n, int V, const Grid &g, float *accum,
                          float *denom, float *maxr, int num_sms, cudaStream_t s);
}  // namespace cgs

using namespace cgs;

namespace {

bool sizes_ok(int64_t n, int32_t V, const cgs_config *c)
{
    if (n < 1 || V < 1 || V > kMaxViews) return false;
    if ((int64_t)V * n >= (int64_t)1 << 32) return false;
    Grid g = make_grid(*c);
    if (g.Tv * V >= ((int64_t)1 << 31)) return false;
    return true;
}

int num_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 132;
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
    if (dev >= 0 && dev < 64) cache[dev] = v;
    return v;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return CGS_OK;
    fprintf(stderr, "libcgs: CUDA error: %s\n", cudaGetErrorString(e));
    return CGS_ERR_CUDA;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int64_t cgs_param_count(int64_t n, int32_t sh_degree)
{
    if (n < 0 || sh_degree < 0 || sh_degree > 3) return -1;
    return param_layout(n, sh_degree).total;
}

int64_t cgs_tiles_per_view(const cgs_config *cfg)
{
    if (!cfg_ok(cfg)) return -1;
    return make_grid(*cfg).Tv;
}

int cgs_preprocess(const float *params, int64_t n, const cgs_camera *cams, int32_t V, const cgs_config *cfg,
                   float *rec, float *slot_grad, int32_t *status_dev, void *stream)
{
    (void)status_dev;
    if (!params || !cams || !rec || !cfg_ok(cfg) || !sizes_ok(n, V, cfg)) return CGS_ERR_ARG;
    if (!aligned16(rec) || (slot_grad && !aligned16(slot_grad)) || !aligned16(cams)) return CGS_ERR_ARG;
    Grid g = make_grid(*cfg);
    return cuda_status(preprocess_fwd(params, n, cfg->sh_degree, cams, V, g, cfg->near_z, rec, slot_grad,
                                      (cudaStream_t)stream));
}

size_t cgs_bin_sort_workspace(int64_t capacity, int64_t n, int32_t V, const cgs_config *cfg)
{
    if (!cfg_ok(cfg) || V < 1 || capacity < 0 || n < 1) return 0;
    return bin_ws_bytes(capacity, n, V, make_grid(*cfg).Tv, num_sms());
}

int cgs_bin_sort(const float *rec, int64_t n, int32_t V, const cgs_config *cfg, void *workspace,
                 size_t workspace_bytes, int64_t capacity, uint32_t *vals, uint32_t *ranges, uint32_t *tile_order,
                 int64_t *n_inst_dev, int32_t *status_dev, void *stream)
{
    if (!rec || !workspace || !ranges || !n_inst_dev || !cfg_ok(cfg) || !sizes_ok(n, V, cfg)) return CGS_ERR_ARG;
    if (capacity < 0 || capacity > 0xffffffffll || (capacity > 0 && !vals)) return CGS_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0 || !aligned16(rec)) return CGS_ERR_ARG;
    Grid g = make_grid(*cfg);
    if (workspace_bytes < bin_ws_bytes(capacity, n, V, g.Tv, num_sms())) return CGS_ERR_WORKSPACE;
    return cuda_status(bin_sort(rec, n, V, g, workspace, capacity, vals, ranges, tile_order, n_inst_dev,
                                status_dev, num_sms(), (cudaStream_t)stream));
}

size_t cgs_render_fwd_workspace(int32_t V, const cgs_config *cfg)
{
    if (!cfg_ok(cfg) || V < 1) return 0;
    return align256(sizeof(float) * kPartials * (size_t)make_grid(*cfg).Tv * V);
}

int cgs_render_fwd(const float *rec, const uint32_t *vals, const uint32_t *ranges, const uint32_t *tile_order,
                   int32_t V, const cgs_config *cfg, const float *view_weight, const float *tgt_rgb,
                   const float *tgt_depth, float *img, float *depth, float *t_final, uint32_t *last,
                   float *loss_view, int32_t *depth_count, void *workspace, size_t workspace_bytes,
                   int32_t *status_dev, void *stream)
{
    if (!rec || !vals || !ranges || !img || !depth || !t_final || !last || !cfg_ok(cfg)) return CGS_ERR_ARG;
    if (V < 1 || V > kMaxViews || !aligned16(rec)) return CGS_ERR_ARG;
    if (tgt_depth && !tgt_rgb) return CGS_ERR_ARG;
    if (tgt_rgb && (!loss_view || !depth_count)) return CGS_ERR_ARG;
    if (!workspace) return CGS_ERR_ARG;
    if (workspace_bytes < cgs_render_fwd_workspace(V, cfg)) return CGS_ERR_WORKSPACE;
    Grid g = make_grid(*cfg);
    if (g.Tv * V >= ((int64_t)1 << 31)) return CGS_ERR_ARG;
    RasterFwdArgs a;
    a.rec = reinterpret_cast<const float4 *>(rec);
    a.vals = vals;
    a.ranges = ranges;
    a.order = tile_order;
    a.g = g;
    a.V = V;
    a.bg0 = cfg->bg[0];
    a.bg1 = cfg->bg[1];
    a.bg2 = cfg->bg[2];
    a.tgt_rgb = tgt_rgb;
    a.tgt_depth = tgt_depth;
    a.img = img;
    a.depth = depth;
    a.tfin = t_final;
    a.last = last;
    a.partials = static_cast<float *>(workspace);
    a.ck4 = nullptr;
    a.ckD = nullptr;
    a.bucket_start = nullptr;
    a.max_buckets = 0;
    a.count_blend = cfg->count_work != 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = raster_fwd(a, cfg->tile, cfg->batch_depth, s);
    if (e == cudaSuccess && tgt_rgb)
        e = loss_reduce(a.partials, g, V, view_weight, cfg->lambda_depth, loss_view, depth_count, status_dev, s);
    return cuda_status(e);
}

int cgs_raster_bwd(const float *rec, const uint32_t *vals, const uint32_t *ranges, const uint32_t *tile_order,
                   int32_t V, const cgs_config *cfg, const float *view_weight, const float *img, const float *depth,
                   const float *t_final, const uint32_t *last, const float *tgt_rgb, const float *tgt_depth,
                   const int32_t *depth_count, const float *dl_dimg, const float *dl_ddepth, float *slot_grad,
                   uint32_t *work, int32_t *status_dev, void *stream)
{
    (void)status_dev;
    if (!rec || !vals || !ranges || !t_final || !last || !slot_grad || !cfg_ok(cfg)) return CGS_ERR_ARG;
    if (V < 1 || V > kMaxViews || !aligned16(rec) || !aligned16(slot_grad)) return CGS_ERR_ARG;
    if (!dl_dimg && (!tgt_rgb || !img)) return CGS_ERR_ARG;
    if (!dl_dimg && tgt_depth && (!depth || !depth_count)) return CGS_ERR_ARG;
    Grid g = make_grid(*cfg);
    if (g.Tv * V >= ((int64_t)1 << 31)) return CGS_ERR_ARG;
    RasterBwdArgs a;
    a.rec = reinterpret_cast<const float4 *>(rec);
    a.vals = vals;
    a.ranges = ranges;
    a.order = tile_order;
    a.g = g;
    a.V = V;
    a.bg0 = cfg->bg[0];
    a.bg1 = cfg->bg[1];
    a.bg2 = cfg->bg[2];
    a.weight = view_weight;
    a.img = img;
    a.depth = depth;
    a.tfin = t_final;
    a.last = last;
    a.tgt_rgb = tgt_rgb;
    a.tgt_depth = dl_dimg ? nullptr : tgt_depth;
    a.depth_count = depth_count;
    a.lambda_d = cfg->lambda_depth;
    a.dl_dimg = dl_dimg;
    a.dl_ddepth = dl_ddepth;
    a.sgrad = slot_grad;
    a.work = work;
    const int bd = cfg->batch_depth_bwd ? cfg->batch_depth_bwd : cfg->batch_depth;
    return cuda_status(raster_bwd(a, cfg->tile, bd, (cudaStream_t)stream));
}

int cgs_preprocess_bwd(const float *params, int64_t n, const cgs_camera *cams, int32_t V, const cgs_config *cfg,
                       const float *rec, const float *slot_grad, float *param_grad, int32_t accumulate, float *accum,
                       float *denom, float *max_r2d, int32_t *status_dev, void *stream)
{
    (void)status_dev;
    if (!params || !cams || !rec || !slot_grad || !param_grad || !cfg_ok(cfg) || !sizes_ok(n, V, cfg))
        return CGS_ERR_ARG;
    if (!aligned16(rec) || !aligned16(slot_grad) || !aligned16(cams)) return CGS_ERR_ARG;
    if ((accum || denom || max_r2d) && !(accum && denom && max_r2d)) return CGS_ERR_ARG;
    Grid g = make_grid(*cfg);
    return cuda_status(preprocess_bwd(params, n, cfg->sh_degree, cams, V, g, cfg->near_z, rec, slot_grad,
                                      param_grad, accumulate, accum, denom, max_r2d, (cudaStream_t)stream));
}

int cgs_render_bwd(const float *params, int64_t n, const cgs_camera *cams, int32_t V, const cgs_config *cfg,
                   const float *rec, const uint32_t *vals, const uint32_t *ranges, const uint32_t *tile_order,
                   const float *view_weight, const float *img, const float *depth, const float *t_final,
                   const uint32_t *last, const float *tgt_rgb, const float *tgt_depth, const int32_t *depth_count,
                   const float *dl_dimg, const float *dl_ddepth, float *slot_grad, float *param_grad,
                   int32_t accumulate, float *accum, float *denom, float *max_r2d, uint32_t *work,
                   int32_t *status_dev, void *stream)
{
    if (!params || !cams || !param_grad || !cfg_ok(cfg) || !sizes_ok(n, V, cfg)) return CGS_ERR_ARG;
    int st = cgs_raster_bwd(rec, vals, ranges, tile_order, V, cfg, view_weight, img, depth, t_final, last, tgt_rgb,
                            tgt_depth, depth_count, dl_dimg, dl_ddepth, slot_grad, work, status_dev, stream);
    if (st != CGS_OK) return st;
    return cgs_preprocess_bwd(params, n, cams, V, cfg, rec, slot_grad, param_grad, accumulate, accum, denom,
                              max_r2d, status_dev, stream);
}

int cgs_densify_stats(const float *rec, const float *slot_grad, int64_t n, int32_t V, const cgs_config *cfg,
                      float *accum, float *denom, float *max_r2d, void *stream)
{
    if (!rec || !slot_grad || !accum || !denom || !max_r2d || !cfg_ok(cfg) || !sizes_ok(n, V, cfg))
        return CGS_ERR_ARG;
    if (!aligned16(rec) || !aligned16(slot_grad)) return CGS_ERR_ARG;
    Grid g = make_grid(*cfg);
    return cuda_status(densify_stats(rec, slot_grad, n, V, g, accum, denom, max_r2d, num_sms(), (cudaStream_t)stream));
}

int cgs_adam(float *params, const float *grads, float *m, float *v, int64_t n, int32_t sh_degree, const float *lr,
             float beta1, float beta2, float eps, int32_t step, int32_t *step_dev, float lambda_o, float *loss_o,
             void *stream)
{
    if (!params || !grads || !m || !v || !lr || n < 1 || sh_degree < 0 || sh_degree > 3) return CGS_ERR_ARG;
    if (!step_dev && step < 1) return CGS_ERR_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f)) return CGS_ERR_ARG;
    return cuda_status(adam(params, grads, m, v, n, sh_degree, lr, beta1, beta2, eps, step, step_dev, lambda_o,
                            loss_o, num_sms(), (cudaStream_t)stream));
}

const char *cgs_status_string(int status)
{
    switch (status) {
    case CGS_OK: return "ok";
    case CGS_ERR_ARG: return "invalid argument";
    case CGS_ERR_WORKSPACE: return "workspace too small";
    case CGS_ERR_CUDA: return "CUDA launch error";
    case CGS_ERR_CAPACITY: return "tile instance capacity exceeded (lists truncated)";
    case CGS_ERR_NONFINITE: return "non-finite loss";
    case CGS_ERR_TIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
    }
}

}  // extern "C"
