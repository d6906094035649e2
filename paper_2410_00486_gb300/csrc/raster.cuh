// Arguments of the raster kernels (forward blend + fused loss, backward blend).
#pragma once

#include "cgs_internal.cuh"

namespace cgs {

struct RasterFwdArgs {
    const float4 *rec;
    const uint32_t *vals, *ranges, *order;
    Grid g;
    int V;
    float bg0, bg1, bg2;
    const float *tgt_rgb, *tgt_depth;
    float *img, *depth, *tfin;
    uint32_t *last;
    float *partials;   // [Ttot][kPartials], see below
};

// Per-tile partial sums written by the forward: sum |r_rgb|, sum |r_depth| over valid
// depth pixels, valid depth count, (splat, pixel) pairs evaluated, pairs blended.
constexpr int kPartials = 5;

struct RasterBwdArgs {
    const float4 *rec;
    const uint32_t *vals, *ranges, *order;
    Grid g;
    int V;
    float bg0, bg1, bg2;
    const float *weight;
    const float *img, *depth, *tfin;
    const uint32_t *last;
    const float *tgt_rgb, *tgt_depth;
    const int32_t *depth_count;
    float lambda_d;
    const float *dl_dimg, *dl_ddepth;
    float *sgrad;
};

// Map a work item to (view, tile x, tile y).
__device__ __forceinline__ void item_tile(const uint32_t *order, const Grid &g, int64_t &tile, int &view, int &tx,
                                          int &ty)
{
    tile = order ? (int64_t)order[blockIdx.x] : (int64_t)blockIdx.x;
    view = (int)(tile / g.Tv);
    const int t = (int)(tile - (int64_t)view * g.Tv);
    ty = t / g.Tx;
    tx = t - ty * g.Tx;
}

cudaError_t raster_fwd(const RasterFwdArgs &a, int B, int BD, cudaStream_t s);
cudaError_t raster_bwd(const RasterBwdArgs &a, int B, int BD, cudaStream_t s);

}  // namespace cgs
