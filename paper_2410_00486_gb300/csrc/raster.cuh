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
    // optional checkpoints for the splat-wise backward (null = none): the state of every
    // pixel before list positions 32, 64, ... of its tile
    float4 *ck4;                 // [bucket][B*B] (T, C0, C1, C2)
    float *ckD;                  // [bucket][B*B] depth
    const uint32_t *bucket_start;  // [Ttot + 1] first bucket of each tile
    int64_t max_buckets;
    bool count_blend;              // count blended pairs (partial 4); else it is written as 0
};

// Checkpoint bucket of list positions [32 k, 32 k + 32) of a tile.
constexpr int kBucket = 32;

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

// Pixels per thread in the raster kernels: a thread owns several vertically adjacent pixels,
// so the staged splat is read from shared memory once for PPT pixels and the backward's
// per-(warp, splat) reduction covers 32*PPT pixels.
// The forward keeps two (its per-thread state is small and occupancy pays), the
// backward four (fewer warp reductions per pixel).
constexpr int kPPTFwd = 2;
constexpr int kPPTBwd = 4;

// Pixels per thread for tile edge B: P, but at least one full warp per tile.
template <int B, int P>
__host__ __device__ constexpr int ppt_for()
{
    return (B * B / P >= 32) ? P : (B * B / 32);
}

// Tile row (0..B-1) of a thread's first pixel; its pixel p lies G p rows further down,
// G = 32 / B the number of B-wide row groups a warp spans.  The warp's pixels with the
// same p thus form a block of G adjacent rows (B = 16: rows 2p, 2p + 1 of the warp's
// eight), so a splat that covers few rows leaves whole p-steps of the warp idle, where
// rows p, p + 4 (consecutive rows per thread) would keep every p-step busy.
template <int B, int P>
__device__ __forceinline__ int thread_row0()
{
    constexpr int G = B >= 32 ? 1 : 32 / B;
    const int grp = (int)threadIdx.x / B;
    return (grp / G) * G * P + grp % G;
}
template <int B>
__host__ __device__ constexpr int row_step()
{
    return B >= 32 ? 1 : 32 / B;
}

// Resident warps per SM each raster kernel is compiled for (__launch_bounds__ minimum
// blocks): the register budget is 64K / (warps x 32), 64 registers at 32 warps.  Both
// kernels are latency-bound and gain from more resident warps than their natural
// register counts allow; the backward spills at 36 warps (56 registers) and measured
// slower there (5.15 vs 4.88 ms on the 16-view window).
constexpr int kFwdMinWarps = 32;
constexpr int kBwdMinWarps = 32;
template <int B, int P, int MinWarps>
__host__ __device__ constexpr int min_blocks_for()
{
    return MinWarps / (B * B / ppt_for<B, P>() / 32) > 0 ? MinWarps / (B * B / ppt_for<B, P>() / 32) : 1;
}

// Staged splat, derived exactly from its record (negation and scaling by 1/2 are exact):
//   s0 = (u, v, -A/2, -B), s1 = (-C/2, opacity, depth, tau), s2 = (r, g, b, -)
// where tau = -ln(255 opacity): alpha = opacity exp(power) < 1/255 exactly when
// power < tau, so both raster kernels test the exponent against tau and evaluate the
// exponential only for pairs that can blend.
__device__ __forceinline__ void stage_splat(const float4 &r0, const float4 &r1, float tau, float4 &t0, float4 &t1)
{
    t0 = make_float4(r0.x, r0.y, -0.5f * r0.z, -r0.w);
    t1 = make_float4(-0.5f * r1.x, r1.y, r1.z, tau);
}

// Exponent of the projected Gaussian at a pixel from a staged splat, with explicit
// roundings so every raster kernel computes the same bits:
//   power = (-A/2 dx) dx + dy ((-C/2) dy + (-B) dx),  dx = u - x, dy = v - y.
// The dx terms are shared by the pixels of a column: power_x gives them once, and
// power_at finishes a pixel with two fused multiply-adds.
struct PowerX {
    float a, b;   // (-A/2 dx) dx and (-B) dx
};
__device__ __forceinline__ PowerX power_x(const float4 &t0, float dx)
{
    return PowerX{__fmul_rn(__fmul_rn(t0.z, dx), dx), __fmul_rn(t0.w, dx)};
}
__device__ __forceinline__ float power_at(const PowerX &x, float hC, float dy)
{
    return fmaf(dy, fmaf(hC, dy, x.b), x.a);
}
__device__ __forceinline__ float staged_power(const float4 &t0, float hC, float dx, float dy)
{
    return power_at(power_x(t0, dx), hC, dy);
}

cudaError_t raster_fwd(const RasterFwdArgs &a, int B, int BD, cudaStream_t s);
cudaError_t raster_bwd(const RasterBwdArgs &a, int B, int BD, cudaStream_t s);

}  // namespace cgs
