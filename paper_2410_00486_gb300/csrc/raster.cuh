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
    uint32_t *work;   // persistent launch: the work counter (null: one block per tile)
};

// Map a work item (a block index, or an item taken from a work counter) to (view, tile x,
// tile y).
__device__ __forceinline__ void item_tile(const uint32_t *order, const Grid &g, int64_t &tile, int &view, int &tx,
                                          int &ty, uint32_t item)
{
    tile = order ? (int64_t)order[item] : (int64_t)item;
    view = (int)(tile / g.Tv);
    const int t = (int)(tile - (int64_t)view * g.Tv);
    ty = t / g.Tx;
    tx = t - ty * g.Tx;
}

// Pixels per thread in the raster kernels: a thread owns several pixels of one column, so
// the staged splat is read from shared memory once for PPT pixels and the backward's
// per-(warp, splat) reduction covers 32*PPT pixels.
// The forward keeps two (its per-thread state is small and occupancy pays; four measured
// slower), the backward eight: one warp per 16x16 tile, half the warp reductions per pixel
// of four pixels, which were a third of its time (3.84 vs 4.04 ms on the 16-view window).
constexpr int kPPTFwd = 2;
constexpr int kPPTBwd = 8;

// Pixels per thread for tile edge B: P, but at least one full warp per tile.
template <int B, int P>
__host__ __device__ constexpr int ppt_for()
{
    return (B * B / P >= 32) ? P : (B * B / 32);
}

// Tile row (0..B-1) of a thread's first pixel; its pixel p lies G p rows further down,
// G = 32 / B the number of B-wide row groups a warp spans.  The warp's pixels with the
// same p thus form a block of G adjacent rows (B = 16: rows 2p and 2p + 1 of the warp's
// rows), so a splat that covers few rows leaves whole p-steps of the warp idle; with
// consecutive rows per thread every p-step would hold rows spread over the warp's span.
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
// blocks): the register budget is 64K / (warps x 32).  The forward runs at 32 warps (64
// registers, 56 used; 36 or 40 gain nothing).  The backward keeps the per-pixel loss
// gradients in shared memory (read once per blended pixel) and runs at 28 warps (72
// registers): measured on the 16-view window with 32-splat batches, 20 warps (all state in
// registers, 96 registers) 3.76 ms, 26 warps 3.58, 28 warps 3.58, 30 and 32 warps (which
// spill) 4.47 and 4.46 ms.
constexpr int kFwdMinWarps = 32;
constexpr int kBwdMinWarps = 28;
template <int B, int P, int MinWarps>
__host__ __device__ constexpr int min_blocks_for()
{
    return MinWarps / (B * B / ppt_for<B, P>() / 32) > 0 ? MinWarps / (B * B / ppt_for<B, P>() / 32) : 1;
}

// Staged splat, derived from its record with the exponent in base 2 (every term scaled
// by log2 e, one rounding each), so alpha = opacity 2^power2 takes the hardware's base-2
// exponential (PTX ex2.approx) and no multiply per pair:
//   s0 = (u, v, -A/2 L, -B L), s1 = (-C/2 L, opacity, depth, -tau L),  L = log2 e,
// where tau = -ln(255 opacity) < 0: alpha = opacity exp(power) < 1/255 exactly when
// power < tau.  The exponent of a positive-definite conic is at most 0, so a pair can
// blend exactly when |power| <= -tau: one compare per pair (a rounded power a hair above 0,
// at a pixel within rounding of the splat's centre, counts as 0, where the exact power
// lies); the exponential is evaluated only for pairs that pass.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
__device__ __forceinline__ void stage_splat(const float4 &r0, const float4 &r1, float tau, float4 &t0, float4 &t1)
{
    t0 = make_float4(r0.x, r0.y, __fmul_rn(r0.z, -0.5f * kLog2e), __fmul_rn(r0.w, -kLog2e));
    t1 = make_float4(__fmul_rn(r1.x, -0.5f * kLog2e), r1.y, r1.z, __fmul_rn(tau, -kLog2e));
}

// 1/x (PTX rcp.approx.ftz) for x = 1 - alpha in [0.01, 1].
__device__ __forceinline__ float rcp_fast(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2^x (PTX ex2.approx.ftz; |x| is at most -tau L < 9 here, so nothing is flushed).
__device__ __forceinline__ float exp2_fast(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exponent of the projected Gaussian at a pixel from a staged splat (in base-2 units, the
// staged terms carrying log2 e), with explicit roundings so every raster kernel computes
// the same bits:
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
