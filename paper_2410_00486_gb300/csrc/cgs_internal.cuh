// Internal helpers shared by the libcgs kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cgs.h"

namespace cgs {

constexpr int kRec4 = 3;             // float4s per record / slot gradient (12 floats)
constexpr unsigned kFull = 0xffffffffu;

// Layout of the flat parameter vector (see cgs.h).
struct Layout {
    int64_t means, scales, quats, opac, dc, rest, total;
    int K;
};

__host__ __device__ inline Layout param_layout(int64_t n, int deg)
{
    Layout L;
    L.K = (deg + 1) * (deg + 1);
    L.means = 0;
    L.scales = 3 * n;
    L.quats = 6 * n;
    L.opac = 10 * n;
    L.dc = 11 * n;
    L.rest = 14 * n;
    L.total = 14 * n + 3 * (int64_t)(L.K - 1) * n;
    return L;
}

// Record a device-side condition; the first one wins.
__device__ __forceinline__ void set_status(int32_t *st, int code)
{
    if (st) atomicCAS(st, 0, code);
}

// Argument checks shared by every entry point that takes a cgs_config (host code).
constexpr int kMaxViews = 1024;

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

inline bool cfg_ok(const cgs_config *c)
{
    if (!c) return false;
    if (c->width < 1 || c->height < 1 || c->width > (1 << 16) || c->height > (1 << 16)) return false;
    if (c->tile != 8 && c->tile != 16 && c->tile != 32) return false;
    if (c->batch_depth != 32 && c->batch_depth != 64 && c->batch_depth != 128 && c->batch_depth != 256) return false;
    if (c->batch_depth_bwd != 0 && c->batch_depth_bwd != 32 && c->batch_depth_bwd != 64 &&
        c->batch_depth_bwd != 128 && c->batch_depth_bwd != 256)
        return false;
    if (c->sh_degree < 0 || c->sh_degree > 3) return false;
    if (!(c->near_z > 0.f) || !isfinite(c->near_z)) return false;
    return true;
}

// Geometry of the tile grid, passed by value to kernels.
struct Grid {
    int W, H, B, log2B, Tx, Ty;
    int64_t Tv;      // tiles per view
    int rect_lists;  // binning: list a slot in every tile of its rect (no reach test)
};

inline int ilog2(int x)
{
    int l = 0;
    while ((1 << l) < x) l++;
    return l;
}

inline Grid make_grid(const cgs_config &c)
{
    Grid g;
    g.W = c.width;
    g.H = c.height;
    g.B = c.tile;
    g.log2B = ilog2(c.tile);
    g.Tx = (c.width + c.tile - 1) / c.tile;
    g.Ty = (c.height + c.tile - 1) / c.tile;
    g.Tv = (int64_t)g.Tx * g.Ty;
    g.rect_lists = c.rect_lists != 0;
    return g;
}

// Tile rectangle of a splat: [x0, x1) x [y0, y1) in tile units.  Since r and B are
// integers, floor((u - r)/B) = floor((floor(u) - r)/B), so only floor(u) enters and the
// result is exact; B is a power of two, so floor division is an arithmetic shift.
struct Rect { int x0, x1, y0, y1; };

__device__ __forceinline__ Rect tile_rect(float u, float v, int r, const Grid &g)
{
    // keep the integer conversion in range for far off-screen centres
    int fu = (int)fminf(fmaxf(floorf(u), -1.0e8f), 1.0e8f);
    int fv = (int)fminf(fmaxf(floorf(v), -1.0e8f), 1.0e8f);
    Rect R;
    R.x0 = min(max((fu - r) >> g.log2B, 0), g.Tx);
    R.x1 = min(max((fu + r + g.B - 1) >> g.log2B, 0), g.Tx);
    R.y0 = min(max((fv - r) >> g.log2B, 0), g.Ty);
    R.y1 = min(max((fv + r + g.B - 1) >> g.log2B, 0), g.Ty);
    return R;
}

// Whether a projected splat can reach alpha >= 1/255 at a pixel centre of the box
// [bx0, bx1] x [by0, by1]: tile lists keep a slot only in such tiles of its rect.  Every
// operation is one IEEE rounding (explicit intrinsics, no contraction), so the decision is
// a fixed function of the float32 record: tau = -ln(255 o) > 1e-4 (o < 1/255, with a
// margin) reaches nothing; det <= 0 reaches everything; otherwise alpha >= 1/255 needs
// q = A dx^2 + 2 B dx dy + C dy^2 <= -2 tau, widened to t2 = (-2 tau) 1.001 + 1e-3.  The
// ellipse's bounding box (half-extents sqrt(t2 C / det) + 0.01, sqrt(t2 A / det) + 0.01)
// is tested first; then, with the centre outside the box, the minimum of q over the box,
// which lies on an edge where q is a parabola minimised at its clamped vertex.  The
// margins exceed the float32 error of the raster's per-pixel test (power < tau skips)
// unless the exponent's terms cancel by many orders of magnitude (a splat thousands of
// pixels long and under a pixel wide), so a splat left out of a tile is one every pixel
// of the tile would skip.
__device__ __forceinline__ float edge_q(float A, float B2, float C, float ddx, float ddy)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A, ddx), ddx), __fmul_rn(__fmul_rn(B2, ddx), ddy)),
                     __fmul_rn(__fmul_rn(C, ddy), ddy));
}

// The per-splat part of the reach test (one division and square root each), computed once
// per slot; reach_box finishes it for a box.
struct ReachPre {
    float A, B2, C, t2, ex, ey, bc, ba;
    int mode;   // 0 reaches nothing, 1 reaches everything, 2 test the box
};
__device__ __forceinline__ ReachPre reach_prepare(float A, float B, float C, float tau)
{
    ReachPre p{A, __fmul_rn(2.f, B), C, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
    if (!(tau <= 1e-4f)) return p;
    const float det = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
    if (!(det > 0.f)) {
        p.mode = 1;
        return p;
    }
    p.mode = 2;
    p.t2 = __fadd_rn(__fmul_rn(__fmul_rn(-2.f, tau), 1.001f), 1e-3f);
    p.ex = __fadd_rn(__fsqrt_rn(__fdiv_rn(__fmul_rn(p.t2, C), det)), 1e-2f);
    p.ey = __fadd_rn(__fsqrt_rn(__fdiv_rn(__fmul_rn(p.t2, A), det)), 1e-2f);
    p.bc = __fdiv_rn(B, C);
    p.ba = __fdiv_rn(B, A);
    return p;
}
__device__ __forceinline__ bool reach_box(const ReachPre &p, float u, float v, float bx0, float bx1, float by0,
                                          float by1)
{
    // computed without early returns (the lanes of a warp test different tiles): the box
    // check, the centre inside the box, and the minimum over the edges facing the centre
    const float ddx0 = __fsub_rn(u, fminf(fmaxf(u, bx0), bx1));
    const float ddy1 = __fsub_rn(v, fminf(fmaxf(v, by0), by1));
    const float dx = fabsf(ddx0), dy = fabsf(ddy1);
    // q is convex with its minimum at the centre, outside the box: its minimum over the box
    // lies on an edge facing the centre, the vertical edge at the clamped x or the
    // horizontal edge at the clamped y (where the centre is inside the box's x (y) range,
    // that "edge" evaluation gives q at a point of the box, which is no lower than the
    // minimum)
    const float ddy0 = fminf(fmaxf(-__fmul_rn(p.bc, ddx0), __fsub_rn(v, by1)), __fsub_rn(v, by0));
    const float ddx1 = fminf(fmaxf(-__fmul_rn(p.ba, ddy1), __fsub_rn(u, bx1)), __fsub_rn(u, bx0));
    const bool edge = fminf(edge_q(p.A, p.B2, p.C, ddx0, ddy0), edge_q(p.A, p.B2, p.C, ddx1, ddy1)) <= p.t2;
    const bool reach = dx <= p.ex && dy <= p.ey && ((dx == 0.f && dy == 0.f) || edge);
    return p.mode == 2 ? reach : p.mode == 1;
}

constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

}  // namespace cgs
