// Internal helpers shared by the libcgs kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
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

// Geometry of the tile grid, passed by value to kernels.
struct Grid {
    int W, H, B, log2B, Tx, Ty;
    int64_t Tv;   // tiles per view
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

// Exponent of the projected 2-D Gaussian at a pixel, written with explicit
// roundings so the forward and backward kernels take bit-identical decisions:
//   power = dx (-A/2 dx - B dy) + (-C/2 dy) dy,  (dx, dy) = (u - x, v - y).
__device__ __forceinline__ float splat_power(float u, float v, float A, float B, float C,
                                             float px, float py, float &dx, float &dy)
{
    dx = __fsub_rn(u, px);
    dy = __fsub_rn(v, py);
    float t = fmaf(-0.5f * A, dx, __fmul_rn(-B, dy));
    float s = __fmul_rn(__fmul_rn(-0.5f * C, dy), dy);
    return fmaf(dx, t, s);
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

}  // namespace cgs
