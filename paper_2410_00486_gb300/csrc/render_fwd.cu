// Forward blend of Eq. 1 (Sec. III-B, CaRtGS) with the L1 loss fused in.
//
// One block per (view, tile), one thread per pixel.  The tile's depth-sorted list
// is consumed in batches of BD splats: the block gathers the records of a batch
// into shared memory (one coalesced 48-byte record per thread), then every pixel
// walks the batch front to back.  A block-wide vote (__syncthreads_count) ends the
// walk as soon as every pixel of the tile is saturated (T below 1e-4) or done.
#include "raster.cuh"

namespace cgs {

template <int B, int BD>
__global__ void __launch_bounds__(B *B) k_render_fwd(RasterFwdArgs a)
{
    constexpr int NT = B * B;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[BD], s1[BD], s2[BD];
    __shared__ float red[5][NW > 0 ? NW : 1];
    int64_t tile;
    int view, tx, ty;
    item_tile(a.order, a.g, tile, view, tx, ty);
    const int px = tx * B + (int)(threadIdx.x % B), py = ty * B + (int)(threadIdx.x / B);
    const bool inside = px < a.g.W && py < a.g.H;
    const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
    const float fx = (float)px, fy = (float)py;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    uint32_t lst = 0, n_eval = 0, n_blend = 0;
    bool done = !inside;
    for (uint32_t base = start; base < end; base += BD) {
        if (__syncthreads_count(!done) == 0) break;
        for (int i = threadIdx.x; i < BD; i += NT) {
            const uint32_t idx = base + i;
            if (idx < end) {
                const float4 *r = a.rec + kRec4 * (size_t)__ldg(a.vals + idx);
                s0[i] = __ldg(r);
                s1[i] = __ldg(r + 1);
                s2[i] = __ldg(r + 2);
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BD, end - base);
        if (!done) {
            int j = 0;
            for (; j < cnt; j++) {
                const float4 q0 = s0[j];
                const float4 q1 = s1[j];
                float dx, dy;
                const float power = splat_power(q0.x, q0.y, q0.z, q0.w, q1.x, fx, fy, dx, dy);
                if (power > 0.f) continue;
                const float alpha = fminf(kAlphaMax, __fmul_rn(q1.y, __expf(power)));
                if (alpha < kAlphaMin) continue;
                const float testT = __fmul_rn(T, __fsub_rn(1.f, alpha));
                if (testT < kTMin) {
                    done = true;
                    j++;
                    break;
                }
                const float wgt = __fmul_rn(alpha, T);
                const float4 q2 = s2[j];
                C0 = fmaf(q2.x, wgt, C0);
                C1 = fmaf(q2.y, wgt, C1);
                C2 = fmaf(q2.z, wgt, C2);
                D = fmaf(q1.z, wgt, D);
                T = testT;
                lst = base - start + (uint32_t)j + 1u;
                n_blend++;
            }
            n_eval += (uint32_t)j;
        }
    }

    float l_rgb = 0.f, l_d = 0.f, c_d = 0.f;
    if (inside) {
        const size_t HW = (size_t)a.g.W * a.g.H;
        const size_t p = (size_t)py * a.g.W + px;
        const size_t pix = (size_t)view * HW + p;
        const float I0 = fmaf(T, a.bg0, C0), I1 = fmaf(T, a.bg1, C1), I2 = fmaf(T, a.bg2, C2);
        float *im = a.img + (size_t)view * 3 * HW + p;
        im[0] = I0;
        im[HW] = I1;
        im[2 * HW] = I2;
        a.depth[pix] = D;
        a.tfin[pix] = T;
        a.last[pix] = lst;
        if (a.tgt_rgb) {
            const float *tr = a.tgt_rgb + (size_t)view * 3 * HW + p;
            l_rgb = fabsf(I0 - tr[0]) + fabsf(I1 - tr[HW]) + fabsf(I2 - tr[2 * HW]);
            if (a.tgt_depth) {
                const float td = a.tgt_depth[pix];
                if (td > 0.f) {
                    l_d = fabsf(D - td);
                    c_d = 1.f;
                }
            }
        }
    }
    // per-tile partial sums: loss terms and the work counts (pairs evaluated, pairs blended)
    float f_eval = (float)n_eval, f_blend = (float)n_blend;
    for (int off = 16; off > 0; off >>= 1) {
        l_rgb += __shfl_xor_sync(kFull, l_rgb, off);
        l_d += __shfl_xor_sync(kFull, l_d, off);
        c_d += __shfl_xor_sync(kFull, c_d, off);
        f_eval += __shfl_xor_sync(kFull, f_eval, off);
        f_blend += __shfl_xor_sync(kFull, f_blend, off);
    }
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = l_rgb;
        red[1][w] = l_d;
        red[2][w] = c_d;
        red[3][w] = f_eval;
        red[4][w] = f_blend;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        float acc = 0.f;
        for (int i = 0; i < NW; i++) acc += red[threadIdx.x][i];
        a.partials[kPartials * tile + threadIdx.x] = acc;
    }
}

// Per-view loss from the per-tile partial sums, summed in a fixed order (deterministic):
//   L_v = w_v (sum|r_rgb| / (3 H W) + lambda_d sum|r_d| / count)   (count = valid depth pixels)
__global__ void __launch_bounds__(256)
k_loss_reduce(const float *__restrict__ partials, int64_t Tv, const float *__restrict__ weight, double inv3HW,
              float lambda_d, float *__restrict__ loss_view, int32_t *__restrict__ depth_count,
              int32_t *__restrict__ status)
{
    __shared__ double sh[3][256];
    const int v = blockIdx.x;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t t = threadIdx.x; t < Tv; t += blockDim.x) {
        const float *p = partials + kPartials * ((int64_t)v * Tv + t);
        a0 += p[0];
        a1 += p[1];
        a2 += p[2];
    }
    sh[0][threadIdx.x] = a0;
    sh[1][threadIdx.x] = a1;
    sh[2][threadIdx.x] = a2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double w = weight ? (double)weight[v] : 1.0;
        const double cnt = sh[2][0];
        const double L = w * (sh[0][0] * inv3HW + (cnt > 0.0 ? (double)lambda_d * sh[1][0] / cnt : 0.0));
        loss_view[v] = (float)L;
        depth_count[v] = (int32_t)cnt;
        if (!isfinite(L)) set_status(status, CGS_ERR_NONFINITE);
    }
}

template <int B, int BD>
static cudaError_t launch_fwd(const RasterFwdArgs &a, cudaStream_t s)
{
    const int64_t items = a.g.Tv * a.V;
    k_render_fwd<B, BD><<<(unsigned)items, B * B, 0, s>>>(a);
    return cudaGetLastError();
}

template <int B>
static cudaError_t launch_fwd_bd(const RasterFwdArgs &a, int BD, cudaStream_t s)
{
    switch (BD) {
    case 32: return launch_fwd<B, 32>(a, s);
    case 64: return launch_fwd<B, 64>(a, s);
    case 128: return launch_fwd<B, 128>(a, s);
    default: return launch_fwd<B, 256>(a, s);
    }
}

cudaError_t raster_fwd(const RasterFwdArgs &a, int B, int BD, cudaStream_t s)
{
    switch (B) {
    case 8: return launch_fwd_bd<8>(a, BD, s);
    case 16: return launch_fwd_bd<16>(a, BD, s);
    default: return launch_fwd_bd<32>(a, BD, s);
    }
}

cudaError_t loss_reduce(const float *partials, const Grid &g, int V, const float *weight, float lambda_d,
                        float *loss_view, int32_t *depth_count, int32_t *status, cudaStream_t s)
{
    const double inv3HW = 1.0 / (3.0 * (double)g.W * (double)g.H);
    k_loss_reduce<<<V, 256, 0, s>>>(partials, g.Tv, weight, inv3HW, lambda_d, loss_view, depth_count, status);
    return cudaGetLastError();
}

}  // namespace cgs
