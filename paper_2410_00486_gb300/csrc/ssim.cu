// Photometric loss of Eq. 9 (Sec. III-C.3, CaRtGS) with its SSIM term:
//   L_v = w_v [ (1 - l) mean |img - tgt| + l (1 - mean SSIM(img, tgt)) + lambda_d mean_valid |D - D*| ]
// and its pixel gradients, for the raster backward's pixel-gradient input.
//
// SSIM per pixel and channel from window means (11x11 Gaussian, sigma 1.5, zero padding):
//   S = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx + sy + C2)),
//   sx = E[x^2] - mx^2, sy = E[y^2] - my^2, sxy = E[xy] - mx my.
// dS/dx at pixel q gathers, through the window, dS/dmx, dS/dE[x^2] and dS/dE[xy] of every
// pixel p whose window covers q:  dL/dx(q) = -(l / M) [ G*a + 2 x G*b + y G*c ](q),
// M = 3 H W, with a, b, c the per-pixel partials (k_ssim_fwd writes them; k_ssim_bwd blurs
// them).  Both kernels use 32x32 output tiles with a 5-pixel apron staged in shared
// memory, one separable pass per direction.
#include <math.h>
#include <stdio.h>

#include "cgs_internal.cuh"

namespace cgs {

constexpr int kSsimR = 5;                    // window radius
constexpr int kSsimT = 32;                   // output tile edge
constexpr int kSsimIn = kSsimT + 2 * kSsimR;  // staged edge
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;
constexpr int kRB = 4;                       // outputs per thread along a blur pass

struct SsimTaps {
    float g[2 * kSsimR + 1];
};

// per-view accumulators: sum S, sum |x - y|, sum |D - D*| (valid)
constexpr int kSsimAcc = 3;

__global__ void __launch_bounds__(256)
k_ssim_fwd(const float *__restrict__ img, const float *__restrict__ tgt, int W, int H, SsimTaps t,
           float *__restrict__ amap, float *__restrict__ bmap, float *__restrict__ cmap, double *__restrict__ acc)
{
    // rows padded by one float: the passes' lane patterns then hit distinct banks
    __shared__ float sx[kSsimIn][kSsimIn + 1], sy[kSsimIn][kSsimIn + 1];
    __shared__ float hm[5][kSsimIn][kSsimT + 1];
    __shared__ float red[2][8];
    const int vc = blockIdx.z;                     // view * 3 + channel
    const size_t plane = (size_t)vc * W * H;
    const int x0 = blockIdx.x * kSsimT - kSsimR, y0 = blockIdx.y * kSsimT - kSsimR;
    for (int i = threadIdx.x; i < kSsimIn * kSsimIn; i += blockDim.x) {
        const int r = i / kSsimIn, c = i % kSsimIn;
        const int gx = x0 + c, gy = y0 + r;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        sx[r][c] = in ? img[plane + (size_t)gy * W + gx] : 0.f;
        sy[r][c] = in ? tgt[plane + (size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    // horizontal pass, kRB adjacent outputs per thread from kRB + 10 staged values
    for (int i = threadIdx.x; i < kSsimIn * (kSsimT / kRB); i += blockDim.x) {
        const int r = i / (kSsimT / kRB), c0 = (i % (kSsimT / kRB)) * kRB;
        // the staged values and their products, formed once for the kRB outputs
        float xs[kRB + 2 * kSsimR], ys[kRB + 2 * kSsimR], xx[kRB + 2 * kSsimR], yy[kRB + 2 * kSsimR],
            xy[kRB + 2 * kSsimR];
#pragma unroll
        for (int k = 0; k < kRB + 2 * kSsimR; k++) {
            xs[k] = sx[r][c0 + k];
            ys[k] = sy[r][c0 + k];
            xx[k] = xs[k] * xs[k];
            yy[k] = ys[k] * ys[k];
            xy[k] = xs[k] * ys[k];
        }
#pragma unroll
        for (int o = 0; o < kRB; o++) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
            for (int k = 0; k < 2 * kSsimR + 1; k++) {
                const float w = t.g[k];
                a0 = fmaf(w, xs[o + k], a0);
                a1 = fmaf(w, ys[o + k], a1);
                a2 = fmaf(w, xx[o + k], a2);
                a3 = fmaf(w, yy[o + k], a3);
                a4 = fmaf(w, xy[o + k], a4);
            }
            hm[0][r][c0 + o] = a0;
            hm[1][r][c0 + o] = a1;
            hm[2][r][c0 + o] = a2;
            hm[3][r][c0 + o] = a3;
            hm[4][r][c0 + o] = a4;
        }
    }
    __syncthreads();
    float sS = 0.f, sR = 0.f;
    // vertical pass: kRB rows of one column per thread (kSsimT x kSsimT / kRB = 256 items)
    for (int i = threadIdx.x; i < kSsimT * (kSsimT / kRB); i += blockDim.x) {
        const int c = i % kSsimT, r0 = (i / kSsimT) * kRB;
        float mom[5][kRB];
#pragma unroll
        for (int m = 0; m < 5; m++) {
            float col[kRB + 2 * kSsimR];
#pragma unroll
            for (int k = 0; k < kRB + 2 * kSsimR; k++) col[k] = hm[m][r0 + k][c];
#pragma unroll
            for (int o = 0; o < kRB; o++) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < 2 * kSsimR + 1; k++) a = fmaf(t.g[k], col[o + k], a);
                mom[m][o] = a;
            }
        }
#pragma unroll
        for (int o = 0; o < kRB; o++) {
            const int r = r0 + o;
            const int gx = blockIdx.x * kSsimT + c, gy = blockIdx.y * kSsimT + r;
            if (gx >= W || gy >= H) continue;
            const float mx = mom[0][o], my = mom[1][o];
            const float sxx = mom[2][o] - mx * mx, syy = mom[3][o] - my * my, sxy = mom[4][o] - mx * my;
            const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
            const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
            const float inv = __fdividef(1.f, B1 * B2);
            const float S = A1 * A2 * inv;
            const float dA1 = A2 * inv, dA2 = A1 * inv, dB1 = -S * (B2 * inv), dB2 = -S * (B1 * inv);
            const size_t q = plane + (size_t)gy * W + gx;
            amap[q] = 2.f * my * (dA1 - dA2) + 2.f * mx * (dB1 - dB2);
            bmap[q] = dB2;
            cmap[q] = 2.f * dA2;
            sS += S;
            sR += fabsf(sx[r + kSsimR][c + kSsimR] - sy[r + kSsimR][c + kSsimR]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sS += __shfl_xor_sync(kFull, sS, o);
        sR += __shfl_xor_sync(kFull, sR, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sS;
        red[1][threadIdx.x >> 5] = sR;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            a += red[0][i];
            b += red[1][i];
        }
        const int v = vc / 3;
        atomicAdd(acc + kSsimAcc * v + 0, a);
        atomicAdd(acc + kSsimAcc * v + 1, b);
    }
}

__global__ void __launch_bounds__(256)
k_ssim_bwd(const float *__restrict__ img, const float *__restrict__ tgt, const float *__restrict__ depth,
           const float *__restrict__ tgt_depth, const int32_t *__restrict__ depth_count,
           const float *__restrict__ weight, int W, int H, SsimTaps t, float lam, float lambda_d,
           const float *__restrict__ amap, const float *__restrict__ bmap, const float *__restrict__ cmap,
           float *__restrict__ dl_dimg, float *__restrict__ dl_ddepth, double *__restrict__ acc)
{
    __shared__ float sa[3][kSsimIn][kSsimIn + 1];
    __shared__ float hb[3][kSsimIn][kSsimT + 1];
    __shared__ float red[8];
    const int vc = blockIdx.z, v = vc / 3, ch = vc % 3;
    const size_t plane = (size_t)vc * W * H;
    const int x0 = blockIdx.x * kSsimT - kSsimR, y0 = blockIdx.y * kSsimT - kSsimR;
    for (int i = threadIdx.x; i < kSsimIn * kSsimIn; i += blockDim.x) {
        const int r = i / kSsimIn, c = i % kSsimIn;
        const int gx = x0 + c, gy = y0 + r;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const size_t q = plane + (size_t)gy * W + gx;
        sa[0][r][c] = in ? amap[q] : 0.f;
        sa[1][r][c] = in ? bmap[q] : 0.f;
        sa[2][r][c] = in ? cmap[q] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSsimIn * (kSsimT / kRB); i += blockDim.x) {
        const int r = i / (kSsimT / kRB), c0 = (i % (kSsimT / kRB)) * kRB;
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float row[kRB + 2 * kSsimR];
#pragma unroll
            for (int k = 0; k < kRB + 2 * kSsimR; k++) row[k] = sa[m][r][c0 + k];
#pragma unroll
            for (int o = 0; o < kRB; o++) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < 2 * kSsimR + 1; k++) a = fmaf(t.g[k], row[o + k], a);
                hb[m][r][c0 + o] = a;
            }
        }
    }
    __syncthreads();
    const float M = 3.f * (float)W * (float)H;
    const float wv = weight ? weight[v] : 1.f;
    const int cnt = depth_count ? depth_count[v] : 0;
    float sD = 0.f;
    for (int i = threadIdx.x; i < kSsimT * (kSsimT / kRB); i += blockDim.x) {
        const int c = i % kSsimT, r0 = (i / kSsimT) * kRB;
        const int gx = blockIdx.x * kSsimT + c;
        // image and target of the thread's pixels, loaded before the blur so the loads overlap it
        float xs[kRB], ys[kRB];
#pragma unroll
        for (int o = 0; o < kRB; o++) {
            const int gy = blockIdx.y * kSsimT + r0 + o;
            const bool in = gx < W && gy < H;
            const size_t q = plane + (size_t)(in ? gy : 0) * W + (in ? gx : 0);
            xs[o] = in ? img[q] : 0.f;
            ys[o] = in ? tgt[q] : 0.f;
        }
        float bl[3][kRB];
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float col[kRB + 2 * kSsimR];
#pragma unroll
            for (int k = 0; k < kRB + 2 * kSsimR; k++) col[k] = hb[m][r0 + k][c];
#pragma unroll
            for (int o = 0; o < kRB; o++) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < 2 * kSsimR + 1; k++) a = fmaf(t.g[k], col[o + k], a);
                bl[m][o] = a;
            }
        }
#pragma unroll
        for (int o = 0; o < kRB; o++) {
            const int gy = blockIdx.y * kSsimT + r0 + o;
            if (gx >= W || gy >= H) continue;
            const float ba = bl[0][o], bb = bl[1][o], bc = bl[2][o];
            const size_t q = plane + (size_t)gy * W + gx;
            const float xv = xs[o], yv = ys[o];
            const float sgn = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
            dl_dimg[q] = wv * ((1.f - lam) * sgn / M - lam / M * (ba + 2.f * xv * bb + yv * bc));
            if (ch == 0 && dl_ddepth) {
                const size_t pix = (size_t)v * W * H + (size_t)gy * W + gx;
                float gd = 0.f;
                if (tgt_depth && cnt > 0) {
                    const float td = tgt_depth[pix];
                    if (td > 0.f) {
                        const float dd = depth[pix] - td;
                        gd = wv * lambda_d * (dd > 0.f ? 1.f : (dd < 0.f ? -1.f : 0.f)) / (float)cnt;
                        sD += fabsf(dd);
                    }
                }
                dl_ddepth[pix] = gd;
            }
        }
    }
    if (ch == 0) {
        for (int o = 16; o > 0; o >>= 1) sD += __shfl_xor_sync(kFull, sD, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sD;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
            atomicAdd(acc + kSsimAcc * v + 2, s);
        }
    }
}

__global__ void k_ssim_loss_final(const double *__restrict__ acc, const int32_t *__restrict__ depth_count,
                                  const float *__restrict__ weight, int V, double M, float lam, float lambda_d,
                                  float *__restrict__ loss_view, int32_t *__restrict__ status)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const double w = weight ? (double)weight[v] : 1.0;
    const int cnt = depth_count ? depth_count[v] : 0;
    const double L = w * ((1.0 - lam) * acc[kSsimAcc * v + 1] / M + lam * (1.0 - acc[kSsimAcc * v + 0] / M) +
                          (cnt > 0 ? (double)lambda_d * acc[kSsimAcc * v + 2] / cnt : 0.0));
    loss_view[v] = (float)L;
    if (!isfinite(L)) set_status(status, CGS_ERR_NONFINITE);
}

}  // namespace cgs

using namespace cgs;

extern "C" {

size_t cgs_ssim_workspace(int32_t V, const cgs_config *cfg)
{
    if (!cfg || V < 1 || cfg->width < 1 || cfg->height < 1) return 0;
    const size_t maps = 3 * (size_t)V * 3 * (size_t)cfg->width * cfg->height * sizeof(float);
    return ((maps + 255) & ~(size_t)255) + (size_t)V * kSsimAcc * sizeof(double);
}

int cgs_ssim_loss(const float *img, const float *tgt_rgb, const float *depth, const float *tgt_depth,
                  const int32_t *depth_count, int32_t V, const cgs_config *cfg, const float *view_weight,
                  float lambda_ssim, float *loss_view, float *dl_dimg, float *dl_ddepth, void *workspace,
                  size_t workspace_bytes, int32_t *status_dev, void *stream)
{
    if (!img || !tgt_rgb || !loss_view || !dl_dimg || !workspace || !cfg || V < 1) return CGS_ERR_ARG;
    if (cfg->width < 1 || cfg->height < 1 || cfg->width > (1 << 16) || cfg->height > (1 << 16)) return CGS_ERR_ARG;
    if (tgt_depth && (!depth || !depth_count || !dl_ddepth)) return CGS_ERR_ARG;
    if (!(lambda_ssim >= 0.f && lambda_ssim <= 1.f)) return CGS_ERR_ARG;
    if (workspace_bytes < cgs_ssim_workspace(V, cfg) || ((uintptr_t)workspace & 255) != 0) return CGS_ERR_WORKSPACE;
    const int W = cfg->width, H = cfg->height;
    const size_t plane_all = (size_t)V * 3 * W * H;
    float *amap = static_cast<float *>(workspace);
    float *bmap = amap + plane_all, *cmap = bmap + plane_all;
    const size_t maps = 3 * plane_all * sizeof(float);
    double *acc = reinterpret_cast<double *>(static_cast<char *>(workspace) + ((maps + 255) & ~(size_t)255));
    SsimTaps t;
    double sum = 0.0, gd[2 * kSsimR + 1];
    for (int k = 0; k < 2 * kSsimR + 1; k++) {
        const double x = k - kSsimR;
        gd[k] = exp(-(x * x) / (2.0 * 1.5 * 1.5));
        sum += gd[k];
    }
    for (int k = 0; k < 2 * kSsimR + 1; k++) t.g[k] = (float)(gd[k] / sum);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * kSsimAcc * V, s);
    const dim3 grid((W + kSsimT - 1) / kSsimT, (H + kSsimT - 1) / kSsimT, 3 * V);
    if (e == cudaSuccess) {
        k_ssim_fwd<<<grid, 256, 0, s>>>(img, tgt_rgb, W, H, t, amap, bmap, cmap, acc);
        k_ssim_bwd<<<grid, 256, 0, s>>>(img, tgt_rgb, depth, tgt_depth, depth_count, view_weight, W, H, t,
                                        lambda_ssim, cfg->lambda_depth, amap, bmap, cmap, dl_dimg,
                                        tgt_depth ? dl_ddepth : nullptr, acc);
        k_ssim_loss_final<<<(V + 63) / 64, 64, 0, s>>>(acc, tgt_depth ? depth_count : nullptr, view_weight, V,
                                                       3.0 * W * H, lambda_ssim, cfg->lambda_depth, loss_view,
                                                       status_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        fprintf(stderr, "libcgs: CUDA error: %s\n", cudaGetErrorString(e));
        return CGS_ERR_CUDA;
    }
    return CGS_OK;
}

}  // extern "C"
