// Adaptive density control (Sec. III-A.3 "splitting and cloning ... guided by gradients
// and the size", Sec. IV-A: densify with the positional-gradient threshold tau_p and
// remove Gaussians with opacity below eps_alpha), on the device.
//
// k_densify_plan classifies every Gaussian in float32 (0 prune, 1 keep, 2 keep + clone,
// 3 split into two) from its average view-space gradient accum/denom, its largest
// log-scale and its opacity logit, against thresholds rounded once from double on the
// host; k_count_scan turns the per-Gaussian output counts into output positions and the
// new Gaussian count; k_densify_apply writes the new parameter vector and Adam state
// (clones and split children start with zero moments), each Gaussian's outputs
// consecutive.  Split children are mean + R(q) (s * z) with caller-supplied standard
// normal z, scale s / 1.6, other attributes copied.
#include <math.h>
#include <stdio.h>

#include "cgs_internal.cuh"

namespace cgs {

constexpr float kLogSplitDiv = 0.47000362924573558f;   // ln(1.6)

__global__ void k_densify_plan(const float *__restrict__ P, int64_t n, const float *__restrict__ accum,
                               const float *__restrict__ denom, float t_grad, float t_logs, float t_logit,
                               uint32_t *__restrict__ code, uint32_t *__restrict__ count)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const float den = denom[g];
        const float grad = den > 0.f ? __fdiv_rn(accum[g], den) : 0.f;
        const bool high = grad >= t_grad;
        const float *ls = P + 3 * n + 3 * g;
        const bool small = fmaxf(fmaxf(ls[0], ls[1]), ls[2]) <= t_logs;
        const bool prune = P[10 * n + g] < t_logit;
        const uint32_t c = prune ? 0u : (high ? (small ? 2u : 3u) : 1u);
        code[g] = c;
        count[g] = c == 0u ? 0u : (c == 1u ? 1u : 2u);
    }
}

// Single-block exclusive scan of count[0..n) into off[0..n], off[n] = total (warp chunks,
// coalesced loads).
__global__ void __launch_bounds__(1024)
k_count_scan(const uint32_t *__restrict__ count, int64_t n, uint32_t *__restrict__ off, int64_t *__restrict__ total_out)
{
    __shared__ unsigned long long wtot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (n + 31) / 32;
    const int64_t lo = (int64_t)w * per, hi = min(n, lo + per);
    unsigned long long s = 0;
    for (int64_t t = lo + lane; t < hi; t += 32) s += count[t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) wtot[w] = s;
    __syncthreads();
    unsigned long long run = 0, total = 0;
    for (int i = 0; i < 32; i++) {
        run += (i < w) ? wtot[i] : 0ull;
        total += wtot[i];
    }
    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t t = base + lane;
        const unsigned long long c = t < hi ? count[t] : 0ull;
        unsigned long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (t < hi) off[t] = (uint32_t)(run + incl - c);
        run += __shfl_sync(kFull, incl, 31);
    }
    if (threadIdx.x == 0) {
        off[n] = (uint32_t)total;
        *total_out = (int64_t)total;
    }
}

// Copy Gaussian g of the input layout (n) to index j of the output layout (m); with
// moments if src_m is non-null, else zero moments.
__device__ __forceinline__ void copy_gaussian(const float *__restrict__ P, const float *__restrict__ Mi,
                                              const float *__restrict__ Vi, int64_t n, int64_t g, float *__restrict__ Po,
                                              float *__restrict__ Mo, float *__restrict__ Vo, int64_t m, int64_t j,
                                              int K, bool moments)
{
    const int widths[6] = {3, 3, 4, 1, 3, 3 * (K - 1)};
    int64_t oi = 0, oo = 0;
    for (int gi = 0; gi < 6; gi++) {
        const int w = widths[gi];
        for (int c = 0; c < w; c++) {
            Po[oo + (int64_t)w * j + c] = P[oi + (int64_t)w * g + c];
            Mo[oo + (int64_t)w * j + c] = moments ? Mi[oi + (int64_t)w * g + c] : 0.f;
            Vo[oo + (int64_t)w * j + c] = moments ? Vi[oi + (int64_t)w * g + c] : 0.f;
        }
        oi += (int64_t)w * n;
        oo += (int64_t)w * m;
    }
}

__global__ void k_densify_apply(const float *__restrict__ P, const float *__restrict__ Mi, const float *__restrict__ Vi,
                                int64_t n, int K, const uint32_t *__restrict__ code, const uint32_t *__restrict__ off,
                                const float *__restrict__ normals, int64_t m, float *__restrict__ Po,
                                float *__restrict__ Mo, float *__restrict__ Vo)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = code[g];
        const int64_t j = off[g];
        if (c == 0u) continue;
        if (j + (c == 1u ? 1 : 2) > m) continue;   // never write past the caller's n_out
        if (c == 1u || c == 2u) copy_gaussian(P, Mi, Vi, n, g, Po, Mo, Vo, m, j, K, true);
        if (c == 2u) copy_gaussian(P, Mi, Vi, n, g, Po, Mo, Vo, m, j + 1, K, false);
        if (c == 3u) {
            const float *q = P + 6 * n + 4 * g;
            const float inv = 1.0f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
            const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                                2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                                2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
            const float *ls = P + 3 * n + 3 * g;
            const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
            for (int k = 0; k < 2; k++) {
                const int64_t jj = j + k;
                copy_gaussian(P, Mi, Vi, n, g, Po, Mo, Vo, m, jj, K, false);
                const float *zz = normals + 6 * g + 3 * k;
                const float d0 = s[0] * zz[0], d1 = s[1] * zz[1], d2 = s[2] * zz[2];
                for (int r = 0; r < 3; r++)
                    Po[3 * jj + r] = P[3 * g + r] + (R[3 * r] * d0 + R[3 * r + 1] * d1 + R[3 * r + 2] * d2);
                for (int r = 0; r < 3; r++) Po[3 * m + 3 * jj + r] = ls[r] - kLogSplitDiv;
            }
        }
    }
}

}  // namespace cgs

using namespace cgs;

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
int st_of(cudaError_t e)
{
    if (e == cudaSuccess) return CGS_OK;
    fprintf(stderr, "libcgs: CUDA error: %s\n", cudaGetErrorString(e));
    return CGS_ERR_CUDA;
}
}  // namespace

extern "C" {

size_t cgs_densify_workspace(int64_t n)
{
    if (n < 0) return 0;
    return al256(sizeof(uint32_t) * (size_t)n) * 2 + al256(sizeof(uint32_t) * ((size_t)n + 1));
}

int cgs_densify_plan(const float *params, int64_t n, int32_t sh_degree, const float *accum, const float *denom,
                     double tau_p, double scale_thr, double eps_alpha, void *workspace, size_t workspace_bytes,
                     int64_t *n_out_dev, void *stream)
{
    if (!params || !accum || !denom || !workspace || !n_out_dev || n < 1 || sh_degree < 0 || sh_degree > 3)
        return CGS_ERR_ARG;
    if (!(scale_thr > 0.0) || !(eps_alpha > 0.0 && eps_alpha < 1.0) || !(tau_p >= 0.0)) return CGS_ERR_ARG;
    if (2 * n + 1 >= ((int64_t)1 << 32)) return CGS_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0) return CGS_ERR_ARG;
    if (workspace_bytes < cgs_densify_workspace(n)) return CGS_ERR_WORKSPACE;
    uint32_t *code = static_cast<uint32_t *>(workspace);
    uint32_t *count = reinterpret_cast<uint32_t *>(static_cast<char *>(workspace) + al256(sizeof(uint32_t) * n));
    uint32_t *off = reinterpret_cast<uint32_t *>(static_cast<char *>(workspace) + 2 * al256(sizeof(uint32_t) * n));
    const float t_grad = (float)tau_p;
    const float t_logs = (float)log(scale_thr);
    const float t_logit = (float)log(eps_alpha / (1.0 - eps_alpha));
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_densify_plan<<<blocks, 256, 0, s>>>(params, n, accum, denom, t_grad, t_logs, t_logit, code, count);
    k_count_scan<<<1, 1024, 0, s>>>(count, n, off, n_out_dev);
    return st_of(cudaGetLastError());
}

int cgs_densify_apply(const float *params, const float *m, const float *v, int64_t n, int32_t sh_degree,
                      const void *workspace, size_t workspace_bytes, const float *normals, int64_t n_out,
                      float *params_out, float *m_out, float *v_out, void *stream)
{
    if (!params || !m || !v || !workspace || !normals || n < 1 || n_out < 0 || sh_degree < 0 || sh_degree > 3)
        return CGS_ERR_ARG;
    if (n_out > 0 && (!params_out || !m_out || !v_out)) return CGS_ERR_ARG;
    if (workspace_bytes < cgs_densify_workspace(n)) return CGS_ERR_WORKSPACE;
    if (n_out > 2 * n) return CGS_ERR_ARG;
    const uint32_t *code = static_cast<const uint32_t *>(workspace);
    const uint32_t *off =
        reinterpret_cast<const uint32_t *>(static_cast<const char *>(workspace) + 2 * al256(sizeof(uint32_t) * n));
    const int K = (sh_degree + 1) * (sh_degree + 1);
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_densify_apply<<<blocks, 256, 0, s>>>(params, m, v, n, K, code, off, normals, n_out, params_out, m_out, v_out);
    return st_of(cudaGetLastError());
}

}  // extern "C"
