// Fused optimiser step and densification statistics.
//
// cgs_adam: one pass over the flat parameter vector (params, grads, m, v read once,
// params, m, v written once; 28 bytes per element).  The opacity regulariser of
// Eqs. 10-11 (Sec. III-C.3, CaRtGS), lambda_o/N sum sigmoid(logit), is folded into
// the gradient of the opacity group in the same pass.  Vectorised with float4
// when the four arrays are 16-byte aligned.
//
// cgs_densify_stats: per visible slot, the view-space (NDC) norm of dL_v/d(u, v),
// the visible-view count and the largest screen radius (Sec. III-A.3, Sec. IV-A).
#include <algorithm>

#include "cgs_internal.cuh"

namespace cgs {

struct AdamArgs {
    float *p;
    const float *g;
    float *m, *v;
    int64_t total;
    int64_t bnd[5];     // group starts of log_scales, quats, opacity, sh_dc, sh_rest
    float lr[6];
    float b1, b2, eps, rbc1, rbc2sqrt;   // 1/(1 - b1^t), 1/sqrt(1 - b2^t) (host step)
    const int32_t *step_dev;             // if set: t is read here instead
    float lam_over_n;
    int64_t opac0, opac1;
    float *loss_o;
};

// Learning rate of flat element i: its group's, chosen by comparisons with the group
// starts (a select chain in registers, not an indexed load).
__device__ __forceinline__ float lr_of(int64_t i, const AdamArgs &a)
{
    float lr = a.lr[0];
    lr = i >= a.bnd[0] ? a.lr[1] : lr;
    lr = i >= a.bnd[1] ? a.lr[2] : lr;
    lr = i >= a.bnd[2] ? a.lr[3] : lr;
    lr = i >= a.bnd[3] ? a.lr[4] : lr;
    lr = i >= a.bnd[4] ? a.lr[5] : lr;
    return lr;
}

// Bias corrections of the step held on the device, computed in double by one thread of
// the block and shared (FP64 is slow on this part: a pow per thread cost more than the
// whole element update).
__device__ __forceinline__ void bias_corrections(AdamArgs &a)
{
    if (a.step_dev) {   // uniform over the grid
        __shared__ float bc[2];
        if (threadIdx.x == 0) {
            const double t = (double)*a.step_dev;
            bc[0] = (float)(1.0 / (1.0 - pow((double)a.b1, t)));
            bc[1] = (float)(1.0 / sqrt(1.0 - pow((double)a.b2, t)));
        }
        __syncthreads();
        a.rbc1 = bc[0];
        a.rbc2sqrt = bc[1];
    }
}

__global__ void k_step_inc(int32_t *step) { *step += 1; }

__device__ __forceinline__ float adam_elem(int64_t i, float p, float g, float &m, float &v, const AdamArgs &a,
                                           float &osum)
{
    if (i >= a.opac0 && i < a.opac1) {
        const float o = 1.0f / (1.0f + expf(-p));
        g += a.lam_over_n * o * (1.0f - o);
        osum += o;
    }
    m = fmaf(a.b1, m, (1.0f - a.b1) * g);
    v = fmaf(a.b2, v, (1.0f - a.b2) * g * g);
    const float mh = m * a.rbc1;
    const float denom = sqrtf(v) * a.rbc2sqrt + a.eps;
    return p - lr_of(i, a) * mh / denom;
}

__global__ void __launch_bounds__(256) k_adam_vec(AdamArgs a)
{
    bias_corrections(a);
    float osum = 0.f;
    const int64_t n4 = a.total / 4;
    float4 *p4 = reinterpret_cast<float4 *>(a.p);
    const float4 *g4 = reinterpret_cast<const float4 *>(a.g);
    float4 *m4 = reinterpret_cast<float4 *>(a.m);
    float4 *v4 = reinterpret_cast<float4 *>(a.v);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
        float4 p = p4[q], g = __ldg(g4 + q), m = m4[q], v = v4[q];
        const int64_t i = 4 * q;
        p.x = adam_elem(i, p.x, g.x, m.x, v.x, a, osum);
        p.y = adam_elem(i + 1, p.y, g.y, m.y, v.y, a, osum);
        p.z = adam_elem(i + 2, p.z, g.z, m.z, v.z, a, osum);
        p.w = adam_elem(i + 3, p.w, g.w, m.w, v.w, a, osum);
        p4[q] = p;
        m4[q] = m;
        v4[q] = v;
    }
    // scalar tail
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.total;
         i += (int64_t)gridDim.x * blockDim.x) {
        float m = a.m[i], v = a.v[i];
        a.p[i] = adam_elem(i, a.p[i], a.g[i], m, v, a, osum);
        a.m[i] = m;
        a.v[i] = v;
    }
    if (a.loss_o) {
        for (int off = 16; off > 0; off >>= 1) osum += __shfl_xor_sync(kFull, osum, off);
        if ((threadIdx.x & 31) == 0 && osum != 0.f) atomicAdd(a.loss_o, osum * a.lam_over_n);
    }
}

__global__ void __launch_bounds__(256) k_adam_scalar(AdamArgs a)
{
    bias_corrections(a);
    float osum = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.total; i += (int64_t)gridDim.x * blockDim.x) {
        float m = a.m[i], v = a.v[i];
        a.p[i] = adam_elem(i, a.p[i], a.g[i], m, v, a, osum);
        a.m[i] = m;
        a.v[i] = v;
    }
    if (a.loss_o) {
        for (int off = 16; off > 0; off >>= 1) osum += __shfl_xor_sync(kFull, osum, off);
        if ((threadIdx.x & 31) == 0 && osum != 0.f) atomicAdd(a.loss_o, osum * a.lam_over_n);
    }
}

cudaError_t adam(float *p, const float *g, float *m, float *v, int64_t n, int deg, const float *lr, float b1,
                 float b2, float eps, int step, int32_t *step_dev, float lambda_o, float *loss_o, int num_sms,
                 cudaStream_t s)
{
    const Layout L = param_layout(n, deg);
    AdamArgs a;
    a.p = p;
    a.g = g;
    a.m = m;
    a.v = v;
    a.total = L.total;
    a.bnd[0] = L.scales;
    a.bnd[1] = L.quats;
    a.bnd[2] = L.opac;
    a.bnd[3] = L.dc;
    a.bnd[4] = L.rest;
    for (int i = 0; i < 6; i++) a.lr[i] = lr[i];
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    // bias corrections in double on the host, then rounded once
    a.rbc1 = (float)(1.0 / (1.0 - pow((double)b1, (double)step)));
    a.rbc2sqrt = (float)(1.0 / sqrt(1.0 - pow((double)b2, (double)step)));
    a.lam_over_n = (float)((double)lambda_o / (double)n);
    a.opac0 = L.opac;
    a.opac1 = L.opac + n;
    a.loss_o = loss_o;
    a.step_dev = step_dev;
    if (step_dev) {
        k_step_inc<<<1, 1, 0, s>>>(step_dev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (loss_o) {
        cudaError_t e = cudaMemsetAsync(loss_o, 0, sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    const bool aligned = ((((uintptr_t)p) | ((uintptr_t)g) | ((uintptr_t)m) | ((uintptr_t)v)) & 15) == 0;
    const int threads = 256;
    const int64_t work = aligned ? (L.total + 3) / 4 : L.total;
    const int blocks = (int)std::min<int64_t>((work + threads - 1) / threads, (int64_t)num_sms * 8);
    if (aligned)
        k_adam_vec<<<blocks, threads, 0, s>>>(a);
    else
        k_adam_scalar<<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
k_densify(const float4 *__restrict__ rec, const float4 *__restrict__ sgrad, int64_t n, int V, float halfW, float halfH,
          float *__restrict__ accum, float *__restrict__ denom, float *__restrict__ maxr)
{
    const int64_t total = (int64_t)V * n;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total; s += (int64_t)gridDim.x * blockDim.x) {
        const int r = __float_as_int(__ldg(reinterpret_cast<const float *>(rec + kRec4 * s) + 7));
        if (r <= 0) continue;
        const int64_t g = s % n;
        const float4 G = __ldg(sgrad + kRec4 * s);
        const float gx = G.x * halfW, gy = G.y * halfH;
        atomicAdd(accum + g, sqrtf(gx * gx + gy * gy));
        atomicAdd(denom + g, 1.0f);
        atomicMax(reinterpret_cast<int *>(maxr + g), __float_as_int((float)r));
    }
}

cudaError_t densify_stats(const float *rec, const float *sgrad, int64_t n, int V, const Grid &g, float *accum,
                          float *denom, float *maxr, int num_sms, cudaStream_t s)
{
    const int64_t total = (int64_t)V * n;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 16);
    k_densify<<<blocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(rec), reinterpret_cast<const float4 *>(sgrad), n,
                                     V, 0.5f * (float)g.W, 0.5f * (float)g.H, accum, denom, maxr);
    return cudaGetLastError();
}

}  // namespace cgs
