// Projection of Gaussians into the views of a window (forward) and the chain rule
// back to the parameters (backward).  The projected 2-D Gaussian and the colour c_k
// are the inputs of the blend of Eq. 1 (Sec. III-B, CaRtGS); the projection is the
// EWA splatting of 3DGS the paper builds on.
//
// Work decomposition: a block owns kGB consecutive Gaussians and all V views.  The
// block's slice of every parameter group (contiguous in the SoA vector) is staged
// into shared memory with coalesced loads, so each parameter is read from HBM once
// per window; threads then take (Gaussian, view) items with the Gaussian index
// fastest, which keeps record writes coalesced within each view's slot range.
#include "cgs_internal.cuh"

namespace cgs {

constexpr int kGB = 128;         // Gaussians per block (64: backward 0.53 ms, 128: 0.44 on the 16-view window)
constexpr int kPreThreads = 256;
// Resident blocks per SM the backward is compiled for.  With the covariance staged per
// Gaussian and its chain to scale and rotation run once per Gaussian, three blocks fit
// (at most 85 registers, 73 KB of shared memory on 16 views): 0.404 -> 0.382 ms on the
// 16-view window (two blocks at 124 registers before: 0.415 ms).
constexpr int kPreBwdMinBlocks = 3;
constexpr int kViewChunk = 64;        // views per compaction round of the backward
static_assert(kGB * kViewChunk / kPreThreads <= 32, "a thread's visibility bits of a view chunk fit one word");
constexpr int kCamF = 23;        // staged camera: 20 ABI floats + camera centre

// Real SH normalisation constants (closed forms: sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) x
// the factors of each real polynomial), degree <= 3, Condon-Shortley phase kept.
constexpr float kY0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kY2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float kY3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float kY3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float kY3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float kY3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kY3e = 1.445305721320277f;    // sqrt(105/pi)/4

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    Y[0] = kY0;
    if (DEG >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

// g += sum_k w[k] * grad Y_k(x, y, z) for k >= 1 (gradient w.r.t. the free direction)
template <int DEG>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float *w, float g[3])
{
    if (DEG >= 1) {
        g[1] += -kY1 * w[1];
        g[2] += kY1 * w[2];
        g[0] += -kY1 * w[3];
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        g[0] += kY2a * y * w[4];
        g[1] += kY2a * x * w[4];
        g[1] += -kY2a * z * w[5];
        g[2] += -kY2a * y * w[5];
        g[0] += -2.f * kY2b * x * w[6];
        g[1] += -2.f * kY2b * y * w[6];
        g[2] += 4.f * kY2b * z * w[6];
        g[0] += -kY2a * z * w[7];
        g[2] += -kY2a * x * w[7];
        g[0] += 2.f * kY2c * x * w[8];
        g[1] += -2.f * kY2c * y * w[8];
        if (DEG >= 3) {
            g[0] += -6.f * kY3a * x * y * w[9];
            g[1] += -kY3a * (3.f * xx - 3.f * yy) * w[9];
            g[0] += kY3b * y * z * w[10];
            g[1] += kY3b * x * z * w[10];
            g[2] += kY3b * x * y * w[10];
            g[0] += 2.f * kY3c * x * y * w[11];
            g[1] += -kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
            g[2] += -8.f * kY3c * y * z * w[11];
            g[0] += -6.f * kY3d * x * z * w[12];
            g[1] += -6.f * kY3d * y * z * w[12];
            g[2] += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            g[0] += -kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
            g[1] += 2.f * kY3c * x * y * w[13];
            g[2] += -8.f * kY3c * x * z * w[13];
            g[0] += 2.f * kY3e * x * z * w[14];
            g[1] += -2.f * kY3e * y * z * w[14];
            g[2] += kY3e * (xx - yy) * w[14];
            g[0] += -kY3a * (3.f * xx - 3.f * yy) * w[15];
            g[1] += 6.f * kY3a * x * y * w[15];
        }
    }
}

// Shared-memory view of one block's parameters.
struct Staged {
    const float *means, *scales, *quats, *opac, *dc, *rest, *cams;
    const float *cov;   // 3-D covariance of each Gaussian (view-independent): xx xy xz yy yz zz
};

// Activations and frame of Gaussian gl: scale s = exp(log_scale), unit quaternion qn =
// q / |q| (qinv = 1/|q|), its rotation R, and M = R diag(s), so Sigma = M M^T.
__device__ __forceinline__ void gauss_frame(const Staged &st, int gl, float s[3], float qn[4], float &qinv,
                                            float R[9], float M[9])
{
    for (int i = 0; i < 3; i++) s[i] = expf(st.scales[3 * gl + i]);
    const float *q = st.quats + 4 * gl;
    float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    qinv = 1.0f / sqrtf(qq);
    for (int i = 0; i < 4; i++) qn[i] = q[i] * qinv;
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);     R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);     R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);     R[7] = 2.f * (y * z + w * x);     R[8] = 1.f - 2.f * (x * x + y * y);
    for (int r = 0; r < 3; r++)
        for (int j = 0; j < 3; j++) M[3 * r + j] = R[3 * r + j] * s[j];
}

template <int DEG>
struct Proj {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    bool visible;
    float t[3], itz;
    float S[6];  // 3-D covariance (staged): xx xy xz yy yz zz
    bool xcl, ycl;
    float xs, ys, limx, limy;
    float T0[3], T1[3];
    float a, b, c, A, B, C;
    float u, v;
    int radius;
    float dir[3], dinv;
    float Y[K];
    float rgb[3];
    int mask;
    float o;
};

// Forward projection of Gaussian gl (block-local) into the staged camera `cam`.
template <int DEG>
__device__ __forceinline__ void project(const Staged &st, int gl, const float *cam, const Grid &grid,
                                        float near_z, Proj<DEG> &o)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float *p = st.means + 3 * gl;
    const float *Rc = cam;
    o.visible = false;
    o.radius = 0;
    for (int i = 0; i < 3; i++)
        o.t[i] = fmaf(Rc[3 * i], p[0], fmaf(Rc[3 * i + 1], p[1], fmaf(Rc[3 * i + 2], p[2], cam[9 + i])));
    if (!(o.t[2] > near_z)) return;
    const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];

    for (int i = 0; i < 6; i++) o.S[i] = st.cov[6 * gl + i];

    // perspective Jacobian with the guard band (1.3 x half field of view)
    const float tz = o.t[2];
    o.itz = 1.0f / tz;
    o.limx = 1.3f * (0.5f * (float)grid.W / fx);
    o.limy = 1.3f * (0.5f * (float)grid.H / fy);
    float rx = o.t[0] / tz, ry = o.t[1] / tz;
    o.xcl = (rx > o.limx) || (rx < -o.limx);
    o.ycl = (ry > o.limy) || (ry < -o.limy);
    o.xs = rx > 0.f ? 1.f : -1.f;
    o.ys = ry > 0.f ? 1.f : -1.f;
    float xc = (o.xcl ? o.xs * o.limx : rx) * tz;
    float yc = (o.ycl ? o.ys * o.limy : ry) * tz;
    float itz2 = o.itz * o.itz;
    float J00 = fx * o.itz, J02 = -fx * xc * itz2, J11 = fy * o.itz, J12 = -fy * yc * itz2;
    for (int j = 0; j < 3; j++) {
        o.T0[j] = J00 * Rc[j] + J02 * Rc[6 + j];
        o.T1[j] = J11 * Rc[3 + j] + J12 * Rc[6 + j];
    }
    // 2-D covariance T Sigma T^T + 0.3 I
    float w0[3], w1[3];
    w0[0] = o.S[0] * o.T0[0] + o.S[1] * o.T0[1] + o.S[2] * o.T0[2];
    w0[1] = o.S[1] * o.T0[0] + o.S[3] * o.T0[1] + o.S[4] * o.T0[2];
    w0[2] = o.S[2] * o.T0[0] + o.S[4] * o.T0[1] + o.S[5] * o.T0[2];
    w1[0] = o.S[0] * o.T1[0] + o.S[1] * o.T1[1] + o.S[2] * o.T1[2];
    w1[1] = o.S[1] * o.T1[0] + o.S[3] * o.T1[1] + o.S[4] * o.T1[2];
    w1[2] = o.S[2] * o.T1[0] + o.S[4] * o.T1[1] + o.S[5] * o.T1[2];
    o.a = o.T0[0] * w0[0] + o.T0[1] * w0[1] + o.T0[2] * w0[2] + 0.3f;
    o.b = o.T1[0] * w0[0] + o.T1[1] * w0[1] + o.T1[2] * w0[2];
    o.c = o.T1[0] * w1[0] + o.T1[1] * w1[1] + o.T1[2] * w1[2] + 0.3f;
    float det = o.a * o.c - o.b * o.b;
    if (!(det > 0.f)) return;
    float idet = 1.0f / det;
    o.A = o.c * idet;
    o.B = -o.b * idet;
    o.C = o.a * idet;
    // largest eigenvalue; mid^2 - det written as ((a - c)/2)^2 + b^2 (no cancellation)
    float hd = 0.5f * (o.a - o.c);
    float disc = hd * hd + o.b * o.b;
    float lam = 0.5f * (o.a + o.c) + sqrtf(fmaxf(0.1f, disc));
    float r3 = ceilf(3.0f * sqrtf(lam));
    o.radius = (int)fminf(r3, 16777216.0f);
    o.u = fmaf(fx, o.t[0] / tz, cx);
    o.v = fmaf(fy, o.t[1] / tz, cy);
    Rect rc = tile_rect(o.u, o.v, o.radius, grid);
    if (rc.x1 <= rc.x0 || rc.y1 <= rc.y0) {
        o.radius = 0;
        return;
    }

    // colour from SH at the direction camera centre -> mean
    float d0 = p[0] - cam[20], d1 = p[1] - cam[21], d2 = p[2] - cam[22];
    float dn = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    o.dinv = 1.0f / dn;
    o.dir[0] = d0 * o.dinv;
    o.dir[1] = d1 * o.dinv;
    o.dir[2] = d2 * o.dinv;
    sh_basis<DEG>(o.dir[0], o.dir[1], o.dir[2], o.Y);
    o.mask = 0;
    const float *dc = st.dc + 3 * gl;
    const float *rest = st.rest + 3 * (K - 1) * gl;
    for (int ch = 0; ch < 3; ch++) {
        float acc = o.Y[0] * dc[ch];
        for (int k = 1; k < K; k++) acc = fmaf(o.Y[k], rest[3 * (k - 1) + ch], acc);
        acc += 0.5f;
        if (acc < 0.f) {
            acc = 0.f;
            o.mask |= 1 << ch;
        }
        o.rgb[ch] = acc;
    }
    o.o = 1.0f / (1.0f + expf(-st.opac[gl]));
    o.visible = true;
}

// Stage the block's parameter slices and the cameras into shared memory.
template <int DEG>
__device__ __forceinline__ Staged stage(float *sm, const float *__restrict__ P, int64_t n, int64_t g0,
                                        int cnt, const cgs_camera *__restrict__ cams, int V)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    const Layout L = param_layout(n, DEG);
    Staged st;
    float *cur = sm;
    const int widths[6] = {3, 3, 4, 1, 3, 3 * (K - 1)};
    const int64_t offs[6] = {L.means, L.scales, L.quats, L.opac, L.dc, L.rest};
    const float **dst[6] = {&st.means, &st.scales, &st.quats, &st.opac, &st.dc, &st.rest};
    for (int gi = 0; gi < 6; gi++) {
        const int w = widths[gi];
        if (w == 0) {
            *dst[gi] = cur;
            continue;
        }
        const float *src = P + offs[gi] + (int64_t)w * g0;
        // four loads in flight before their stores: one load and store at a time left each
        // block waiting a memory latency per element it staged (on the 16-view window:
        // backward 0.388 -> 0.337 ms, projection 0.166 -> 0.139 ms; 2, 3, 8 and 16 measured
        // slower)
        const int tot = w * cnt;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 4 * blockDim.x) {
            float x[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + k * (int)blockDim.x;
                x[k] = i < tot ? __ldg(src + i) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = i0 + k * (int)blockDim.x;
                if (i < tot) cur[i] = x[k];
            }
        }
        *dst[gi] = cur;
        cur += w * kGB;
    }
    float *cov = cur;   // filled below, once the parameters are staged
    cur += 6 * kGB;
    // cameras: 20 ABI floats + centre c = -R^T t
    const float *cf = reinterpret_cast<const float *>(cams);
    for (int i = threadIdx.x; i < V * 20; i += blockDim.x) cur[(i / 20) * kCamF + (i % 20)] = __ldg(cf + i);
    __syncthreads();
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        float *c = cur + v * kCamF;
        for (int i = 0; i < 3; i++) c[20 + i] = -(c[i] * c[9] + c[3 + i] * c[10] + c[6 + i] * c[11]);
    }
    st.cams = cur;
    st.cov = cov;
    // Sigma = M M^T of each Gaussian, once for all views
    for (int gl = threadIdx.x; gl < cnt; gl += blockDim.x) {
        float sc[3], qn[4], qinv, R[9], M[9];
        gauss_frame(st, gl, sc, qn, qinv, R, M);
        float *S = cov + 6 * gl;
        S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
        S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
        S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
        S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
        S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
        S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    }
    __syncthreads();
    return st;
}

template <int DEG>
__host__ __device__ constexpr int staged_floats()
{
    return kGB * (14 + 3 * ((DEG + 1) * (DEG + 1) - 1) + 6);   // parameter groups + covariance
}

template <int DEG>
__global__ void __launch_bounds__(kPreThreads)
k_preprocess(const float *__restrict__ P, int64_t n, const cgs_camera *__restrict__ cams, int V,
             Grid grid, float near_z, float4 *__restrict__ rec, float4 *__restrict__ sgrad)
{
    extern __shared__ float sm[];
    const int64_t g0 = (int64_t)blockIdx.x * kGB;
    const int cnt = (int)min((int64_t)kGB, n - g0);
    Staged st = stage<DEG>(sm, P, n, g0, cnt, cams, V);
    for (int it = threadIdx.x; it < kGB * V; it += blockDim.x) {
        const int gl = it % kGB, v = it / kGB;
        if (gl >= cnt) continue;
        const int64_t slot = (int64_t)v * n + g0 + gl;
        Proj<DEG> o;
        project<DEG>(st, gl, st.cams + v * kCamF, grid, near_z, o);
        float4 *r = rec + kRec4 * slot;
        if (!o.visible) {
            // the whole record (radius 0 marks it culled) and slot gradient: with only the
            // radius word written, DRAM read back and rewrote each partly written sector (0.185
            // -> 0.165 ms on the 16-view window)
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            r[0] = zero;
            r[1] = zero;
            r[2] = zero;
            if (sgrad) {
                float4 *gp = sgrad + kRec4 * slot;
                gp[0] = zero;
                gp[1] = zero;
                gp[2] = zero;
            }
            continue;
        }
        r[0] = make_float4(o.u, o.v, o.A, o.B);
        r[1] = make_float4(o.C, o.o, o.t[2], __int_as_float(o.radius));
        // tau = -ln(255 o): alpha >= 1/255 exactly when power >= tau (the tile test and the
        // raster kernels' exponent threshold)
        r[2] = make_float4(o.rgb[0], o.rgb[1], o.rgb[2], -logf(255.0f * o.o));
        if (sgrad) {
            float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 *gp = sgrad + kRec4 * slot;
            gp[0] = zero;
            gp[1] = zero;
            gp[2] = zero;
        }
    }
}

// Backward of one visible slot: accumulates parameter gradients (and dL/dSigma, whose
// chain to scale and rotation sigma_bwd runs once per Gaussian) into the block's shared
// accumulators (acc has the staged layout) with shared-memory atomics.
template <int DEG>
__device__ __forceinline__ void project_bwd(const Staged &st, int gl, const float *cam, const Proj<DEG> &o,
                                            float4 G0, float4 G1, float4 G2, float *acc)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    float *a_means = acc;   // scales and quaternions get theirs once per Gaussian (sigma_bwd)
    float *a_opac = acc + 10 * kGB;
    float *a_dc = acc + 11 * kGB;
    float *a_rest = acc + 14 * kGB;
    const float *Rc = cam;
    const float fx = cam[12], fy = cam[13];
    const float gu = G0.x, gv = G0.y, gA = G0.z, gB = G0.w, gC = G1.x, go = G1.y, gz = G1.z;
    float dmean[3] = {0.f, 0.f, 0.f};

    // colour -> SH coefficients and view direction (0 through a clamped channel)
    float gc[3] = {(o.mask & 1) ? 0.f : G2.x, (o.mask & 2) ? 0.f : G2.y, (o.mask & 4) ? 0.f : G2.z};
    for (int ch = 0; ch < 3; ch++) atomicAdd(&a_dc[3 * gl + ch], o.Y[0] * gc[ch]);
    if (DEG > 0) {
        const float *rest = st.rest + 3 * (K - 1) * gl;
        float wk[K];
        wk[0] = 0.f;
        for (int k = 1; k < K; k++) {
            wk[k] = rest[3 * (k - 1)] * gc[0] + rest[3 * (k - 1) + 1] * gc[1] + rest[3 * (k - 1) + 2] * gc[2];
            for (int ch = 0; ch < 3; ch++) atomicAdd(&a_rest[3 * (K - 1) * gl + 3 * (k - 1) + ch], o.Y[k] * gc[ch]);
        }
        float ddir[3] = {0.f, 0.f, 0.f};
        sh_basis_vjp<DEG>(o.dir[0], o.dir[1], o.dir[2], wk, ddir);
        float dd = ddir[0] * o.dir[0] + ddir[1] * o.dir[1] + ddir[2] * o.dir[2];
        for (int i = 0; i < 3; i++) dmean[i] += (ddir[i] - o.dir[i] * dd) * o.dinv;
    }

    // opacity logit
    atomicAdd(&a_opac[gl], go * o.o * (1.f - o.o));

    // conic Q = Sigma'^-1:  dL/dSigma' = -Q G_Q Q,  G_Q = [[gA, gB/2], [gB/2, gC]]
    const float hB = 0.5f * gB;
    float m00 = o.A * gA + o.B * hB, m01 = o.A * hB + o.B * gC;
    float m10 = o.B * gA + o.C * hB, m11 = o.B * hB + o.C * gC;
    float G00 = -(m00 * o.A + m01 * o.B);
    float G01 = -(m00 * o.B + m01 * o.C);
    float G10 = -(m10 * o.A + m11 * o.B);
    float G11 = -(m10 * o.B + m11 * o.C);
    float Gs = 0.5f * (G01 + G10);
    // rows of G Tm
    float P0[3], P1[3];
    for (int j = 0; j < 3; j++) {
        P0[j] = G00 * o.T0[j] + Gs * o.T1[j];
        P1[j] = Gs * o.T0[j] + G11 * o.T1[j];
    }
    // dL/dSigma = Tm^T G Tm (symmetric) -> GS_ij = T0_i P0_j + T1_i P1_j
    float GS[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) GS[3 * i + j] = o.T0[i] * P0[j] + o.T1[i] * P1[j];
    // dL/dTm = 2 G Tm Sigma
    const float Sf[9] = {o.S[0], o.S[1], o.S[2], o.S[1], o.S[3], o.S[4], o.S[2], o.S[4], o.S[5]};
    float GT0[3], GT1[3];
    for (int j = 0; j < 3; j++) {
        GT0[j] = 2.f * (P0[0] * Sf[j] + P0[1] * Sf[3 + j] + P0[2] * Sf[6 + j]);
        GT1[j] = 2.f * (P1[0] * Sf[j] + P1[1] * Sf[3 + j] + P1[2] * Sf[6 + j]);
    }
    // dL/dJ = dL/dTm Rc^T (entries used by J: 00, 02, 11, 12)
    float GJ00 = GT0[0] * Rc[0] + GT0[1] * Rc[1] + GT0[2] * Rc[2];
    float GJ02 = GT0[0] * Rc[6] + GT0[1] * Rc[7] + GT0[2] * Rc[8];
    float GJ11 = GT1[0] * Rc[3] + GT1[1] * Rc[4] + GT1[2] * Rc[5];
    float GJ12 = GT1[0] * Rc[6] + GT1[1] * Rc[7] + GT1[2] * Rc[8];
    const float itz = o.itz, itz2 = itz * itz, itz3 = itz2 * itz;
    float dt0 = 0.f, dt1 = 0.f, dt2 = 0.f;
    dt2 += GJ00 * (-fx * itz2) + GJ11 * (-fy * itz2);
    if (!o.xcl) {
        dt0 += GJ02 * (-fx * itz2);
        dt2 += GJ02 * (2.f * fx * o.t[0] * itz3);
    } else {
        dt2 += GJ02 * (fx * o.xs * o.limx * itz2);
    }
    if (!o.ycl) {
        dt1 += GJ12 * (-fy * itz2);
        dt2 += GJ12 * (2.f * fy * o.t[1] * itz3);
    } else {
        dt2 += GJ12 * (fy * o.ys * o.limy * itz2);
    }
    // projected centre and depth
    dt0 += gu * fx * itz;
    dt2 -= gu * fx * o.t[0] * itz2;
    dt1 += gv * fy * itz;
    dt2 -= gv * fy * o.t[1] * itz2;
    dt2 += gz;
    for (int i = 0; i < 3; i++) dmean[i] += Rc[i] * dt0 + Rc[3 + i] * dt1 + Rc[6 + i] * dt2;
    for (int i = 0; i < 3; i++) atomicAdd(&a_means[3 * gl + i], dmean[i]);

    // dL/dSigma (symmetric; upper triangle) gathered over the Gaussian's views: the chain to
    // scale and rotation is linear in it and runs once per Gaussian (sigma_bwd)
    float *a_cov = acc + (14 + 3 * (K - 1)) * kGB;
    atomicAdd(&a_cov[6 * gl + 0], GS[0]);
    atomicAdd(&a_cov[6 * gl + 1], GS[1]);
    atomicAdd(&a_cov[6 * gl + 2], GS[2]);
    atomicAdd(&a_cov[6 * gl + 3], GS[4]);
    atomicAdd(&a_cov[6 * gl + 4], GS[5]);
    atomicAdd(&a_cov[6 * gl + 5], GS[8]);
}

// Sigma = M M^T, M = R diag(s), with G = dL/dSigma summed over the views: dL/dM = 2 G M,
// then dL/ds and dL/dR, and the rotation of the unit quaternion back through its
// normalisation; written into the scale and quaternion accumulators of Gaussian gl.
template <int DEG>
__device__ __forceinline__ void sigma_bwd(const Staged &st, int gl, float *acc)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    float *a_scales = acc + 3 * kGB;
    float *a_quats = acc + 6 * kGB;
    const float *a_cov = acc + (14 + 3 * (K - 1)) * kGB;
    float sc[3], qn[4], qinv, R[9], M[9];
    gauss_frame(st, gl, sc, qn, qinv, R, M);
    const float *g6 = a_cov + 6 * gl;
    const float GS[9] = {g6[0], g6[1], g6[2], g6[1], g6[3], g6[4], g6[2], g6[4], g6[5]};
    float GR[9];
    for (int j = 0; j < 3; j++) {
        float ds = 0.f;
        for (int r = 0; r < 3; r++) {
            float gm = 2.f * (GS[3 * r] * M[j] + GS[3 * r + 1] * M[3 + j] + GS[3 * r + 2] * M[6 + j]);
            ds += gm * R[3 * r + j];
            GR[3 * r + j] = gm * sc[j];
        }
        a_scales[3 * gl + j] = ds * sc[j];
    }
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    float dq0 = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    float dq1 = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] +
                       w * GR[7] - 2.f * x * GR[8]);
    float dq2 = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] +
                       z * GR[7] - 2.f * y * GR[8]);
    float dq3 = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] +
                       x * GR[6] + y * GR[7]);
    float pr = dq0 * w + dq1 * x + dq2 * y + dq3 * z;
    a_quats[4 * gl + 0] = (dq0 - w * pr) * qinv;
    a_quats[4 * gl + 1] = (dq1 - x * pr) * qinv;
    a_quats[4 * gl + 2] = (dq2 - y * pr) * qinv;
    a_quats[4 * gl + 3] = (dq3 - z * pr) * qinv;
}

template <int DEG>
__global__ void __launch_bounds__(kPreThreads, kPreBwdMinBlocks)
k_preprocess_bwd(const float *__restrict__ P, int64_t n, const cgs_camera *__restrict__ cams, int V,
                 Grid grid, float near_z, const float4 *__restrict__ rec, const float4 *__restrict__ sgrad,
                 float *__restrict__ pgrad, int accumulate, float *__restrict__ accum,
                 float *__restrict__ denom, float *__restrict__ max_r2d)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int NS = staged_floats<DEG>();
    extern __shared__ float sm[];
    const int64_t g0 = (int64_t)blockIdx.x * kGB;
    const int cnt = (int)min((int64_t)kGB, n - g0);
    float *acc = sm;                    // gradient accumulators, staged layout
    float *dstat = sm + NS;             // densify stats: accum, denom, max radius (3 x kGB)
    for (int i = threadIdx.x; i < NS + 3 * kGB; i += blockDim.x) acc[i] = 0.f;
    // visible (view, Gaussian) items of the block, compacted (per chunk of kViewChunk views)
    // so that the chain rule runs with full warps: most slots of a view are culled
    uint16_t *items = reinterpret_cast<uint16_t *>(sm + 2 * NS + 3 * kGB + V * kCamF);
    __shared__ int wcount[kPreThreads / 32];
    Staged st = stage<DEG>(sm + NS + 3 * kGB, P, n, g0, cnt, cams, V);
    const bool stats = accum != nullptr;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int v0 = 0; v0 < V; v0 += kViewChunk) {
        const int nit = kGB * min(kViewChunk, V - v0);
        int nitems = 0;
        // visibility of this thread's items of the chunk, all loads in flight together
        // (one bit per round of kPreThreads items)
        uint32_t vismask = 0;
#pragma unroll 8
        for (int c0 = 0, rb = 0; c0 < nit; c0 += kPreThreads, rb++) {
            const int it = c0 + (int)threadIdx.x;
            const int gl = it % kGB, v = v0 + it / kGB;
            if (it < nit && gl < cnt) {
                const float *r = reinterpret_cast<const float *>(rec + kRec4 * ((int64_t)v * n + g0 + gl));
                if (__float_as_int(__ldg(r + 7)) > 0) vismask |= 1u << rb;
            }
        }
        for (int c0 = 0, rb = 0; c0 < nit; c0 += kPreThreads, rb++) {
            const int it = c0 + (int)threadIdx.x;
            const bool vis = (vismask >> rb) & 1u;
            const unsigned b = __ballot_sync(kFull, vis);
            if (lane == 0) wcount[wp] = __popc(b);
            __syncthreads();
            int off = nitems, tot = 0;
            for (int i = 0; i < kPreThreads / 32; i++) {
                off += i < wp ? wcount[i] : 0;
                tot += wcount[i];
            }
            if (vis) items[off + __popc(b & ((1u << lane) - 1u))] = (uint16_t)it;
            nitems += tot;
            __syncthreads();
        }
        for (int k = threadIdx.x; k < nitems; k += blockDim.x) {
            const int it = items[k];
            const int gl = it % kGB, v = v0 + it / kGB;
            const int64_t slot = (int64_t)v * n + g0 + gl;
            const float4 *r = rec + kRec4 * slot;
            const int rad = __float_as_int(__ldg(reinterpret_cast<const float *>(r) + 7));
            const float4 *gp = sgrad + kRec4 * slot;
            float4 G0 = gp[0], G1 = gp[1], G2 = gp[2];
            Proj<DEG> o;
            project<DEG>(st, gl, st.cams + v * kCamF, grid, near_z, o);
            if (!o.visible) continue;   // cannot happen for a slot the forward marked visible
            project_bwd<DEG>(st, gl, st.cams + v * kCamF, o, G0, G1, G2, acc);
            if (stats) {
                float gx = G0.x * 0.5f * (float)grid.W, gy = G0.y * 0.5f * (float)grid.H;
                atomicAdd(&dstat[gl], sqrtf(gx * gx + gy * gy));
                atomicAdd(&dstat[kGB + gl], 1.0f);
                atomicMax(reinterpret_cast<int *>(&dstat[2 * kGB + gl]), __float_as_int((float)rad));
            }
        }
        __syncthreads();   // the item list is rebuilt for the next chunk of views
    }
    for (int gl = threadIdx.x; gl < cnt; gl += blockDim.x) sigma_bwd<DEG>(st, gl, acc);
    __syncthreads();
    // write the block's slice of every group (coalesced)
    const Layout L = param_layout(n, DEG);
    const int widths[6] = {3, 3, 4, 1, 3, 3 * (K - 1)};
    const int64_t offs[6] = {L.means, L.scales, L.quats, L.opac, L.dc, L.rest};
    int soff = 0;
    for (int gi = 0; gi < 6; gi++) {
        const int w = widths[gi];
        if (w == 0) continue;
        float *dst = pgrad + offs[gi] + (int64_t)w * g0;
        const float *src = acc + soff;
        for (int i = threadIdx.x; i < w * cnt; i += blockDim.x) dst[i] = accumulate ? dst[i] + src[i] : src[i];
        soff += w * kGB;
    }
    if (stats) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            accum[g0 + i] += dstat[i];
            denom[g0 + i] += dstat[kGB + i];
            max_r2d[g0 + i] = fmaxf(max_r2d[g0 + i], dstat[2 * kGB + i]);
        }
    }
}

template <int DEG>
static size_t pre_smem(int V)
{
    return sizeof(float) * (staged_floats<DEG>() + (size_t)V * kCamF);
}

template <int DEG>
static cudaError_t launch_pre(const float *P, int64_t n, const cgs_camera *cams, int V, const Grid &g,
                              float near_z, float4 *rec, float4 *sgrad, cudaStream_t s)
{
    size_t smem = pre_smem<DEG>(V);
    auto k = k_preprocess<DEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (int)((n + kGB - 1) / kGB);
    k<<<blocks, kPreThreads, smem, s>>>(P, n, cams, V, g, near_z, rec, sgrad);
    return cudaGetLastError();
}

template <int DEG>
static cudaError_t launch_pre_bwd(const float *P, int64_t n, const cgs_camera *cams, int V, const Grid &g,
                                  float near_z, const float4 *rec, const float4 *sgrad, float *pgrad,
                                  int accumulate, float *accum, float *denom, float *maxr, cudaStream_t s)
{
    size_t smem = sizeof(float) * (2 * (size_t)staged_floats<DEG>() + 3 * kGB + (size_t)V * kCamF) +
                  sizeof(uint16_t) * (size_t)kGB * min(V, kViewChunk);
    auto k = k_preprocess_bwd<DEG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (int)((n + kGB - 1) / kGB);
    k<<<blocks, kPreThreads, smem, s>>>(P, n, cams, V, g, near_z, rec, sgrad, pgrad, accumulate, accum,
                                        denom, maxr);
    return cudaGetLastError();
}

cudaError_t preprocess_fwd(const float *P, int64_t n, int deg, const cgs_camera *cams, int V, const Grid &g,
                           float near_z, float *rec, float *sgrad, cudaStream_t s)
{
    float4 *r4 = reinterpret_cast<float4 *>(rec), *g4 = reinterpret_cast<float4 *>(sgrad);
    switch (deg) {
    case 0: return launch_pre<0>(P, n, cams, V, g, near_z, r4, g4, s);
    case 1: return launch_pre<1>(P, n, cams, V, g, near_z, r4, g4, s);
    case 2: return launch_pre<2>(P, n, cams, V, g, near_z, r4, g4, s);
    default: return launch_pre<3>(P, n, cams, V, g, near_z, r4, g4, s);
    }
}

cudaError_t preprocess_bwd(const float *P, int64_t n, int deg, const cgs_camera *cams, int V, const Grid &g,
                           float near_z, const float *rec, const float *sgrad, float *pgrad, int accumulate,
                           float *accum, float *denom, float *maxr, cudaStream_t s)
{
    const float4 *r4 = reinterpret_cast<const float4 *>(rec), *g4 = reinterpret_cast<const float4 *>(sgrad);
    switch (deg) {
    case 0: return launch_pre_bwd<0>(P, n, cams, V, g, near_z, r4, g4, pgrad, accumulate, accum, denom, maxr, s);
    case 1: return launch_pre_bwd<1>(P, n, cams, V, g, near_z, r4, g4, pgrad, accumulate, accum, denom, maxr, s);
    case 2: return launch_pre_bwd<2>(P, n, cams, V, g, near_z, r4, g4, pgrad, accumulate, accum, denom, maxr, s);
    default: return launch_pre_bwd<3>(P, n, cams, V, g, near_z, r4, g4, pgrad, accumulate, accum, denom, maxr, s);
    }
}

}  // namespace cgs
