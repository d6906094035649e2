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

// ------------------------------------------------------------ geometric densification
// A keyframe's coloured point cloud becomes Gaussians (Sec. III-A.3, III-B; the 3DGS
// initialisation): mean = point, isotropic log-scale log sqrt(max(d2, 1e-7)) with d2 the
// mean squared distance to the 3 nearest other points (exact), identity rotation,
// opacity logit(init), SH DC (rgb - 1/2) / Y_0^0, higher bands 0.
//
// Exact k-NN on a uniform grid: bounding box and moments (k_bbox); the grid spans the box
// cut to mean +- 3 standard deviations per axis, points outside fall into the border cells
// (so a few far outliers do not stretch the cells); cell size (k_grid_setup) about one point
// per cell of the box's volume, face area or length, whichever is largest, and at most
// kGridCap cells per axis; counting sort of point ids by cell (k_cell_count, k_count_scan, k_cell_scatter),
// then per point a search over growing rings of cells that stops once the distance to
// the unsearched region, less a rounding margin, is at least the third-best distance.

constexpr int kGridCap = 128;
constexpr int kKnn = 3;
constexpr float kKnnFloor = 1e-7f;
constexpr float kShC0 = 0.28209479177387814f;

struct GridInfo {
    float lo[3];
    float h;
    int G[3];
    float margin;
    uint32_t box[6];   // sortable encodings: min x, y, z, then max x, y, z
    double sum[3], sumsq[3];
};

__host__ __device__ inline int64_t grid_cell_budget(int64_t m)
{
    return m + 3 * (int64_t)kGridCap * kGridCap + 3 * kGridCap + 1;
}

__device__ __forceinline__ uint32_t f2sortable(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float sortable2f(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bbox(const float *__restrict__ xyz, int64_t m, GridInfo *__restrict__ gi, int32_t *status)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; a++) {
            const float x = xyz[3 * i + a];
            if (!isfinite(x)) {
                bad = true;
                continue;
            }
            lo[a] = fminf(lo[a], x);
            hi[a] = fmaxf(hi[a], x);
            s1[a] += x;
            s2[a] += (double)x * x;
        }
    for (int a = 0; a < 3; a++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(kFull, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(kFull, hi[a], o));
            s1[a] += __shfl_xor_sync(kFull, s1[a], o);
            s2[a] += __shfl_xor_sync(kFull, s2[a], o);
        }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) set_status(status, CGS_ERR_NONFINITE);
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; a++) {
            if (lo[a] <= hi[a]) {
                atomicMin(&gi->box[a], f2sortable(lo[a]));
                atomicMax(&gi->box[3 + a], f2sortable(hi[a]));
                atomicAdd(&gi->sum[a], s1[a]);
                atomicAdd(&gi->sumsq[a], s2[a]);
            }
        }
}

__global__ void k_grid_setup(GridInfo *__restrict__ gi, int64_t m, int64_t budget)
{
    if (threadIdx.x != 0) return;
    float lo[3], ext[3];
    float emax = 0.f, amax = 0.f;
    const double mm = (double)(m > 0 ? m : 1);
    for (int a = 0; a < 3; a++) {
        const bool any = gi->box[a] != 0xffffffffu;
        const float blo = any ? sortable2f(gi->box[a]) : 0.f;
        const float bhi = any ? sortable2f(gi->box[3 + a]) : 0.f;
        const double mu = gi->sum[a] / mm;
        const double sd = sqrt(fmax(gi->sumsq[a] / mm - mu * mu, 0.0));
        lo[a] = fmaxf(blo, (float)(mu - 3.0 * sd));
        const float hi = fmaxf(fminf(bhi, (float)(mu + 3.0 * sd)), lo[a]);
        ext[a] = fmaxf(hi - lo[a], 0.f);
        emax = fmaxf(emax, ext[a]);
        amax = fmaxf(amax, fmaxf(fabsf(blo), fabsf(bhi)));
    }
    // extents in ascending order: e0 <= e1 <= e2
    float e0 = fminf(ext[0], fminf(ext[1], ext[2])), e2 = emax;
    float e1 = ext[0] + ext[1] + ext[2] - e0 - e2;
    const double vol = (double)ext[0] * ext[1] * ext[2];
    double h = cbrt(vol / mm);
    h = fmax(h, sqrt((double)e1 * e2 / mm));
    h = fmax(h, (double)e2 / mm);
    h = fmax(h, (double)emax / kGridCap);
    if (!(h > 0.0)) h = 1.0;
    float hf = (float)h;
    int G[3];
    for (int it = 0; it < 64; it++) {          // the cell count stays within the caller's budget
        for (int a = 0; a < 3; a++) {
            const int c = (int)ceil((double)ext[a] / hf);
            G[a] = c < 1 ? 1 : (c > kGridCap ? kGridCap : c);
        }
        if ((int64_t)G[0] * G[1] * G[2] <= budget) break;
        hf *= 1.0625f;
    }
    for (int a = 0; a < 3; a++) {
        gi->G[a] = G[a];
        gi->lo[a] = lo[a];
    }
    gi->h = hf;
    // the float cell index of a point can be off by one near a cell face: a point counted in
    // an unsearched cell may lie this much closer than the face
    gi->margin = 8.f * 1.2e-7f * (amax + 2.f * hf);
}

__device__ __forceinline__ int cell_axis(float x, float lo, float h, int G)
{
    int c = (int)floorf((x - lo) / h);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

__global__ void k_cell_count(const float *__restrict__ xyz, int64_t m, const GridInfo *__restrict__ gi,
                             uint32_t *__restrict__ cell_of, uint32_t *__restrict__ count)
{
    const GridInfo g = *gi;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int cx = cell_axis(xyz[3 * i], g.lo[0], g.h, g.G[0]);
        const int cy = cell_axis(xyz[3 * i + 1], g.lo[1], g.h, g.G[1]);
        const int cz = cell_axis(xyz[3 * i + 2], g.lo[2], g.h, g.G[2]);
        const uint32_t c = (uint32_t)cx + (uint32_t)g.G[0] * ((uint32_t)cy + (uint32_t)g.G[1] * (uint32_t)cz);
        cell_of[i] = c;
        atomicAdd(count + c, 1u);
    }
}

__global__ void k_cell_scatter(int64_t m, const uint32_t *__restrict__ cell_of, const uint32_t *__restrict__ off,
                               uint32_t *__restrict__ count, uint32_t *__restrict__ ids)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cell_of[i];
        ids[off[c] + atomicSub(count + c, 1u) - 1u] = (uint32_t)i;
    }
}

__device__ __forceinline__ void knn_insert(float d, float (&best)[kKnn], int &nb)
{
    if (nb < kKnn) {
        best[nb++] = d;
    } else if (d < best[kKnn - 1]) {
        best[kKnn - 1] = d;
    } else {
        return;
    }
#pragma unroll
    for (int a = kKnn - 1; a > 0; a--)
        if (a < nb && best[a] < best[a - 1]) {
            const float t = best[a];
            best[a] = best[a - 1];
            best[a - 1] = t;
        }
}

__device__ __forceinline__ void knn_cell(const float *__restrict__ xyz, const uint32_t *__restrict__ off,
                                         const uint32_t *__restrict__ ids, uint32_t cell, uint32_t i, float px,
                                         float py, float pz, float (&best)[kKnn], int &nb)
{
    for (uint32_t q = off[cell]; q < off[cell + 1]; q++) {
        const uint32_t j = ids[q];
        if (j == i) continue;
        const float ex = xyz[3 * j] - px, ey = xyz[3 * j + 1] - py, ez = xyz[3 * j + 2] - pz;
        knn_insert(ex * ex + ey * ey + ez * ez, best, nb);
    }
}

// One thread per point, in cell order.  Writes Gaussian n + i of the output layout (m_out).
__global__ void __launch_bounds__(128)
k_knn_init(const float *__restrict__ xyz, const float *__restrict__ rgb, int64_t m, const GridInfo *__restrict__ gi,
           const uint32_t *__restrict__ cell_of, const uint32_t *__restrict__ off, const uint32_t *__restrict__ ids,
           int K, float logit, int64_t n, int64_t n_out, float *__restrict__ Po)
{
    const GridInfo g = *gi;
    const int want = m - 1 < kKnn ? (int)(m - 1) : kKnn;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = ids[t];
        const float px = xyz[3 * i], py = xyz[3 * i + 1], pz = xyz[3 * i + 2];
        const uint32_t c = cell_of[i];
        const int cx = (int)(c % (uint32_t)g.G[0]), cy = (int)((c / (uint32_t)g.G[0]) % (uint32_t)g.G[1]),
                  cz = (int)(c / ((uint32_t)g.G[0] * (uint32_t)g.G[1]));
        float best[kKnn];
        int nb = 0;
        const int rmax = want > 0 ? max(g.G[0], max(g.G[1], g.G[2])) : -1;
        for (int r = 0; r <= rmax; r++) {
            const int z0 = max(-r, -cz), z1 = min(r, g.G[2] - 1 - cz);
            const int y0 = max(-r, -cy), y1 = min(r, g.G[1] - 1 - cy);
            const int x0 = max(-r, -cx), x1 = min(r, g.G[0] - 1 - cx);
            for (int dz = z0; dz <= z1; dz++)
                for (int dy = y0; dy <= y1; dy++) {
                    // cells at Chebyshev distance exactly r: whole rows on the faces dz = +-r or
                    // dy = +-r, else only dx = -r and dx = +r
                    const bool face = dz == -r || dz == r || dy == -r || dy == r;
                    const uint32_t row = (uint32_t)g.G[0] * ((uint32_t)(cy + dy) + (uint32_t)g.G[1] * (uint32_t)(cz + dz));
                    if (face) {
                        for (int dx = x0; dx <= x1; dx++)
                            knn_cell(xyz, off, ids, row + (uint32_t)(cx + dx), i, px, py, pz, best, nb);
                    } else {
                        if (-r >= x0) knn_cell(xyz, off, ids, row + (uint32_t)(cx - r), i, px, py, pz, best, nb);
                        if (r <= x1) knn_cell(xyz, off, ids, row + (uint32_t)(cx + r), i, px, py, pz, best, nb);
                    }
                }
            // distance from the point to the region outside the searched block of cells
            float bound = INFINITY;
            const float p[3] = {px, py, pz};
            const int cc3[3] = {cx, cy, cz};
            for (int a = 0; a < 3; a++) {
                if (cc3[a] - r > 0) bound = fminf(bound, p[a] - (g.lo[a] + (float)(cc3[a] - r) * g.h));
                if (cc3[a] + r < g.G[a] - 1) bound = fminf(bound, (g.lo[a] + (float)(cc3[a] + r + 1) * g.h) - p[a]);
            }
            if (bound == INFINITY) break;                   // every cell searched
            const float b = bound - g.margin;
            if (nb >= want && b > 0.f && b * b >= best[want - 1] * (1.f + 1e-6f)) break;
        }
        float d2 = 0.f;
        for (int a = 0; a < nb; a++) d2 += best[a];
        d2 = nb ? d2 / (float)nb : 0.f;
        const float ls = 0.5f * logf(fmaxf(d2, kKnnFloor));
        const int64_t j = n + i;
        for (int a = 0; a < 3; a++) {
            Po[3 * j + a] = xyz[3 * i + a];
            Po[3 * n_out + 3 * j + a] = ls;
            Po[11 * n_out + 3 * j + a] = (rgb[3 * i + a] - 0.5f) / kShC0;
        }
        Po[6 * n_out + 4 * j] = 1.f;
        Po[6 * n_out + 4 * j + 1] = 0.f;
        Po[6 * n_out + 4 * j + 2] = 0.f;
        Po[6 * n_out + 4 * j + 3] = 0.f;
        Po[10 * n_out + j] = logit;
        for (int a = 0; a < 3 * (K - 1); a++) Po[14 * n_out + (int64_t)3 * (K - 1) * j + a] = 0.f;
    }
}

// Gaussians 0..n-1 of the input layout (n) to the same indices of the output layout.
__global__ void k_copy_prefix(const float *__restrict__ P, const float *__restrict__ Mi, const float *__restrict__ Vi,
                              int64_t n, int K, int64_t n_out, float *__restrict__ Po, float *__restrict__ Mo,
                              float *__restrict__ Vo)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
        copy_gaussian(P, Mi, Vi, n, g, Po, Mo, Vo, n_out, g, K, true);
}

// Zero Adam moments of Gaussians n..n_out-1.
__global__ void k_zero_tail(int64_t n, int K, int64_t n_out, float *__restrict__ Mo, float *__restrict__ Vo)
{
    const int widths[6] = {3, 3, 4, 1, 3, 3 * (K - 1)};
    for (int64_t g = n + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_out;
         g += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = 0;
        for (int gi = 0; gi < 6; gi++) {
            for (int c = 0; c < widths[gi]; c++) {
                Mo[o + (int64_t)widths[gi] * g + c] = 0.f;
                Vo[o + (int64_t)widths[gi] * g + c] = 0.f;
            }
            o += (int64_t)widths[gi] * n_out;
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

size_t cgs_points_workspace(int64_t n_points)
{
    if (n_points < 1) return 0;
    const int64_t B = grid_cell_budget(n_points);
    return al256(sizeof(GridInfo)) + 2 * al256(sizeof(uint32_t) * (size_t)n_points) +
           2 * al256(sizeof(uint32_t) * ((size_t)B + 1)) + al256(sizeof(int64_t));
}

int cgs_points_to_gaussians(const float *params, const float *m, const float *v, int64_t n, int32_t sh_degree,
                            const float *xyz, const float *rgb, int64_t n_points, float init_opacity,
                            void *workspace, size_t workspace_bytes, float *params_out, float *m_out,
                            float *v_out, int32_t *status_dev, void *stream)
{
    if (n < 0 || n_points < 0 || n + n_points < 1 || sh_degree < 0 || sh_degree > 3) return CGS_ERR_ARG;
    if (n > 0 && (!params || !m || !v)) return CGS_ERR_ARG;
    if (!params_out || !m_out || !v_out) return CGS_ERR_ARG;
    if (n_points > 0 && (!xyz || !rgb || !workspace)) return CGS_ERR_ARG;
    if (!(init_opacity > 0.f && init_opacity < 1.f)) return CGS_ERR_ARG;
    if (grid_cell_budget(n_points) + 1 >= ((int64_t)1 << 32)) return CGS_ERR_ARG;
    const int K = (sh_degree + 1) * (sh_degree + 1);
    const int64_t n_out = n + n_points;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t big = n > n_points ? n : n_points;
    const int blocks = (int)((big + 255) / 256 < 4096 ? (big + 255) / 256 : 4096);
    if (n > 0) k_copy_prefix<<<blocks, 256, 0, s>>>(params, m, v, n, K, n_out, params_out, m_out, v_out);
    if (n_points == 0) return st_of(cudaGetLastError());
    if (((uintptr_t)workspace & 255) != 0) return CGS_ERR_ARG;
    if (workspace_bytes < cgs_points_workspace(n_points)) return CGS_ERR_WORKSPACE;
    const int64_t B = grid_cell_budget(n_points);
    char *w = static_cast<char *>(workspace);
    GridInfo *gi = reinterpret_cast<GridInfo *>(w);
    w += al256(sizeof(GridInfo));
    uint32_t *cell_of = reinterpret_cast<uint32_t *>(w);
    w += al256(sizeof(uint32_t) * n_points);
    uint32_t *ids = reinterpret_cast<uint32_t *>(w);
    w += al256(sizeof(uint32_t) * n_points);
    uint32_t *count = reinterpret_cast<uint32_t *>(w);
    w += al256(sizeof(uint32_t) * (B + 1));
    uint32_t *off = reinterpret_cast<uint32_t *>(w);
    w += al256(sizeof(uint32_t) * (B + 1));
    int64_t *total = reinterpret_cast<int64_t *>(w);
    cudaError_t e = cudaMemsetAsync(gi, 0, sizeof(GridInfo), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gi->box, 0xff, 3 * sizeof(uint32_t), s);   // minima start high
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * (B + 1), s);
    if (e != cudaSuccess) return st_of(e);
    const float logit = logf(init_opacity / (1.f - init_opacity));
    const int pb = (int)((n_points + 255) / 256 < 1024 ? (n_points + 255) / 256 : 1024);
    k_bbox<<<pb, 256, 0, s>>>(xyz, n_points, gi, status_dev);
    k_grid_setup<<<1, 32, 0, s>>>(gi, n_points, B);
    k_cell_count<<<pb, 256, 0, s>>>(xyz, n_points, gi, cell_of, count);
    k_count_scan<<<1, 1024, 0, s>>>(count, B, off, total);
    k_cell_scatter<<<pb, 256, 0, s>>>(n_points, cell_of, off, count, ids);
    const int kb = (int)((n_points + 127) / 128 < 8192 ? (n_points + 127) / 128 : 8192);
    k_knn_init<<<kb, 128, 0, s>>>(xyz, rgb, n_points, gi, cell_of, off, ids, K, logit, n, n_out, params_out);
    k_zero_tail<<<pb, 256, 0, s>>>(n, K, n_out, m_out, v_out);
    return st_of(cudaGetLastError());
}

}  // extern "C"
