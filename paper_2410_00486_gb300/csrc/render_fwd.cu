// Forward blend of Eq. 1 (Sec. III-B, CaRtGS) with the L1 loss fused in.
//
// One block per (view, tile), two pixels of one column per thread (4 rows apart).  The
// tile's depth-sorted list (only splats that can reach alpha >= 1/255 in the tile: the
// binning's test) is consumed in batches of BD splats: the block gathers the records of a
// batch (48 bytes each, one per thread) into shared memory; every pixel then walks the
// batch front to back, rejecting a pair on its base-2 exponent (|power| > -tau, both
// scaled by log2 e) before any exponential.  A block-wide vote (__syncthreads_count) ends the walk
// as soon as every pixel of the tile is saturated (T below 1e-4).
#include "raster.cuh"

namespace cgs {

// Row coordinate of a finished pixel (outside the image, or saturated): a quiet NaN, so
// its exponent is NaN and it fails the alpha test with no branch of its own.
__device__ constexpr float kNoRow = __builtin_nanf("");

template <int B, int BD, bool CKPT, bool COUNT>
__global__ void __launch_bounds__(B *B / ppt_for<B, kPPTFwd>(), (min_blocks_for<B, kPPTFwd, kFwdMinWarps>())) k_render_fwd(RasterFwdArgs a)
{
    constexpr int PPT = ppt_for<B, kPPTFwd>();
    constexpr int NT = B * B / PPT;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[BD], s1[BD], s2[BD];
    __shared__ float red[5][NW];
    int64_t tile;
    int view, tx, ty;
    item_tile(a.order, a.g, tile, view, tx, ty, blockIdx.x);
    // Warp w owns the 8x8 block w of the tile (blocks row-major, B / 8 per row); lane l
    // takes column l % 8 of it and rows l / 8 and l / 8 + 4, so each step over a thread's
    // pixels covers 8 columns x 4 rows: a compact footprint, where fewer steps hold a
    // splat's edge, so fewer of a warp's lanes idle in the blend (1.721 -> 1.667 ms on the
    // 16-view window against 16 columns x 2 rows, images identical)
    static_assert(PPT == 2 && NT * 2 == B * B, "two pixels per thread");
    const int wq = (int)threadIdx.x >> 5, lq = (int)threadIdx.x & 31;
    const int col = 8 * (wq % (B / 8)) + (lq & 7);
    const int row0 = 8 * (wq / (B / 8)) + (lq >> 3);
    constexpr int G = 4;
    const int px = tx * B + col;
    const int py0 = ty * B + row0;   // row of pixel p: py0 + G p
    const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
    const float fx = (float)px;

    float fy[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT];
    uint32_t lst[PPT];
    bool done[PPT];
    bool tdone = true;
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        fy[p] = (float)(py0 + G * p);
        T[p] = 1.f;
        C0[p] = C1[p] = C2[p] = D[p] = 0.f;
        lst[p] = 0;
        done[p] = !(px < a.g.W && py0 + G * p < a.g.H);
        if (done[p]) fy[p] = kNoRow;
        tdone = tdone && done[p];
    }
    uint32_t n_eval = 0, n_blend = 0, active = 0;
    uint32_t next_ck = kBucket;   // next checkpoint boundary (list position)
    const int64_t ck_base = CKPT ? (int64_t)a.bucket_start[tile] : 0;
    const int pix0 = row0 * B + col;   // pixel index in the tile
#pragma unroll
    for (int p = 0; p < PPT; p++) active += done[p] ? 0u : 1u;
    for (uint32_t base = start; base < end; base += BD) {
        if (__syncthreads_count(!tdone) == 0) break;
        // stage the batch (every entry of a tile's list can reach the tile: the binning
        // left out the rest)
        const int cnt = (int)min((uint32_t)BD, end - base);
        for (int i = threadIdx.x; i < cnt; i += NT) {
            const uint32_t idx = base + (uint32_t)i;
            const float4 *r = a.rec + kRec4 * (size_t)__ldg(a.vals + idx);
            const float4 r2 = __ldg(r + 2);
            stage_splat(__ldg(r), __ldg(r + 1), r2.w, s0[i], s1[i]);
            s2[i] = r2;
        }
        __syncthreads();
        if (!tdone) {
#pragma unroll 4
            for (int j = 0; j < cnt; j++) {
                const uint32_t pos = base - start + (uint32_t)j;   // list position of splat j
                if (CKPT) {
                    // save the state of this thread's pixels at every boundary up to this splat
                    while (next_ck <= pos) {
                        const int64_t bk = ck_base + (int64_t)(next_ck / kBucket);
                        if (bk < a.max_buckets) {
#pragma unroll
                            for (int p = 0; p < PPT; p++) {
                                const int64_t q = bk * (B * B) + pix0 + G * p * B;
                                a.ck4[q] = make_float4(T[p], C0[p], C1[p], C2[p]);
                                a.ckD[q] = D[p];
                            }
                        }
                        next_ck += kBucket;
                    }
                }
                const float4 q0 = s0[j];
                const float4 q1 = s1[j];
                const float4 q2 = s2[j];
                const PowerX pxs = power_x(q0, __fsub_rn(q0.x, fx));
#pragma unroll
                for (int p = 0; p < PPT; p++) {
                    const float power = power_at(pxs, q1.x, __fsub_rn(q0.y, fy[p]));
                    // the alpha >= 1/255 test; a finished pixel (row NaN, so power NaN) fails it
                    if (!(fabsf(power) <= q1.w)) continue;
                    const float alpha = fminf(kAlphaMax, __fmul_rn(q1.y, exp2_fast(power)));
                    const float wgt = __fmul_rn(alpha, T[p]);
                    const float testT = __fsub_rn(T[p], wgt);   // T (1 - alpha)
                    if (testT < kTMin) {
                        done[p] = true;
                        fy[p] = kNoRow;
                        active--;
                        n_eval += pos + 1u;    // work count: list entries this pixel evaluated
                        if (active == 0u) goto walked;   // every pixel of the thread is finished
                        continue;
                    }
                    C0[p] = fmaf(q2.x, wgt, C0[p]);
                    C1[p] = fmaf(q2.y, wgt, C1[p]);
                    C2[p] = fmaf(q2.z, wgt, C2[p]);
                    D[p] = fmaf(q1.z, wgt, D[p]);
                    T[p] = testT;
                    lst[p] = pos + 1u;
                    if (COUNT) n_blend++;
                }
            }
        walked:
            tdone = true;
#pragma unroll
            for (int p = 0; p < PPT; p++) tdone = tdone && done[p];
        }
    }

    n_eval += active * (end - start);   // pixels that never stopped evaluated the whole list
    float l_rgb = 0.f, l_d = 0.f, c_d = 0.f;
    const size_t HW = (size_t)a.g.W * a.g.H;
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        const int py = py0 + G * p;
        if (!(px < a.g.W && py < a.g.H)) continue;
        const size_t q = (size_t)py * a.g.W + px;
        const size_t pix = (size_t)view * HW + q;
        const float I0 = fmaf(T[p], a.bg0, C0[p]), I1 = fmaf(T[p], a.bg1, C1[p]), I2 = fmaf(T[p], a.bg2, C2[p]);
        float *im = a.img + (size_t)view * 3 * HW + q;
        im[0] = I0;
        im[HW] = I1;
        im[2 * HW] = I2;
        a.depth[pix] = D[p];
        a.tfin[pix] = T[p];
        a.last[pix] = lst[p];
        if (a.tgt_rgb) {
            const float *tr = a.tgt_rgb + (size_t)view * 3 * HW + q;
            l_rgb += fabsf(I0 - tr[0]) + fabsf(I1 - tr[HW]) + fabsf(I2 - tr[2 * HW]);
            if (a.tgt_depth) {
                const float td = a.tgt_depth[pix];
                if (td > 0.f) {
                    l_d += fabsf(D[p] - td);
                    c_d += 1.f;
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
    const int nt = B * B / ppt_for<B, kPPTFwd>();
    if (a.ck4)   // the checkpointing forward does not count blended pairs
        k_render_fwd<B, BD, true, false><<<(unsigned)items, nt, 0, s>>>(a);
    else if (a.count_blend)
        k_render_fwd<B, BD, false, true><<<(unsigned)items, nt, 0, s>>>(a);
    else
        k_render_fwd<B, BD, false, false><<<(unsigned)items, nt, 0, s>>>(a);
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

// ---------------------------------------------------------------------------------
// cgs_render_fwd_noalloc: the forward render with its scratch inside the library.
//
// Some callers cannot hand the library a workspace: a real-time mapping thread that
// must not allocate once it is running (a device allocation can block in the CUDA driver
// and miss the frame budget), or code that only ever sees the input and output
// buffers of another framework.  For them the per-tile partial sums live in this
// file-scope device array, sized for kNoAllocMaxTiles tiles (V * tiles per view);
// every GPU that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------------
#include <mutex>
#include <stdio.h>

namespace cgs {

constexpr int64_t kNoAllocMaxTiles = 65536;
static __device__ __align__(256) float g_fwd_scratch[kNoAllocMaxTiles * kPartials];

// Device address of g_fwd_scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is queried with
// cudaGetSymbolAddress once per device (with that device current) and cached.
static float *noalloc_scratch()
{
    static std::mutex mu;
    static float *ptr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fwd_scratch);
        if (e != cudaSuccess) {
            fprintf(stderr, "libcgs: cudaGetSymbolAddress(scratch) failed: %s\n", cudaGetErrorString(e));
            return nullptr;
        }
        ptr[dev] = static_cast<float *>(p);
    }
    return ptr[dev];
}

}  // namespace cgs

extern "C" int cgs_render_fwd_noalloc(const float *rec, const uint32_t *vals, const uint32_t *ranges,
                                      const uint32_t *tile_order, int32_t V, const cgs_config *cfg,
                                      const float *view_weight, const float *tgt_rgb, const float *tgt_depth,
                                      float *img, float *depth, float *t_final, uint32_t *last, float *loss_view,
                                      int32_t *depth_count, int32_t *status_dev, void *stream)
{
    using namespace cgs;
    // the same argument checks as cgs_render_fwd (without the workspace)
    if (!rec || !vals || !ranges || !img || !depth || !t_final || !last || !cfg_ok(cfg)) return CGS_ERR_ARG;
    if (V < 1 || V > kMaxViews || !aligned16(rec)) return CGS_ERR_ARG;
    if (tgt_depth && !tgt_rgb) return CGS_ERR_ARG;
    if (tgt_rgb && (!loss_view || !depth_count)) return CGS_ERR_ARG;
    const Grid g = make_grid(*cfg);
    if (g.Tv * V > kNoAllocMaxTiles) {
        fprintf(stderr, "libcgs: cgs_render_fwd_noalloc: %lld tiles exceed the built-in maximum of %lld\n",
                (long long)(g.Tv * V), (long long)kNoAllocMaxTiles);
        return CGS_ERR_WORKSPACE;
    }
    float *scratch = noalloc_scratch();
    if (!scratch) return CGS_ERR_CUDA;
    RasterFwdArgs a;
    a.rec = reinterpret_cast<const float4 *>(rec);
    a.vals = vals;
    a.ranges = ranges;
    a.order = tile_order;
    a.g = g;
    a.V = V;
    a.bg0 = cfg->bg[0];
    a.bg1 = cfg->bg[1];
    a.bg2 = cfg->bg[2];
    a.tgt_rgb = tgt_rgb;
    a.tgt_depth = tgt_depth;
    a.img = img;
    a.depth = depth;
    a.tfin = t_final;
    a.last = last;
    a.partials = scratch;   // every entry the reduction reads is written first: nothing to clear
    a.ck4 = nullptr;
    a.ckD = nullptr;
    a.bucket_start = nullptr;
    a.max_buckets = 0;
    a.count_blend = cfg->count_work != 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = raster_fwd(a, cfg->tile, cfg->batch_depth, s);
    if (e == cudaSuccess && tgt_rgb)
        e = loss_reduce(a.partials, g, V, view_weight, cfg->lambda_depth, loss_view, depth_count, status_dev, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "libcgs: CUDA error: %s\n", cudaGetErrorString(e));
        return CGS_ERR_CUDA;
    }
    return CGS_OK;
}
