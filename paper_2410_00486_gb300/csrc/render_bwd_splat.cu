// Splat-wise backward of the blend (Sec. III-C.1, Fig. 4a, CaRtGS; Eqs. 2-4), the
// parallelisation the paper adopts in place of the pixel-wise one.
//
// Forward side (cgs_render_fwd_ckpt): the forward saves, for every pixel, its state
// X_{i,j} = (T, accumulated colour, accumulated depth) before list positions 32, 64, ...
// of its tile ("pixel states for every 32nd splat").  Buckets are counted per tile as
// ceil(len / 32) by k_bucket_scan; only boundaries a still-active pixel reaches are
// written.
//
// Backward side (k_render_bwd_splat): one block per tile; each warp takes buckets of 32
// consecutive list positions, one splat per lane.  The per-pixel constants of the tile
// (pixel gradients, final colour/depth, last position) are staged in shared memory and
// the bucket's 256 checkpoints are copied into the warp's shared-memory slice.  Pixel
// states then flow through the warp as a pipeline: at step s lane i holds pixel s - i,
// applies its splat (state after splats 0..i-1 of the bucket, X_{i,j} -> X_{i+1,j}) and
// hands the state to lane i + 1 with one shuffle per state value.  Each lane accumulates
// its splat's gradient over all pixels in registers (Eq. 4) and issues its ten atomic
// adds once per tile.  The colour behind splat i comes from the final colour:
// C_final - C_{i+1}, with C_{i+1} recomputed by exactly the forward's operation sequence,
// so every decision and value equals the forward's.
#include <algorithm>
#include <stdio.h>

#include "raster.cuh"

namespace cgs {

constexpr int kSplatThreads = 128;
constexpr int kSplatWarps = kSplatThreads / 32;

// bucket_start[t] = sum over tiles t' < t of ceil(len_t' / 32); bucket_start[Ttot] = total.
__global__ void __launch_bounds__(1024)
k_bucket_scan(const uint32_t *__restrict__ ranges, int64_t Ttot, int64_t max_buckets,
              uint32_t *__restrict__ bucket_start, int32_t *__restrict__ status)
{
    __shared__ unsigned long long wtot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (Ttot + 31) / 32;
    const int64_t lo = (int64_t)w * per, hi = min(Ttot, lo + per);
    unsigned long long s = 0;
    for (int64_t t = lo + lane; t < hi; t += 32) s += (ranges[2 * t + 1] - ranges[2 * t] + kBucket - 1) / kBucket;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if (lane == 0) wtot[w] = s;
    __syncthreads();
    unsigned long long run = 0, total = 0;
    for (int i = 0; i < 32; i++) {
        run += (i < w) ? wtot[i] : 0ull;
        total += wtot[i];
    }
    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t t = base + lane;
        const unsigned long long c = t < hi ? (ranges[2 * t + 1] - ranges[2 * t] + kBucket - 1) / kBucket : 0ull;
        unsigned long long incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        if (t < hi) bucket_start[t] = (uint32_t)min(run + incl - c, 0xffffffffull);
        run += __shfl_sync(kFull, incl, 31);
    }
    if (threadIdx.x == 0) {
        bucket_start[Ttot] = (uint32_t)min(total, 0xffffffffull);
        if ((int64_t)total > max_buckets) set_status(status, CGS_ERR_CAPACITY);
    }
}

template <int B>
__global__ void __launch_bounds__(kSplatThreads)
k_render_bwd_splat(RasterBwdArgs a, const float4 *__restrict__ ck4, const float *__restrict__ ckD,
                   const uint32_t *__restrict__ bucket_start, int64_t max_buckets)
{
    constexpr int NP = B * B;
    __shared__ float4 pA[NP];              // (gI0, gI1, gI2, gD)
    __shared__ float4 pB[NP];              // final colour (without background) and depth
    __shared__ float2 pC[NP];              // (T_final (bg . gI), last as bits)
    __shared__ float4 sck[kSplatWarps][NP];  // the warp's bucket checkpoints (T, C)
    __shared__ float sckD[kSplatWarps][NP];
    __shared__ uint32_t smax[kSplatWarps];
    int64_t tile;
    int view, tx, ty;
    item_tile(a.order, a.g, tile, view, tx, ty, blockIdx.x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t start = a.ranges[2 * tile];
    const uint32_t len = a.ranges[2 * tile + 1] - start;
    const size_t HW = (size_t)a.g.W * a.g.H;

    uint32_t m = 0;
    for (int p = threadIdx.x; p < NP; p += kSplatThreads) {
        const int px = tx * B + p % B, py = ty * B + p / B;
        float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), fb = ga;
        float bgdot = 0.f;
        uint32_t lst = 0;
        if (px < a.g.W && py < a.g.H) {
            const size_t q = (size_t)py * a.g.W + px;
            const size_t pix = (size_t)view * HW + q;
            lst = min(a.last[pix], len);
            const float Tf = a.tfin[pix];
            const float *im = a.img + (size_t)view * 3 * HW + q;
            if (a.dl_dimg) {
                const float *gi = a.dl_dimg + (size_t)view * 3 * HW + q;
                ga = make_float4(gi[0], gi[HW], gi[2 * HW], a.dl_ddepth ? a.dl_ddepth[pix] : 0.f);
            } else {
                const float wv = a.weight ? a.weight[view] : 1.f;
                const float sc = wv / (3.f * (float)HW);
                const float *tr = a.tgt_rgb + (size_t)view * 3 * HW + q;
                ga.x = sc * ((im[0] > tr[0]) ? 1.f : ((im[0] < tr[0]) ? -1.f : 0.f));
                ga.y = sc * ((im[HW] > tr[HW]) ? 1.f : ((im[HW] < tr[HW]) ? -1.f : 0.f));
                ga.z = sc * ((im[2 * HW] > tr[2 * HW]) ? 1.f : ((im[2 * HW] < tr[2 * HW]) ? -1.f : 0.f));
                if (a.tgt_depth) {
                    const float td = a.tgt_depth[pix];
                    const int cnt = a.depth_count[view];
                    const float dd = a.depth[pix] - td;
                    if (td > 0.f && cnt > 0)
                        ga.w = wv * a.lambda_d * ((dd > 0.f) ? 1.f : ((dd < 0.f) ? -1.f : 0.f)) / (float)cnt;
                }
            }
            // final accumulated colour without the background: img = C + T_final bg
            fb = make_float4(im[0] - Tf * a.bg0, im[HW] - Tf * a.bg1, im[2 * HW] - Tf * a.bg2, a.depth[pix]);
            bgdot = Tf * (a.bg0 * ga.x + a.bg1 * ga.y + a.bg2 * ga.z);
        }
        pA[p] = ga;
        pB[p] = fb;
        pC[p] = make_float2(bgdot, __uint_as_float(lst));
        m = max(m, lst);
    }
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(kFull, m, off));
    if (lane == 0) smax[w] = m;
    __syncthreads();
    uint32_t maxlast = 0;
    for (int i = 0; i < kSplatWarps; i++) maxlast = max(maxlast, smax[i]);
    const int nbk = (int)((maxlast + kBucket - 1) / kBucket);
    const int64_t bbase = bucket_start[tile];
    for (int k = w; k < nbk; k += kSplatWarps) {
        const uint32_t pos = (uint32_t)(k * kBucket + lane);
        bool keep = false;
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0, q2 = q0;
        uint32_t slot = 0;
        if (pos < maxlast) {
            slot = __ldg(a.vals + start + pos);
            const float4 *r = a.rec + kRec4 * (size_t)slot;
            keep = true;
            q2 = __ldg(r + 2);
            stage_splat(__ldg(r), __ldg(r + 1), q2.w, q0, q1);
        }
        if (__ballot_sync(kFull, keep) == 0u) continue;
        // this bucket's checkpoints (state before position 32 k) into the warp's slice
        const int64_t bk = bbase + k;
        for (int p = lane; p < NP; p += 32) {
            if (k == 0 || bk >= max_buckets) {
                sck[w][p] = make_float4(1.f, 0.f, 0.f, 0.f);
                sckD[w][p] = 0.f;
            } else {
                sck[w][p] = ck4[bk * NP + p];
                sckD[w][p] = ckD[bk * NP + p];
            }
        }
        __syncwarp();
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f, g6 = 0.f, g8 = 0.f, g9 = 0.f, g10 = 0.f;
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
        for (int st = 0; st < NP + 31; st++) {
            // pipeline: take the state lane - 1 produced one step ago; lane 0 starts pixel st
            const float rT = __shfl_up_sync(kFull, T, 1), rC0 = __shfl_up_sync(kFull, C0, 1);
            const float rC1 = __shfl_up_sync(kFull, C1, 1), rC2 = __shfl_up_sync(kFull, C2, 1);
            const float rD = __shfl_up_sync(kFull, D, 1);
            const int p = st - lane;
            if (lane == 0) {
                if (st < NP) {
                    const float4 c = sck[w][st];
                    T = c.x;
                    C0 = c.y;
                    C1 = c.z;
                    C2 = c.w;
                    D = sckD[w][st];
                }
            } else {
                T = rT;
                C0 = rC0;
                C1 = rC1;
                C2 = rC2;
                D = rD;
            }
            if (!keep || p < 0 || p >= NP) continue;
            const float2 pc = pC[p];
            if (!(pos < __float_as_uint(pc.y))) continue;
            const float dx = __fsub_rn(q0.x, (float)(tx * B + p % B));
            const float dy = __fsub_rn(q0.y, (float)(ty * B + p / B));
            const float power = staged_power(q0, q1.x, dx, dy);
            if (!(fabsf(power) <= q1.w)) continue;
            const float G = exp2_fast(power);
            const float araw = __fmul_rn(q1.y, G);
            const float alpha = fminf(kAlphaMax, araw);
            // the forward's blend step, bit for bit
            const float wT = __fmul_rn(alpha, T);
            const float n0 = fmaf(q2.x, wT, C0), n1 = fmaf(q2.y, wT, C1), n2 = fmaf(q2.z, wT, C2);
            const float nD = fmaf(q1.z, wT, D);
            const float4 ga = pA[p], fb = pB[p];
            const float inv_om = rcp_fast(__fsub_rn(1.f, alpha));
            g8 += wT * ga.x;
            g9 += wT * ga.y;
            g10 += wT * ga.z;
            g6 += wT * ga.w;
            // dI/dalpha = c T - (C_final - C_after) / (1 - alpha) - T_final bg / (1 - alpha)
            const float dLda = ga.x * (q2.x * T - (fb.x - n0) * inv_om) + ga.y * (q2.y * T - (fb.y - n1) * inv_om) +
                               ga.z * (q2.z * T - (fb.z - n2) * inv_om) + ga.w * (q1.z * T - (fb.w - nD) * inv_om) -
                               pc.x * inv_om;
            if (!(araw > kAlphaMax)) {
                const float dp = dLda * alpha;
                g5 += dLda * G;
                const float dpx = dp * dx, dpy = dp * dy;
                g0 += dpx;
                g1 += dpy;
                g2 += dpx * dx;
                g3 += dpx * dy;
                g4 += dpy * dy;
            }
            C0 = n0;
            C1 = n1;
            C2 = n2;
            D = nD;
            T = __fsub_rn(T, wT);   // T (1 - alpha), rounded as the forward does
        }
        if (keep) {
            float *gp = a.sgrad + (size_t)slot * 12;
            // staged q0.z = -A/2, q0.w = -B, q1.x = -C/2
            atomicAdd(gp + 0, kLn2 * (2.f * q0.z * g0 + q0.w * g1));   // staged terms carry log2 e
            atomicAdd(gp + 1, kLn2 * (2.f * q1.x * g1 + q0.w * g0));
            atomicAdd(gp + 2, -0.5f * g2);
            atomicAdd(gp + 3, -g3);
            atomicAdd(gp + 4, -0.5f * g4);
            atomicAdd(gp + 5, g5);
            atomicAdd(gp + 6, g6);
            atomicAdd(gp + 8, g8);
            atomicAdd(gp + 9, g9);
            atomicAdd(gp + 10, g10);
        }
        __syncwarp();
    }
}

}  // namespace cgs

using namespace cgs;

namespace {

bool cfg_valid(const cgs_config *c)
{
    if (!c) return false;
    if (c->width < 1 || c->height < 1 || c->width > (1 << 16) || c->height > (1 << 16)) return false;
    if (c->tile != 8 && c->tile != 16 && c->tile != 32) return false;
    if (c->batch_depth != 32 && c->batch_depth != 64 && c->batch_depth != 128 && c->batch_depth != 256) return false;
    return true;
}

int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return CGS_OK;
    fprintf(stderr, "libcgs: CUDA error: %s\n", cudaGetErrorString(e));
    return CGS_ERR_CUDA;
}

}  // namespace

namespace cgs {
cudaError_t loss_reduce(const float *partials, const Grid &g, int V, const float *weight, float lambda_d,
                        float *loss_view, int32_t *depth_count, int32_t *status, cudaStream_t s);
}

extern "C" {

size_t cgs_ckpt_bytes(int64_t max_buckets, const cgs_config *cfg)
{
    if (!cfg_valid(cfg) || max_buckets < 0) return 0;
    return (size_t)max_buckets * (size_t)cfg->tile * (size_t)cfg->tile * (sizeof(float4) + sizeof(float));
}

int cgs_render_fwd_ckpt(const float *rec, const uint32_t *vals, const uint32_t *ranges, const uint32_t *tile_order,
                        int32_t V, const cgs_config *cfg, const float *view_weight, const float *tgt_rgb,
                        const float *tgt_depth, float *img, float *depth, float *t_final, uint32_t *last,
                        float *loss_view, int32_t *depth_count, void *workspace, size_t workspace_bytes, float *ckpt,
                        int64_t max_buckets, uint32_t *bucket_start, int32_t *status_dev, void *stream)
{
    if (!rec || !vals || !ranges || !img || !depth || !t_final || !last || !cfg_valid(cfg)) return CGS_ERR_ARG;
    if (V < 1 || V > 1024 || ((uintptr_t)rec & 15) != 0 || !ckpt || ((uintptr_t)ckpt & 15) != 0) return CGS_ERR_ARG;
    if (!bucket_start || max_buckets < 0 || !workspace) return CGS_ERR_ARG;
    if (tgt_depth && !tgt_rgb) return CGS_ERR_ARG;
    if (tgt_rgb && (!loss_view || !depth_count)) return CGS_ERR_ARG;
    const Grid g = make_grid(*cfg);
    if (g.Tv * V >= ((int64_t)1 << 31)) return CGS_ERR_ARG;
    if (workspace_bytes < sizeof(float) * kPartials * (size_t)g.Tv * V) return CGS_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    k_bucket_scan<<<1, 1024, 0, s>>>(ranges, g.Tv * V, max_buckets, bucket_start, status_dev);
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
    a.partials = static_cast<float *>(workspace);
    a.ck4 = reinterpret_cast<float4 *>(ckpt);
    a.ckD = ckpt + 4 * (size_t)max_buckets * cfg->tile * cfg->tile;
    a.bucket_start = bucket_start;
    a.max_buckets = max_buckets;
    a.count_blend = cfg->count_work != 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = raster_fwd(a, cfg->tile, cfg->batch_depth, s);
    if (e == cudaSuccess && tgt_rgb)
        e = loss_reduce(a.partials, g, V, view_weight, cfg->lambda_depth, loss_view, depth_count, status_dev, s);
    return status_of(e);
}

int cgs_raster_bwd_splat(const float *rec, const uint32_t *vals, const uint32_t *ranges, const uint32_t *tile_order,
                         int32_t V, const cgs_config *cfg, const float *view_weight, const float *img,
                         const float *depth, const float *t_final, const uint32_t *last, const float *tgt_rgb,
                         const float *tgt_depth, const int32_t *depth_count, const float *dl_dimg,
                         const float *dl_ddepth, const float *ckpt, int64_t max_buckets, const uint32_t *bucket_start,
                         float *slot_grad, int32_t *status_dev, void *stream)
{
    (void)status_dev;
    if (!rec || !vals || !ranges || !t_final || !last || !slot_grad || !img || !depth || !cfg_valid(cfg))
        return CGS_ERR_ARG;
    if (V < 1 || V > 1024 || ((uintptr_t)rec & 15) != 0 || ((uintptr_t)slot_grad & 15) != 0) return CGS_ERR_ARG;
    if (!ckpt || ((uintptr_t)ckpt & 15) != 0 || !bucket_start || max_buckets < 0) return CGS_ERR_ARG;
    if (!dl_dimg && !tgt_rgb) return CGS_ERR_ARG;
    if (!dl_dimg && tgt_depth && !depth_count) return CGS_ERR_ARG;
    const Grid g = make_grid(*cfg);
    if (g.Tv * V >= ((int64_t)1 << 31)) return CGS_ERR_ARG;
    RasterBwdArgs a;
    a.rec = reinterpret_cast<const float4 *>(rec);
    a.vals = vals;
    a.ranges = ranges;
    a.order = tile_order;
    a.g = g;
    a.V = V;
    a.bg0 = cfg->bg[0];
    a.bg1 = cfg->bg[1];
    a.bg2 = cfg->bg[2];
    a.weight = view_weight;
    a.img = img;
    a.depth = depth;
    a.tfin = t_final;
    a.last = last;
    a.tgt_rgb = tgt_rgb;
    a.tgt_depth = dl_dimg ? nullptr : tgt_depth;
    a.depth_count = depth_count;
    a.lambda_d = cfg->lambda_depth;
    a.dl_dimg = dl_dimg;
    a.dl_ddepth = dl_ddepth;
    a.sgrad = slot_grad;
    a.work = nullptr;
    const float4 *ck4 = reinterpret_cast<const float4 *>(ckpt);
    const float *ckD = ckpt + 4 * (size_t)max_buckets * cfg->tile * cfg->tile;
    const unsigned items = (unsigned)(g.Tv * V);
    cudaStream_t s = (cudaStream_t)stream;
    switch (cfg->tile) {
    case 8: k_render_bwd_splat<8><<<items, kSplatThreads, 0, s>>>(a, ck4, ckD, bucket_start, max_buckets); break;
    case 16: k_render_bwd_splat<16><<<items, kSplatThreads, 0, s>>>(a, ck4, ckD, bucket_start, max_buckets); break;
    default: return CGS_ERR_ARG;   // 32x32 tiles: the per-warp checkpoint slice exceeds shared memory
    }
    return status_of(cudaGetLastError());
}

}  // extern "C"
