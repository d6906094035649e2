// Backward of the blend (Eqs. 2-4, Sec. III-C.1, CaRtGS), pixel-parallel.
//
// One block per (view, tile), eight pixels of one column per thread (one warp per 16x16
// tile; two pixels on 8x8 tiles), walking the tile's list back to front from the block's
// largest `last`.
// A tile's list holds only splats that can reach alpha >= 1/255 in it (the binning's
// test), the same list the forward walked.  Each pixel recomputes alpha exactly as the
// forward did (same rounding, same decisions) and its transmittance from the stored final T,
// T_j = T_{j+1} / (1 - alpha_j), so no per-pixel splat list is kept.  A thread blends its
// pixels in pairs: when either pixel of a pair blends splat j, both run through the blend
// (the other with alpha = 0, which leaves its state as it is), so the two dependency chains
// interleave.
//
// With R_j the colour behind splat j normalised by the transmittance just after it,
// R_last = bg and R_{j-1} = a_j c_j + (1 - a_j) R_j (depth alike, starting at 0),
//   dL/dalpha_j = T_j [ gI . (c_j - R_j) + gD (z_j - Rz_j) ],
// so a pixel only carries the scalar S_j = gI . R_j + gD Rz_j, updated by the same
// recursion with c_j . gI + z_j gD in place of the colour.
//
// The per-(splat, pixel) gradients of a thread's pixels are added in registers (the
// pixels share dx, so the dx moments are formed once per thread), then a warp's rows of
// ten sums are added through shared memory (each lane stores its row, thirty lanes add
// one field over a third of the rows each, two shuffles join the thirds), after which
// ten lanes each issue one atomic add into the slot's gradient record; when only a few
// lanes contributed they add their own sums directly instead.  Warps where no pixel
// blended the splat skip it (vote).
//
// The per-pixel loss gradients (three channels and depth) are constant during the walk and
// live in shared memory, read once per blended pixel; that leaves 72 registers a thread,
// so 28 warps stay resident.  With a work counter the grid is persistent: as many blocks
// as are resident on the GPU take (view, tile) items in the sort's longest-first order
// from the counter until none is left.
#include "raster.cuh"

namespace cgs {

// Splats to which at most this many lanes of a warp contribute are added with per-lane
// atomics (L2 reductions); more contributors go through the warp sum.  Measured on the
// 16-view window with the persistent 28-warp kernel (raster backward ms): 4 lanes 3.366,
// 8 lanes 3.347, 10 lanes 3.340, 12 lanes 3.344, 16 lanes 3.419, 20 lanes 3.580, 24 lanes
// 3.877; folding a half-warp onto the other and adding from 16 lanes was twice as slow
// (same-address atomics serialise).
constexpr int kDirectLanes = 10;

// Row stride (floats) of the per-warp reduction buffer: ten fields padded to 12.
constexpr int kRedStride = 12;
constexpr int kRedRows = 33;   // 32 lanes and a zero row

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

template <int B, int BD>
__global__ void __launch_bounds__(B *B / ppt_for<B, kPPTBwd>(), (min_blocks_for<B, kPPTBwd, kBwdMinWarps>())) k_render_bwd(RasterBwdArgs a)
{
    constexpr int PPT = ppt_for<B, kPPTBwd>();
    constexpr int NT = B * B / PPT;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[BD], s1[BD], s2[BD];
    __shared__ uint32_t sslot[BD];
    __shared__ uint32_t smax[NW];
    __shared__ __align__(16) float red[NW * kRedRows * kRedStride];   // per warp
    __shared__ float4 sgi[PPT * NT];   // per pixel p of thread t at [p NT + t]: dL/dimg (3 channels), dL/ddepth
    __shared__ uint32_t s_item;
    for (int i = threadIdx.x; i < NW * kRedStride; i += NT)   // the zero row of every warp's buffer
        red[(i / kRedStride) * (kRedRows * kRedStride) + 32 * kRedStride + i % kRedStride] = 0.f;
    const uint32_t n_items = (uint32_t)(a.g.Tv * a.V);
    for (uint32_t it = 0;; it++) {
    uint32_t item = blockIdx.x;
    if (a.work) {
        __syncthreads();   // the previous item's reads of s_item and of the shared state are done
        if (threadIdx.x == 0) s_item = atomicAdd(a.work, 1u);
        __syncthreads();
        item = s_item;
        if (item >= n_items) break;
    } else if (it > 0) {
        break;
    }
    int64_t tile;
    int view, tx, ty;
    item_tile(a.order, a.g, tile, view, tx, ty, item);
    const int lane = threadIdx.x & 31;
    const int px = tx * B + (int)(threadIdx.x % B);
    constexpr int G = row_step<B>();
    const int py0 = ty * B + thread_row0<B, PPT>();   // row of pixel p: py0 + G p
    const float fx = (float)px;
    const uint32_t start = a.ranges[2 * tile];
    const uint32_t len = a.ranges[2 * tile + 1] - start;
    const size_t HW = (size_t)a.g.W * a.g.H;

    // per-pixel state: transmittance, pixel gradients, and S = (colour behind) . gI +
    // (depth behind) gD, where "behind" starts as the background (no depth) and follows
    // R <- alpha c + (1 - alpha) R towards the front
    float T[PPT], S[PPT];
    const float fy0 = (float)py0;   // row of pixel p: fy0 + G p (exact)
    uint32_t lst[PPT];
    uint32_t m = 0;
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        const int py = py0 + G * p;
        lst[p] = 0;
        T[p] = 1.f;
        S[p] = 0.f;
        float gI0 = 0.f, gI1 = 0.f, gI2 = 0.f, gD = 0.f;
        if (!(px < a.g.W && py < a.g.H)) {
            sgi[p * NT + threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const size_t q = (size_t)py * a.g.W + px;
        const size_t pix = (size_t)view * HW + q;
        // never walk past the tile's list, whatever `last` holds
        lst[p] = min(a.last[pix], len);
        T[p] = a.tfin[pix];
        if (a.dl_dimg) {
            const float *gi = a.dl_dimg + (size_t)view * 3 * HW + q;
            gI0 = gi[0];
            gI1 = gi[HW];
            gI2 = gi[2 * HW];
            gD = a.dl_ddepth ? a.dl_ddepth[pix] : 0.f;
        } else {
            const float w = a.weight ? a.weight[view] : 1.f;
            const float sc = w / (3.f * (float)HW);
            const float *im = a.img + (size_t)view * 3 * HW + q;
            const float *tr = a.tgt_rgb + (size_t)view * 3 * HW + q;
            gI0 = sc * sgnf(im[0] - tr[0]);
            gI1 = sc * sgnf(im[HW] - tr[HW]);
            gI2 = sc * sgnf(im[2 * HW] - tr[2 * HW]);
            if (a.tgt_depth) {
                const float td = a.tgt_depth[pix];
                const int cnt = a.depth_count[view];
                if (td > 0.f && cnt > 0) gD = w * a.lambda_d * sgnf(a.depth[pix] - td) / (float)cnt;
            }
        }
        sgi[p * NT + threadIdx.x] = make_float4(gI0, gI1, gI2, gD);
        S[p] = a.bg0 * gI0 + a.bg1 * gI1 + a.bg2 * gI2;
        m = max(m, lst[p]);
    }
    // block-wide largest `last`: the walk starts there
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(kFull, m, off));
    if (lane == 0) smax[threadIdx.x / 32] = m;
    __syncthreads();
    uint32_t maxlast = 0;
    for (int i = 0; i < NW; i++) maxlast = max(maxlast, smax[i]);

    for (int bend = (int)maxlast; bend > 0; bend -= BD) {
        const int bstart = max(0, bend - BD);
        const int nraw = bend - bstart;
        __syncthreads();
        // stage positions [bstart, bend) (every entry can reach the tile: the binning's test)
        for (int c0 = 0; c0 < BD; c0 += NT) {
            const int i = c0 + (int)threadIdx.x;
            if (i >= nraw) break;
            const uint32_t slot = __ldg(a.vals + start + bstart + i);
            const float4 *r = a.rec + kRec4 * (size_t)slot;
            const float4 r2 = __ldg(r + 2);
            stage_splat(__ldg(r), __ldg(r + 1), r2.w, s0[i], s1[i]);
            s2[i] = r2;
            sslot[i] = slot;
        }
        __syncthreads();
        // two splats per loop trip, so one splat's loads and tests overlap the other's blend and
        // sums (3.470 -> 3.426 ms on the 16-view window; four per trip spill: 3.87 ms)
#pragma unroll 2
        for (int j = nraw - 1; j >= 0; j--) {
            const uint32_t pos = (uint32_t)(bstart + j);   // list position of splat j
            const float4 q0 = s0[j];
            const float4 q1 = s1[j];
            const float4 q2 = s2[j];
            const float dx = __fsub_rn(q0.x, fx);
            const PowerX pxs = power_x(q0, dx);
            // per-thread sums over its pixels: colour / depth / opacity gradients, and the
            // moments sum dp, sum dp dy, sum dp dy^2 of dp = dL/dpower (dx is shared)
            float gr = 0.f, gg = 0.f, gb = 0.f, gz = 0.f, go = 0.f, sdp = 0.f, sdpy = 0.f, sdpyy = 0.f;
            bool contrib = false;
            // pixels in pairs: a pair where either pixel blends runs both through the blend
            // (the other with G = 0, so alpha = 0 and its state is kept), so the two chains
            // interleave
#pragma unroll
            for (int p2 = 0; p2 < PPT; p2 += 2) {
                float dyv[2], pw[2];
                bool k[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int p = p2 + h;
                    dyv[h] = __fsub_rn(q0.y, fy0 + (float)(G * p));
                    pw[h] = power_at(pxs, q1.x, dyv[h]);
                    k[h] = pos < lst[p] && fabsf(pw[h]) <= q1.w;
                }
                // a warp-uniform branch (vote) rather than a divergent one: a lane whose pair
                // blends nothing runs the pair with alpha = 0, which changes nothing (3.337 ->
                // 3.297 ms on the 16-view window)
                const bool pair = k[0] || k[1];
                contrib = contrib || pair;
                if (!__any_sync(kFull, pair)) continue;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int p = p2 + h;
                    const float dy = dyv[h];
                    const float4 gi = sgi[p * NT + threadIdx.x];   // dL/dimg, dL/ddepth of pixel p
                    const float G = k[h] ? exp2_fast(pw[h]) : 0.f;
                    const float araw = __fmul_rn(q1.y, G);
                    const float alpha = fminf(kAlphaMax, araw);
                    const float inv_om = rcp_fast(__fsub_rn(1.f, alpha));
                    T[p] = k[h] ? T[p] * inv_om : T[p];               // transmittance before splat j
                    const float wT = alpha * T[p];
                    gr = fmaf(wT, gi.x, gr);
                    gg = fmaf(wT, gi.y, gg);
                    gb = fmaf(wT, gi.z, gb);
                    gz = fmaf(wT, gi.w, gz);
                    const float cg = fmaf(q1.z, gi.w, fmaf(q2.z, gi.z, fmaf(q2.y, gi.y, q2.x * gi.x)));
                    const float diff = cg - S[p];
                    S[p] = fmaf(alpha, diff, S[p]);
                    // dalpha/dpower = alpha, dalpha/dopacity = G, both 0 where alpha is clamped
                    const float dLda = araw > kAlphaMax ? 0.f : diff * T[p];
                    go = fmaf(dLda, G, go);
                    const float dp = dLda * alpha;
                    const float dpy = dp * dy;
                    sdp += dp;
                    sdpy += dpy;
                    sdpyy = fmaf(dpy, dy, sdpyy);
                }
            }
            const unsigned who = __ballot_sync(kFull, contrib);
            if (who == 0u) continue;
            // raw moments of dp over this thread's pixels: sum dp dx, dp dy, dp dx^2, dp dx dy, dp dy^2
            const float m0 = sdp * dx, m3 = sdpy * dx;
            if (__popc(who) <= kDirectLanes) {
                // few contributing lanes: each adds its sums directly
                if (contrib) {
                    float *g = a.sgrad + (size_t)sslot[j] * 12;
                    const float hA = q0.z, nB = q0.w, hC = q1.x;
                    atomicAdd(g + 0, kLn2 * (2.f * hA * m0 + nB * sdpy));   // staged terms carry log2 e
                    atomicAdd(g + 1, kLn2 * (2.f * hC * sdpy + nB * m0));
                    atomicAdd(g + 2, -0.5f * (m0 * dx));
                    atomicAdd(g + 3, -m3);
                    atomicAdd(g + 4, -0.5f * sdpyy);
                    atomicAdd(g + 5, go);
                    atomicAdd(g + 6, gz);
                    atomicAdd(g + 8, gr);
                    atomicAdd(g + 9, gg);
                    atomicAdd(g + 10, gb);
                }
                continue;
            }
            {
                // warp sum of the ten fields through shared memory: every lane stores its
                // row, then lanes 10g + f (g < 3, f < 10) add field f over rows g, g + 3,
                // g + 6, ... and three shuffles combine the groups (row stride 12 floats:
                // the 16-byte stores are conflict-free, the column reads nearly so)
                float *buf = red + (size_t)(threadIdx.x >> 5) * (kRedRows * kRedStride);
                __syncwarp();   // the previous sum's column reads are done before the rows are rewritten
                float4 *row = reinterpret_cast<float4 *>(buf + lane * kRedStride);
                row[0] = make_float4(m0, sdpy, m0 * dx, m3);
                row[1] = make_float4(sdpyy, go, gz, gr);
                row[2] = make_float4(gg, gb, 0.f, 0.f);
                __syncwarp();
                const int g = lane / 10, f = lane - 10 * g;
                float sum = 0.f;
                if (lane < 30) {
                    // rows g, g + 3, ..., g + 30; row 32 (group 2's last) is a zero row
                    const float *col = buf + g * kRedStride + f;
#pragma unroll
                    for (int k = 0; k < 11; k++) sum += col[3 * k * kRedStride];
                }
                {
                    const float p1 = __shfl_down_sync(kFull, sum, 10), p2 = __shfl_down_sync(kFull, sum, 20);
                    sum += p1 + p2;   // lanes 0..9: field sums (groups 0, 1, 2)
                }
                // fields 0 and 1 (first moments) sit in lanes 0 and 1: exchange them
                const float other = __shfl_xor_sync(kFull, sum, 1);
                // power = -(A dx^2 + C dy^2)/2 - B dx dy with dx = u - x:
                //   dL/du = -(A S_dx + B S_dy), dL/dv = -(C S_dy + B S_dx),
                //   dL/dA = -S_xx / 2, dL/dB = -S_xy, dL/dC = -S_yy / 2
                // (staged q0.z = -A/2, q0.w = -B, q1.x = -C/2)
                const float hC = q1.x;
                if (f == 0) sum = kLn2 * (2.f * q0.z * sum + q0.w * other);   // staged terms carry log2 e
                else if (f == 1) sum = kLn2 * (2.f * hC * sum + q0.w * other);
                else if (f == 2 || f == 4) sum = -0.5f * sum;
                else if (f == 3) sum = -sum;
                // record fields 0..6 (u, v, A, B, C, o, z), 8..10 (r, g, b)
                if (lane < 10) atomicAdd(a.sgrad + (size_t)sslot[j] * 12 + (f < 7 ? f : f + 1), sum);
            }
        }
    }
    }   // work items
}

template <int B, int BD>
static cudaError_t launch_bwd(const RasterBwdArgs &a, cudaStream_t s)
{
    const int nt = B * B / ppt_for<B, kPPTBwd>();
    int64_t blocks = a.g.Tv * a.V;
    if (a.work) {
        // persistent: the resident blocks of the whole GPU (queried once per device and shape)
        static int resident[64] = {0};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!resident[dev]) {
            int per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_bwd<B, BD>, nt, 0);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            resident[dev] = max(1, per_sm) * max(1, sms);
        }
        blocks = min(blocks, (int64_t)resident[dev]);
        e = cudaMemsetAsync(a.work, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
    }
    if (blocks > 0) k_render_bwd<B, BD><<<(unsigned)blocks, nt, 0, s>>>(a);
    return cudaGetLastError();
}

template <int B>
static cudaError_t launch_bwd_bd(const RasterBwdArgs &a, int BD, cudaStream_t s)
{
    switch (BD) {
    case 32: return launch_bwd<B, 32>(a, s);
    case 64: return launch_bwd<B, 64>(a, s);
    case 128: return launch_bwd<B, 128>(a, s);
    default: return launch_bwd<B, 256>(a, s);
    }
}

cudaError_t raster_bwd(const RasterBwdArgs &a, int B, int BD, cudaStream_t s)
{
    switch (B) {
    case 8: return launch_bwd_bd<8>(a, BD, s);
    case 16: return launch_bwd_bd<16>(a, BD, s);
    default: return launch_bwd_bd<32>(a, BD, s);
    }
}

}  // namespace cgs
