// Backward of the blend (Eqs. 2-4, Sec. III-C.1, CaRtGS), pixel-parallel.
//
// One block per (view, tile), four vertically adjacent pixels per thread (two on 8x8
// tiles), walking the tile's list back to front from the block's largest `last`.
// A tile's list holds only splats that can reach alpha >= 1/255 in it (the binning's
// test), the same list the forward walked.  Each pixel recomputes alpha exactly as the forward did (same
// rounding, same decisions) and its transmittance from the stored final T,
// T_j = T_{j+1} / (1 - alpha_j), so no per-pixel splat list is kept.
//
// With R_j the colour behind splat j normalised by the transmittance just after it,
// R_last = bg and R_{j-1} = a_j c_j + (1 - a_j) R_j (depth alike, starting at 0),
//   dL/dalpha_j = T_j [ gI . (c_j - R_j) + gD (z_j - Rz_j) ],
// so a pixel only carries the scalar S_j = gI . R_j + gD Rz_j, updated by the same
// recursion with c_j . gI + z_j gD in place of the colour.
//
// The per-(splat, pixel) gradients of a thread's pixels are added in registers (the
// pixels share dx, so the dx moments are formed once per thread), then a warp's pixels
// are summed with a butterfly reduce-scatter (15 shuffles for 10 fields instead of 50
// for a plain tree per field), after which ten lanes each issue one atomic add into
// the slot's gradient record; when only a few lanes contributed they add their own sums
// directly instead.  Warps where no pixel blended the splat skip it (vote).
#include "raster.cuh"

namespace cgs {

// Splats to which at most this many lanes of a warp contribute are added with per-lane
// atomics (L2 reductions); more contributors go through the warp reduce-scatter.  Measured
// on the 16-view window: 1 lane 5.81 ms, 8 lanes 5.62, 12-16 lanes 5.55, 24 lanes 5.97,
// and every lane direct 25.9 (same-address atomics serialise).
constexpr int kDirectLanes = 12;

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// Reduce-scatter of 16 per-lane values over the warp.  On return lane l holds the
// warp sum of value index ((l>>4)&1)*8 + ((l>>3)&1)*4 + ((l>>2)&1)*2 + ((l>>1)&1).
// Value 7 and values 11..15 are always zero here; the pair (7, 15) needs no shuffle.
__device__ __forceinline__ float warp_reduce_scatter16(float v[16], int lane)
{
    const bool b4 = lane & 16;
#pragma unroll
    for (int i = 0; i < 7; i++) {
        const float mine = b4 ? v[i + 8] : v[i];
        const float other = b4 ? v[i] : v[i + 8];
        v[i] = mine + __shfl_xor_sync(kFull, other, 16);
    }
    v[7] = 0.f;
    const bool b3 = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float mine = b3 ? v[i + 4] : v[i];
        const float other = b3 ? v[i] : v[i + 4];
        v[i] = mine + __shfl_xor_sync(kFull, other, 8);
    }
    const bool b2 = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float mine = b2 ? v[i + 2] : v[i];
        const float other = b2 ? v[i] : v[i + 2];
        v[i] = mine + __shfl_xor_sync(kFull, other, 4);
    }
    const bool b1 = lane & 2;
    {
        const float mine = b1 ? v[1] : v[0];
        const float other = b1 ? v[0] : v[1];
        v[0] = mine + __shfl_xor_sync(kFull, other, 2);
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

template <int B, int BD>
__global__ void __launch_bounds__(B *B / ppt_for<B, kPPTBwd>(), (min_blocks_for<B, kPPTBwd, kBwdMinWarps>())) k_render_bwd(RasterBwdArgs a)
{
    constexpr int PPT = ppt_for<B, kPPTBwd>();
    constexpr int NT = B * B / PPT;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[BD], s1[BD], s2[BD];
    __shared__ uint32_t sslot[BD], spos[BD];
    __shared__ uint32_t smax[NW];
    int64_t tile;
    int view, tx, ty;
    item_tile(a.order, a.g, tile, view, tx, ty);
    const int lane = threadIdx.x & 31;
    const int px = tx * B + (int)(threadIdx.x % B);
    const int py0 = ty * B + (int)(threadIdx.x / B) * PPT;
    const float fx = (float)px;
    const uint32_t start = a.ranges[2 * tile];
    const uint32_t len = a.ranges[2 * tile + 1] - start;
    const size_t HW = (size_t)a.g.W * a.g.H;

    // per-pixel state: transmittance, pixel gradients, and S = (colour behind) . gI +
    // (depth behind) gD, where "behind" starts as the background (no depth) and follows
    // R <- alpha c + (1 - alpha) R towards the front
    float T[PPT], gI0[PPT], gI1[PPT], gI2[PPT], gD[PPT], S[PPT];
    const float fy0 = (float)py0;   // row of pixel p: fy0 + p (exact)
    uint32_t lst[PPT];
    uint32_t m = 0;
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        const int py = py0 + p;
        lst[p] = 0;
        T[p] = 1.f;
        gI0[p] = gI1[p] = gI2[p] = gD[p] = S[p] = 0.f;
        if (!(px < a.g.W && py < a.g.H)) continue;
        const size_t q = (size_t)py * a.g.W + px;
        const size_t pix = (size_t)view * HW + q;
        // never walk past the tile's list, whatever `last` holds
        lst[p] = min(a.last[pix], len);
        T[p] = a.tfin[pix];
        if (a.dl_dimg) {
            const float *gi = a.dl_dimg + (size_t)view * 3 * HW + q;
            gI0[p] = gi[0];
            gI1[p] = gi[HW];
            gI2[p] = gi[2 * HW];
            gD[p] = a.dl_ddepth ? a.dl_ddepth[pix] : 0.f;
        } else {
            const float w = a.weight ? a.weight[view] : 1.f;
            const float sc = w / (3.f * (float)HW);
            const float *im = a.img + (size_t)view * 3 * HW + q;
            const float *tr = a.tgt_rgb + (size_t)view * 3 * HW + q;
            gI0[p] = sc * sgnf(im[0] - tr[0]);
            gI1[p] = sc * sgnf(im[HW] - tr[HW]);
            gI2[p] = sc * sgnf(im[2 * HW] - tr[2 * HW]);
            if (a.tgt_depth) {
                const float td = a.tgt_depth[pix];
                const int cnt = a.depth_count[view];
                if (td > 0.f && cnt > 0) gD[p] = w * a.lambda_d * sgnf(a.depth[pix] - td) / (float)cnt;
            }
        }
        S[p] = a.bg0 * gI0[p] + a.bg1 * gI1[p] + a.bg2 * gI2[p];
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
            spos[i] = (uint32_t)(bstart + i);
        }
        __syncthreads();
        for (int j = nraw - 1; j >= 0; j--) {
            const uint32_t pos = spos[j];
            const float4 q0 = s0[j];
            const float4 q1 = s1[j];
            const float dx = __fsub_rn(q0.x, fx);
            const PowerX pxs = power_x(q0, dx);
            // per-thread sums over its pixels: colour / depth / opacity gradients, and the
            // moments sum dp, sum dp dy, sum dp dy^2 of dp = dL/dpower (dx is shared)
            float gr = 0.f, gg = 0.f, gb = 0.f, gz = 0.f, go = 0.f, sdp = 0.f, sdpy = 0.f, sdpyy = 0.f;
            bool contrib = false;
#pragma unroll
            for (int p = 0; p < PPT; p++) {
                if (!(pos < lst[p])) continue;
                const float dy = __fsub_rn(q0.y, fy0 + (float)p);
                const float power = power_at(pxs, q1.x, dy);
                if (power > 0.f || power < q1.w) continue;
                const float G = __expf(power);
                const float araw = __fmul_rn(q1.y, G);
                const float alpha = fminf(kAlphaMax, araw);
                contrib = true;
                const float4 q2 = s2[j];
                const float inv_om = __fdividef(1.f, __fsub_rn(1.f, alpha));
                T[p] = T[p] * inv_om;                             // transmittance before splat j
                const float wT = alpha * T[p];
                gr = fmaf(wT, gI0[p], gr);
                gg = fmaf(wT, gI1[p], gg);
                gb = fmaf(wT, gI2[p], gb);
                gz = fmaf(wT, gD[p], gz);
                // dL/dalpha = T (c . gI + z gD - S); then fold splat j into S for the
                // splats in front of it
                const float cg = fmaf(q1.z, gD[p], fmaf(q2.z, gI2[p], fmaf(q2.y, gI1[p], q2.x * gI0[p])));
                const float diff = cg - S[p];
                S[p] = fmaf(alpha, diff, S[p]);
                if (!(araw > kAlphaMax)) {
                    // dalpha/dpower = alpha, dalpha/dopacity = G
                    const float dLda = diff * T[p];
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
                    atomicAdd(g + 0, 2.f * hA * m0 + nB * sdpy);
                    atomicAdd(g + 1, 2.f * hC * sdpy + nB * m0);
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
                float v[16];
                v[0] = m0;
                v[1] = sdpy;
                v[2] = m0 * dx;
                v[3] = m3;
                v[4] = sdpyy;
                v[5] = go;
                v[6] = gz;
                v[7] = 0.f;
                v[8] = gr;
                v[9] = gg;
                v[10] = gb;
#pragma unroll
                for (int k = 11; k < 16; k++) v[k] = 0.f;
                float sum = warp_reduce_scatter16(v, lane);
                const int f = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                // fields 0 and 1 sit in lanes that differ in bit 1: exchange the two first moments
                const float other = __shfl_xor_sync(kFull, sum, 2);
                // power = -(A dx^2 + C dy^2)/2 - B dx dy with dx = u - x:
                //   dL/du = -(A S_dx + B S_dy), dL/dv = -(C S_dy + B S_dx),
                //   dL/dA = -S_xx / 2, dL/dB = -S_xy, dL/dC = -S_yy / 2
                // (staged q0.z = -A/2, q0.w = -B, q1.x = -C/2)
                const float hC = q1.x;
                if (f == 0) sum = 2.f * q0.z * sum + q0.w * other;
                else if (f == 1) sum = 2.f * hC * sum + q0.w * other;
                else if (f == 2 || f == 4) sum = -0.5f * sum;
                else if (f == 3) sum = -sum;
                if (!(lane & 1) && f != 7 && f < 11) atomicAdd(a.sgrad + (size_t)sslot[j] * 12 + f, sum);
            }
        }
    }
}

template <int B, int BD>
static cudaError_t launch_bwd(const RasterBwdArgs &a, cudaStream_t s)
{
    const int64_t items = a.g.Tv * a.V;
    k_render_bwd<B, BD><<<(unsigned)items, B * B / ppt_for<B, kPPTBwd>(), 0, s>>>(a);
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
