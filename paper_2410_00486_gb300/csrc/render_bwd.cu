// Backward of the blend (Eqs. 2-4, Sec. III-C.1, CaRtGS), pixel-parallel.
//
// One block per (view, tile), two vertically adjacent pixels per thread, walking the
// tile's list back to front from the block's largest `last`.  Staging applies the
// forward's tile test and exponent threshold, so the same splats are considered.  Each pixel recomputes alpha exactly as
// the forward did (same rounding, same decisions) and its transmittance from the
// stored final T, T_j = T_{j+1} / (1 - alpha_j), so no per-pixel splat list is kept.
// The accumulated colour behind splat j follows acc_j = a_{j+1} c_{j+1} +
// (1 - a_{j+1}) acc_{j+1}, and
//   dL/dalpha_j = T_j sum_c gI_c (c_j - acc_j) + T_j gD (z_j - accD_j)
//                 - T_final (bg . gI) / (1 - alpha_j).
// The per-(splat, pixel) gradients of a thread's two pixels are added in registers,
// then the 64 pixels of a warp are summed with a butterfly reduce-scatter (15 shuffles
// for 10 fields instead of 50 for a plain tree per field), after which ten lanes each
// issue one atomic add into the slot's gradient record.  Warps where no pixel blended
// the splat skip it (vote).
#include "raster.cuh"

namespace cgs {

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
__global__ void __launch_bounds__(B *B / ppt_for<B, kPPTBwd>()) k_render_bwd(RasterBwdArgs a)
{
    constexpr int PPT = ppt_for<B, kPPTBwd>();
    constexpr int NT = B * B / PPT;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[BD], s1[BD], s2[BD];
    __shared__ uint32_t sslot[BD], spos[BD];
    __shared__ uint32_t smax[NW];
    __shared__ int wcnt[NW];
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

    // per-pixel state
    float fy[PPT], T[PPT], gI0[PPT], gI1[PPT], gI2[PPT], gD[PPT], bgdot[PPT];
    float acc0[PPT], acc1[PPT], acc2[PPT], accD[PPT];
    uint32_t lst[PPT];
    uint32_t m = 0;
#pragma unroll
    for (int p = 0; p < PPT; p++) {
        const int py = py0 + p;
        fy[p] = (float)py;
        lst[p] = 0;
        T[p] = 1.f;
        gI0[p] = gI1[p] = gI2[p] = gD[p] = bgdot[p] = 0.f;
        acc0[p] = acc1[p] = acc2[p] = accD[p] = 0.f;
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
        bgdot[p] = T[p] * (a.bg0 * gI0[p] + a.bg1 * gI1[p] + a.bg2 * gI2[p]);
        m = max(m, lst[p]);
    }
    // block-wide largest `last`: the walk starts there
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(kFull, m, off));
    if (lane == 0) smax[threadIdx.x / 32] = m;
    __syncthreads();
    uint32_t maxlast = 0;
    for (int i = 0; i < NW; i++) maxlast = max(maxlast, smax[i]);

    const float bx0 = (float)(tx * B), bx1 = (float)(min(tx * B + B, a.g.W) - 1);
    const float by0 = (float)(ty * B), by1 = (float)(min(ty * B + B, a.g.H) - 1);
    for (int bend = (int)maxlast; bend > 0; bend -= BD) {
        const int bstart = max(0, bend - BD);
        const int nraw = bend - bstart;
        __syncthreads();
        // stage positions [bstart, bend), keeping in list order only splats that can
        // touch the tile (the forward applied the same test)
        int cnt = 0;
        for (int c0 = 0; c0 < BD; c0 += NT) {
            const int i = c0 + (int)threadIdx.x;
            bool keep = false;
            float4 r0, r1;
            const float4 *r = nullptr;
            uint32_t slot = 0;
            if (i < nraw) {
                slot = __ldg(a.vals + start + bstart + i);
                r = a.rec + kRec4 * (size_t)slot;
                r0 = __ldg(r);
                r1 = __ldg(r + 1);
                keep = splat_touches_box(r0, r1, bx0, bx1, by0, by1);
            }
            int tot;
            const int pre = block_compact<NW>(keep, wcnt, tot);
            if (keep) {
                const int d = cnt + pre;
                stage_splat(r0, r1, s0[d], s1[d]);
                s2[d] = __ldg(r + 2);
                sslot[d] = slot;
                spos[d] = (uint32_t)(bstart + i);
            }
            cnt += tot;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; j--) {
            const uint32_t pos = spos[j];
            const float4 q0 = s0[j];
            const float4 q1 = s1[j];
            const float dx = __fsub_rn(q0.x, fx);
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; k++) v[k] = 0.f;
            bool contrib = false;
#pragma unroll
            for (int p = 0; p < PPT; p++) {
                if (!(pos < lst[p])) continue;
                const float dy = __fsub_rn(q0.y, fy[p]);
                const float power = staged_power(q0, q1.x, dx, dy);
                if (power > 0.f || power < q1.w) continue;
                const float G = __expf(power);
                const float araw = __fmul_rn(q1.y, G);
                const float alpha = fminf(kAlphaMax, araw);
                contrib = true;
                const float4 q2 = s2[j];
                const float inv_om = __fdividef(1.f, __fsub_rn(1.f, alpha));
                T[p] = T[p] * inv_om;                             // transmittance before splat j
                const float wT = alpha * T[p];
                v[8] += wT * gI0[p];
                v[9] += wT * gI1[p];
                v[10] += wT * gI2[p];
                v[6] += wT * gD[p];
                // acc = colour (and depth) accumulated behind splat j, as seen just after it
                float dLda = (q2.x - acc0[p]) * gI0[p] + (q2.y - acc1[p]) * gI1[p] + (q2.z - acc2[p]) * gI2[p] +
                             (q1.z - accD[p]) * gD[p];
                dLda = dLda * T[p] - bgdot[p] * inv_om;
                // fold splat j in for the splats in front of it: acc <- a c + (1 - a) acc
                acc0[p] = fmaf(alpha, q2.x - acc0[p], acc0[p]);
                acc1[p] = fmaf(alpha, q2.y - acc1[p], acc1[p]);
                acc2[p] = fmaf(alpha, q2.z - acc2[p], acc2[p]);
                accD[p] = fmaf(alpha, q1.z - accD[p], accD[p]);
                if (!(araw > kAlphaMax)) {
                    // dalpha/dpower = alpha, dalpha/dopacity = G.  Raw moments of
                    // dp = dL/dpower are summed here; the conic / centre gradients are
                    // formed from them once per warp after the reduction.
                    const float dp = dLda * alpha;
                    v[5] += dLda * G;
                    const float dpx = dp * dx, dpy = dp * dy;
                    v[0] += dpx;             // sum dp dx
                    v[1] += dpy;             // sum dp dy
                    v[2] += dpx * dx;        // sum dp dx^2
                    v[3] += dpx * dy;        // sum dp dx dy
                    v[4] += dpy * dy;        // sum dp dy^2
                }
            }
            const unsigned who = __ballot_sync(kFull, contrib);
            if (who == 0u) continue;
            if ((who & (who - 1u)) == 0u) {
                // a single contributing lane adds its sums directly
                if (contrib) {
                    float *g = a.sgrad + (size_t)sslot[j] * 12;
                    const float hA = s0[j].z, nB = s0[j].w, hC = s1[j].x;
                    atomicAdd(g + 0, 2.f * hA * v[0] + nB * v[1]);
                    atomicAdd(g + 1, 2.f * hC * v[1] + nB * v[0]);
                    atomicAdd(g + 2, -0.5f * v[2]);
                    atomicAdd(g + 3, -v[3]);
                    atomicAdd(g + 4, -0.5f * v[4]);
                    atomicAdd(g + 5, v[5]);
                    atomicAdd(g + 6, v[6]);
                    atomicAdd(g + 8, v[8]);
                    atomicAdd(g + 9, v[9]);
                    atomicAdd(g + 10, v[10]);
                }
                continue;
            }
            {
                float sum = warp_reduce_scatter16(v, lane);
                const int f = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                // fields 0 and 1 sit in lanes that differ in bit 1: exchange the two first moments
                const float other = __shfl_xor_sync(kFull, sum, 2);
                // power = -(A dx^2 + C dy^2)/2 - B dx dy with dx = u - x:
                //   dL/du = -(A S_dx + B S_dy), dL/dv = -(C S_dy + B S_dx),
                //   dL/dA = -S_xx / 2, dL/dB = -S_xy, dL/dC = -S_yy / 2
                // (staged q0.z = -A/2, q0.w = -B, q1.x = -C/2)
                const float4 q0 = s0[j];
                const float hC = s1[j].x;
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
