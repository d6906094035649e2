// Backward of the blend (Eqs. 2-4, Sec. III-C.1, CaRtGS), pixel-parallel.
//
// One block per (view, tile), one thread per pixel, walking the tile's list back
// to front from the block's largest `last`.  Each pixel recomputes alpha exactly as
// the forward did (same rounding, same decisions) and its transmittance from the
// stored final T, T_j = T_{j+1} / (1 - alpha_j), so no per-pixel splat list is kept.
// The accumulated colour behind splat j follows acc_j = a_{j+1} c_{j+1} +
// (1 - a_{j+1}) acc_{j+1}, and
//   dL/dalpha_j = T_j sum_c gI_c (c_j - acc_j) + T_j gD (z_j - accD_j)
//                 - T_final (bg . gI) / (1 - alpha_j).
// The per-(splat, pixel) gradients of the 32 pixels of a warp are summed with a
// butterfly reduce-scatter (15 shuffles for 10 fields instead of 50 for a plain
// tree per field), after which ten lanes each issue one atomic add into the
// slot's gradient record.  Warps where no pixel blended the splat skip it (vote).
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
__global__ void __launch_bounds__(B *B) k_render_bwd(RasterBwdArgs a)
{
    constexpr int NT = B * B;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[BD], s1[BD], s2[BD];
    __shared__ uint32_t sslot[BD];
    __shared__ uint32_t smax[NW];
    int64_t tile;
    int view, tx, ty;
    item_tile(a.order, a.g, tile, view, tx, ty);
    const int lane = threadIdx.x & 31;
    const int px = tx * B + (int)(threadIdx.x % B), py = ty * B + (int)(threadIdx.x / B);
    const bool inside = px < a.g.W && py < a.g.H;
    const float fx = (float)px, fy = (float)py;

    uint32_t lst = 0;
    float T = 1.f, gI0 = 0.f, gI1 = 0.f, gI2 = 0.f, gD = 0.f, bgdot = 0.f;
    if (inside) {
        const size_t HW = (size_t)a.g.W * a.g.H;
        const size_t p = (size_t)py * a.g.W + px;
        const size_t pix = (size_t)view * HW + p;
        lst = a.last[pix];
        T = a.tfin[pix];
        if (a.dl_dimg) {
            const float *gi = a.dl_dimg + (size_t)view * 3 * HW + p;
            gI0 = gi[0];
            gI1 = gi[HW];
            gI2 = gi[2 * HW];
            gD = a.dl_ddepth ? a.dl_ddepth[pix] : 0.f;
        } else {
            const float w = a.weight ? a.weight[view] : 1.f;
            const float s = w / (3.f * (float)HW);
            const float *im = a.img + (size_t)view * 3 * HW + p;
            const float *tr = a.tgt_rgb + (size_t)view * 3 * HW + p;
            gI0 = s * sgnf(im[0] - tr[0]);
            gI1 = s * sgnf(im[HW] - tr[HW]);
            gI2 = s * sgnf(im[2 * HW] - tr[2 * HW]);
            if (a.tgt_depth) {
                const float td = a.tgt_depth[pix];
                const int cnt = a.depth_count[view];
                if (td > 0.f && cnt > 0) gD = w * a.lambda_d * sgnf(a.depth[pix] - td) / (float)cnt;
            }
        }
        bgdot = T * (a.bg0 * gI0 + a.bg1 * gI1 + a.bg2 * gI2);
    }
    // never walk past the tile's list, whatever `last` holds
    const uint32_t start = a.ranges[2 * tile];
    const uint32_t len = a.ranges[2 * tile + 1] - start;
    lst = min(lst, len);
    // block-wide largest `last`: the walk starts there
    uint32_t m = lst;
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(kFull, m, off));
    if (lane == 0) smax[threadIdx.x / 32] = m;
    __syncthreads();
    uint32_t maxlast = 0;
    for (int i = 0; i < NW; i++) maxlast = max(maxlast, smax[i]);

    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, accD = 0.f;
    float la = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f, lz = 0.f;
    for (int bend = (int)maxlast; bend > 0; bend -= BD) {
        const int bstart = max(0, bend - BD);
        const int cnt = bend - bstart;
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += NT) {
            const uint32_t slot = __ldg(a.vals + start + bstart + i);
            const float4 *r = a.rec + kRec4 * (size_t)slot;
            sslot[i] = slot;
            s0[i] = __ldg(r);
            s1[i] = __ldg(r + 1);
            s2[i] = __ldg(r + 2);
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; j--) {
            const uint32_t pos = (uint32_t)(bstart + j);
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; k++) v[k] = 0.f;
            bool contrib = false;
            if (pos < lst) {
                const float4 q0 = s0[j];
                const float4 q1 = s1[j];
                float dx, dy;
                const float power = splat_power(q0.x, q0.y, q0.z, q0.w, q1.x, fx, fy, dx, dy);
                if (!(power > 0.f)) {
                    const float G = __expf(power);
                    const float araw = __fmul_rn(q1.y, G);
                    const float alpha = fminf(kAlphaMax, araw);
                    if (!(alpha < kAlphaMin)) {
                        contrib = true;
                        const float4 q2 = s2[j];
                        const float om = __fsub_rn(1.f, alpha);
                        T = __fmul_rn(T, __frcp_rn(om));          // transmittance before splat j
                        acc0 = fmaf(la, lc0 - acc0, acc0);         // colour behind splat j
                        acc1 = fmaf(la, lc1 - acc1, acc1);
                        acc2 = fmaf(la, lc2 - acc2, acc2);
                        accD = fmaf(la, lz - accD, accD);
                        la = alpha;
                        lc0 = q2.x;
                        lc1 = q2.y;
                        lc2 = q2.z;
                        lz = q1.z;
                        const float wT = alpha * T;
                        v[8] = wT * gI0;
                        v[9] = wT * gI1;
                        v[10] = wT * gI2;
                        v[6] = wT * gD;
                        float dLda = (q2.x - acc0) * gI0 + (q2.y - acc1) * gI1 + (q2.z - acc2) * gI2 +
                                     (q1.z - accD) * gD;
                        dLda = dLda * T - bgdot / om;
                        if (!(araw > kAlphaMax)) {
                            const float dp = dLda * alpha;          // dalpha/dpower = alpha
                            v[5] = dLda * G;                        // dalpha/dopacity = G
                            v[0] = -dp * (q0.z * dx + q0.w * dy);
                            v[1] = -dp * (q1.x * dy + q0.w * dx);
                            v[2] = -0.5f * dp * dx * dx;
                            v[3] = -dp * dx * dy;
                            v[4] = -0.5f * dp * dy * dy;
                        }
                    }
                }
            }
            if (__any_sync(kFull, contrib)) {
                const float sum = warp_reduce_scatter16(v, lane);
                const int f = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
                if (!(lane & 1) && f != 7 && f < 11) atomicAdd(a.sgrad + (size_t)sslot[j] * 12 + f, sum);
            }
        }
    }
}

template <int B, int BD>
static cudaError_t launch_bwd(const RasterBwdArgs &a, cudaStream_t s)
{
    const int64_t items = a.g.Tv * a.V;
    k_render_bwd<B, BD><<<(unsigned)items, B * B, 0, s>>>(a);
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
