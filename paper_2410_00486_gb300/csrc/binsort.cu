// Tile binning of the window's projected splats (one shared sort for all views).
//
// The blending order of Eq. 1 (Sec. III-B, CaRtGS) is depth order within each
// tile.  Instead of a global LSD radix sort over 64-bit (tile, depth) keys, which
// reads and writes every instance once per digit pass, the sort here is
// most-significant-digit first with the tile id as one full-width digit:
//   1. k_count_agg   : per (slot chunk, tile) instance counts in shared memory; a
//                      slot is counted in the tiles of its rect its alpha >= 1/255 ellipse
//                      reaches (reach_box, over the tiles of the ellipse's bounding box),
//                      and a slot with at most 64 such tiles keeps the decisions as a bit
//                      mask for step 3
//   2. k_scan_part,  : exclusive scan -> tile ranges (the digit's bucket offsets), and
//      k_scan_out      the raster work order (tiles by decreasing list length)
//   3. k_scatter_agg : every instance is written once into its tile's bucket as the
//                      64-bit key (depth bits << 32 | slot), in one reserved run per
//                      (chunk, tile); the order inside a bucket is arbitrary
//   4. k_sort_*      : each bucket is sorted in shared memory.  The keys within a tile
//                      are unique (a slot appears once per tile), so the result is one
//                      well-defined order, (depth, slot) ascending, whatever order the
//                      scatter produced.  Depth is positive, so its IEEE bits order
//                      like its values.
// Buckets longer than kSortCapS are listed for a kernel with larger blocks and buffers,
// those longer than kSmallCap for a bitonic kernel with a larger shared-memory buffer;
// buckets beyond that are sorted in place in global memory by one block.  When a
// view's tile histogram does not fit in shared memory, k_count / k_scatter do steps 1
// and 3 with global atomics.
#include <algorithm>

#include "cgs_internal.cuh"

namespace cgs {

constexpr int kSmallCap = 2048;      // keys per tile sorted in shared memory by k_sort_tiles
constexpr int kBigThreads = 1024;
constexpr int kBigCap = 16384;       // keys held in shared memory by the big-tile kernel
constexpr uint64_t kPadKey = ~0ull;  // larger than any real key
constexpr size_t kAggMaxSmem = 96 * 1024;   // per-view tile histogram in shared memory
// Slots of a view per block of the count and scatter passes: 2048, or 1024 when 2048 would
// leave fewer than four blocks per SM.  Measured (whole sort, ms): the 16-view 300k window
// 0.844 / 0.831 / 0.862 / 1.024 for 1024 / 2048 / 4096 / 8192; one 100k view 0.101 / 0.115 /
// 0.153 (49 blocks of 2048 slots for 152 SMs).
constexpr int kChunkLarge = 2048, kChunkSmall = 1024;
static int chunk_for(int64_t n, int64_t V, int num_sms)
{
    return (n + kChunkLarge - 1) / kChunkLarge * V >= 4 * (int64_t)num_sms ? kChunkLarge : kChunkSmall;
}

// Scan of the per-tile counts: blocks of kScanThreads threads, kScanPer entries each.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanSpan = kScanThreads * kScanPer;
constexpr int kLenBuckets = 33;   // list-length buckets of the work order: 0 (empty), 1 + floor(log2 len)

struct BinWs {
    uint32_t *count;     // [Ttot + 1]
    uint32_t *cursor;    // [Ttot]
    uint32_t *nbig;      // [1]
    uint32_t *nmid;      // [1]
    uint32_t *big;       // [Ttot]: tiles for k_sort_big
    uint32_t *mid;       // [Ttot]: tiles for k_sort_tiles_l
    unsigned long long *part;   // [scan blocks]: instance total of each scan block
    uint32_t *bhist;     // [scan blocks x kLenBuckets]: list-length bucket histogram per scan block
    uint32_t *bcount;    // [chunks x Ttot]: per (slot chunk, tile) instance counts
    uint4 *slotrec;      // [V n]: per slot, the count pass's reach decisions (SlotBin)
    uint64_t *keys;      // [capacity]
};

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Sections: counters (one memset), big-tile list, per-chunk counts and per-slot bin
// records (shared-memory path only), keys.
static size_t ws_layout(int64_t capacity, int64_t Ttot, int64_t chunk_counts, int64_t slots, BinWs *w, void *base)
{
    size_t head = align256(sizeof(uint32_t) * (2 * (size_t)Ttot + 3));
    size_t bigb = 2 * align256(sizeof(uint32_t) * (size_t)Ttot);
    const size_t nsb = (size_t)((Ttot + kScanSpan - 1) / kScanSpan);
    size_t scb = align256(sizeof(unsigned long long) * nsb) + align256(sizeof(uint32_t) * kLenBuckets * nsb);
    size_t chb = align256(sizeof(uint32_t) * (size_t)chunk_counts);
    size_t mkb = chunk_counts > 0 ? align256(sizeof(uint4) * (size_t)slots) : 0;
    size_t keyb = align256(sizeof(uint64_t) * (size_t)(capacity > 0 ? capacity : 1));
    if (w && base) {
        char *b = static_cast<char *>(base);
        w->count = reinterpret_cast<uint32_t *>(b);
        w->cursor = w->count + Ttot + 1;
        w->nbig = w->cursor + Ttot;
        w->nmid = w->nbig + 1;
        w->big = reinterpret_cast<uint32_t *>(b + head);
        w->mid = reinterpret_cast<uint32_t *>(b + head + bigb / 2);
        w->part = reinterpret_cast<unsigned long long *>(b + head + bigb);
        w->bhist = reinterpret_cast<uint32_t *>(b + head + bigb + align256(sizeof(unsigned long long) * nsb));
        w->bcount = reinterpret_cast<uint32_t *>(b + head + bigb + scb);
        w->slotrec = reinterpret_cast<uint4 *>(b + head + bigb + scb + chb);
        w->keys = reinterpret_cast<uint64_t *>(b + head + bigb + scb + chb + mkb);
    }
    return head + bigb + scb + chb + mkb + keyb;
}

// Per-(chunk, tile) counts kept between the count and scatter passes when a view's tile
// histogram fits in shared memory.
static int64_t chunk_count_entries(int64_t n, int64_t V, int64_t Tv, int chunk)
{
    if (sizeof(uint32_t) * (size_t)Tv > kAggMaxSmem) return 0;
    return (n + chunk - 1) / chunk * V * Tv;
}

size_t bin_ws_bytes(int64_t capacity, int64_t n, int64_t V, int64_t Tv, int num_sms)
{
    return ws_layout(capacity, Tv * V, chunk_count_entries(n, V, Tv, chunk_for(n, V, num_sms)), V * n, nullptr,
                     nullptr);
}

__device__ __forceinline__ bool load_slot(const float4 *__restrict__ rec, int64_t slot, float &u, float &v,
                                          float &z, int &r)
{
    const float *rf = reinterpret_cast<const float *>(rec + kRec4 * slot);
    r = __float_as_int(__ldg(rf + 7));
    if (r <= 0) return false;
    float4 a = __ldg(rec + kRec4 * slot);
    u = a.x;
    v = a.y;
    z = __ldg(rf + 6);
    return true;
}

// The per-slot part of the tile reach test (record fields 2, 3, 4: conic; 11: tau).  With
// rect lists every tile of the rect is kept (mode 1, "reaches everything").
__device__ __forceinline__ ReachPre load_reach(const float4 *__restrict__ rec, int64_t slot, const Grid &g)
{
    if (g.rect_lists) return ReachPre{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1};
    const float *rf = reinterpret_cast<const float *>(rec + kRec4 * slot);
    return reach_prepare(__ldg(rf + 2), __ldg(rf + 3), __ldg(rf + 4), __ldg(rf + 11));
}

// Does the slot (centre u, v) belong in tile (tx, ty): can it reach alpha >= 1/255 there?
__device__ __forceinline__ bool in_tile(const ReachPre &e, float u, float v, int tx, int ty, const Grid &g)
{
    const float bx0 = (float)(tx * g.B), bx1 = (float)(min(tx * g.B + g.B, g.W) - 1);
    const float by0 = (float)(ty * g.B), by1 = (float)(min(ty * g.B + g.B, g.H) - 1);
    return reach_box(e, u, v, bx0, bx1, by0, by1);
}

__global__ void k_count(const float4 *__restrict__ rec, int64_t n, int V, Grid g, uint32_t *__restrict__ count)
{
    const int64_t total = (int64_t)V * n;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total; s += (int64_t)gridDim.x * blockDim.x) {
        float u, v, z;
        int r;
        if (!load_slot(rec, s, u, v, z, r)) continue;
        const int64_t view = s / n;
        Rect R = tile_rect(u, v, r, g);
        const ReachPre e = load_reach(rec, s, g);
        uint32_t *base = count + view * g.Tv;
        for (int ty = R.y0; ty < R.y1; ty++)
            for (int tx = R.x0; tx < R.x1; tx++)
                if (in_tile(e, u, v, tx, ty, g)) atomicAdd(base + ty * g.Tx + tx, 1u);
    }
}

// Shared-memory aggregated variants, used when a view's tile histogram fits in shared
// memory: block (c, v) owns slots [c*chunk, (c+1)*chunk) of view v, counts its
// instances per tile in shared memory and touches each global counter once.
constexpr int kAggThreads = 512;
// Three resident blocks per SM (at most 42 registers; the count pass needs 49 unbounded):
// 1.076 -> 1.064 ms for the whole sort on the 16-view window.
constexpr int kAggMinBlocks = 3;

// The tiles of rect R that the box [u - ex, u + ex] x [v - ey, v + ey] of the splat's
// alpha >= 1/255 ellipse (reach_prepare) overlaps, widened by one pixel on every side:
// reach_box's first test (dx <= ex, dy <= ey) fails on every other tile of R.  With |u|,
// |v|, ex, ey at most 2^20 the float sums below are within a quarter pixel of exact, well
// inside the margin; beyond that (or with rect lists) the whole rect is kept.
__device__ __forceinline__ Rect reach_rect(const ReachPre &e, float u, float v, const Rect &R, const Grid &g)
{
    if (e.mode == 0) return Rect{R.x0, R.x0, R.y0, R.y0};   // reaches nothing
    const float lim = 1048576.f;
    if (e.mode == 1 || !(fabsf(u) <= lim && fabsf(v) <= lim && e.ex <= lim && e.ey <= lim)) return R;
    const float inv = 1.f / (float)g.B;   // a power of two: exact
    Rect T;
    T.x0 = max(R.x0, (int)floorf(__fmul_rn(__fsub_rn(__fsub_rn(u, e.ex), 1.f), inv)));
    T.x1 = min(R.x1, (int)floorf(__fmul_rn(__fadd_rn(__fadd_rn(u, e.ex), 1.f), inv)) + 1);
    T.y0 = max(R.y0, (int)floorf(__fmul_rn(__fsub_rn(__fsub_rn(v, e.ey), 1.f), inv)));
    T.y1 = min(R.y1, (int)floorf(__fmul_rn(__fadd_rn(__fadd_rn(v, e.ey), 1.f), inv)) + 1);
    if (T.x1 <= T.x0 || T.y1 <= T.y0) return Rect{R.x0, R.x0, R.y0, R.y0};
    return T;
}

// Calls f(tile in view, key) for every tile of the rects of the visible slots [s0, s1) of
// a view that the slot can reach (in_tile), load-balanced pair by pair over the lanes of
// each warp: a warp takes the next group of 32 slots from the shared counter `next`
// (groups differ widely in work), stages their data in shared memory, forms the prefix
// sum of their item counts, and hands out one item per lane and step; a lane finds the
// slot owning item j by a 5-step binary search over the prefix (shuffles) and reads the
// slot from the stage.  An item is one tile of the slot's reach rect (reach_rect,
// row-major) to test, or, in the scatter pass for a slot with a recorded mask, one set
// bit of the mask.
// Slot bin records (SlotBin, 16 bytes per slot, written by the count pass for every slot
// of the chunk): a slot whose reach rect has at most 64 tiles keeps one bit per tile
// (row-major over that rect) saying whether it passed the reach test, with its depth bits
// and the rect's first tile and width, so the scatter pass emits its tiles from the record
// alone; a larger rect is marked for testing again; a slot that reaches no tile is zero.
constexpr int kMaskTiles = 64;
// SlotBin = (mask low, mask high, depth bits, meta); meta is 0 (no tile), kBinLarge, or
// kBinSmall | (width - 1) << 15 | first tile (tile id in the view, < 2^15).
constexpr uint32_t kBinSmall = 0x80000000u, kBinLarge = 0x40000000u;
static_assert(kAggMaxSmem / sizeof(uint32_t) <= 32768, "first tile of a SlotBin takes 15 bits");

struct PairStage {      // one warp's 32 slots
    float4 a[32];       // u, v, 1/w (reach rect width w), depth bits
    int4 b[32];         // reach rect's first tile (id in the view), w, mask kept, x0 | y0 << 16
    float4 c[32];       // reach test: A, 2B, C, t2
    float4 d[32];       //             ex, ey, B/C, B/A
    int4 e[32];         //             mode; tile mask low and high words
};

// Position of the k-th (from 0) set bit of x; x has more than k set bits.
__device__ __forceinline__ int nth_bit32(uint32_t x, int k)
{
    int pos = 0;
#pragma unroll
    for (int h = 16; h > 0; h >>= 1) {
        const uint32_t lo = x & ((1u << h) - 1u);
        const int c = __popc(lo);
        if (k >= c) {
            k -= c;
            x >>= h;
            pos += h;
        } else {
            x = lo;
        }
    }
    return pos;
}
__device__ __forceinline__ int nth_bit64(uint64_t x, int k)
{
    const uint32_t lo = (uint32_t)x;
    const int c = __popc(lo);
    return k < c ? nth_bit32(lo, k) : 32 + nth_bit32((uint32_t)(x >> 32), k - c);
}

template <bool RECORD, class F>
__device__ __forceinline__ void for_each_tile_pair(const float4 *__restrict__ rec, int64_t n, int view, int64_t s0,
                                                   int64_t s1, const Grid &g, uint32_t *next, PairStage &st,
                                                   uint4 *__restrict__ slotrec, F f)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t grp = 0;
        if (lane == 0) grp = atomicAdd(next, 1u);
        grp = __shfl_sync(kFull, grp, 0);
        const int64_t wb = s0 + 32 * (int64_t)grp;
        if (wb >= s1) break;   // warp-uniform
        const int64_t gi = wb + lane;
        const int64_t slot = (int64_t)view * n + gi;
        int cnt = 0, t0 = 0, w = 0, small = 0, xy0 = 0;
        float u = 0.f, v = 0.f;
        uint32_t zb = 0u;
        ReachPre e{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
        uint64_t mk = 0ull;
        bool test = RECORD;   // slot's tiles come from the reach test (else from its mask)
        if (!RECORD && gi < s1) {
            const uint4 sb = slotrec[slot];
            if (sb.w & kBinSmall) {
                mk = ((uint64_t)sb.y << 32) | sb.x;
                cnt = __popcll(mk);
                zb = sb.z;
                w = (int)((sb.w >> 15) & 63u) + 1;
                t0 = (int)(sb.w & 0x7fffu);
                small = 1;
            } else if (sb.w & kBinLarge) {
                test = true;
            }
        }
        float z;
        int r;
        if (test && gi < s1 && load_slot(rec, slot, u, v, z, r)) {
            const Rect R = tile_rect(u, v, r, g);
            if (R.x1 > R.x0 && R.y1 > R.y0) {
                e = load_reach(rec, slot, g);
                const Rect T = reach_rect(e, u, v, R, g);
                w = T.x1 - T.x0;
                cnt = w * (T.y1 - T.y0);
                t0 = T.y0 * g.Tx + T.x0;
                xy0 = T.x0 | (T.y0 << 16);
                small = RECORD && cnt <= kMaskTiles;
                zb = __float_as_uint(z);
            }
        }
        st.a[lane] = make_float4(u, v, w ? 1.f / (float)w : 0.f, __uint_as_float(zb));
        st.b[lane] = make_int4(t0, w, small, xy0);
        st.c[lane] = make_float4(e.A, e.B2, e.C, e.t2);
        st.d[lane] = make_float4(e.ex, e.ey, e.bc, e.ba);
        st.e[lane] = make_int4(e.mode, (int)(uint32_t)mk, (int)(uint32_t)(mk >> 32), 0);
        __syncwarp();
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        for (int r0 = 0; r0 < total; r0 += 32) {   // warp-uniform
            const int j = r0 + lane;
            int L = 0;   // owner: the number of lanes whose inclusive prefix is <= j
#pragma unroll
            for (int b = 16; b > 0; b >>= 1)
                if (__shfl_sync(kFull, incl, L + b - 1) <= j) L += b;
            const int oend = __shfl_sync(kFull, incl, L), ocnt = __shfl_sync(kFull, cnt, L);
            const int4 ob = st.b[L];
            const bool live = j < total;
            const bool from_mask = !RECORD && ob.z;
            const int k = j - (oend - ocnt);
            bool pass = false;
            if (live) {
                const float4 oa = st.a[L];
                const int idx = from_mask ? nth_bit64(((uint64_t)(uint32_t)st.e[L].z << 32) | (uint32_t)st.e[L].y, k)
                                          : k;   // row-major index into the reach rect
                int row = (int)(((float)idx + 0.5f) * oa.z), col = idx - row * ob.y;
                if (col < 0) {           // the float quotient is within one of the exact one
                    row--;
                    col += ob.y;
                } else if (col >= ob.y) {
                    row++;
                    col -= ob.y;
                }
                const int t = ob.x + row * g.Tx + col;
                if (from_mask) {
                    pass = true;
                } else {
                    const float4 oc = st.c[L], od = st.d[L];
                    const ReachPre oe{oc.x, oc.y, oc.z, oc.w, od.x, od.y, od.z, od.w, st.e[L].x};
                    pass = in_tile(oe, oa.x, oa.y, (ob.w & 0xffff) + col, (ob.w >> 16) + row, g);
                }
                if (pass) {
                    const uint32_t oslot = (uint32_t)((int64_t)view * n + wb + L);
                    f(t, ((uint64_t)__float_as_uint(oa.w) << 32) | (uint64_t)oslot);
                }
            }
            if (RECORD) {
                // this step's decisions for the masked slots: the first lane of each owner's
                // run of lanes ORs the run's bits into the owner's mask (one writer per owner
                // and step)
                const unsigned bal = __ballot_sync(kFull, pass);
                const int first = max(0, (oend - ocnt) - r0);
                if (live && ob.z && lane == first) {
                    const int runlen = min(oend - r0, 32) - first;
                    const uint32_t bits = (bal >> first) & (runlen >= 32 ? kFull : ((1u << runlen) - 1u));
                    const uint64_t m = (((uint64_t)(uint32_t)st.e[L].z << 32) | (uint32_t)st.e[L].y) |
                                       ((uint64_t)bits << k);   // k + runlen <= kMaskTiles
                    st.e[L].y = (int)(uint32_t)m;
                    st.e[L].z = (int)(uint32_t)(m >> 32);
                }
                __syncwarp();
            }
        }
        if (RECORD && gi < s1) {
            uint4 sb = make_uint4(0u, 0u, 0u, 0u);
            if (cnt > 0 && small)
                sb = make_uint4((uint32_t)st.e[lane].y, (uint32_t)st.e[lane].z, zb,
                                kBinSmall | ((uint32_t)(w - 1) << 15) | (uint32_t)t0);
            else if (cnt > 0)
                sb = make_uint4(0u, 0u, zb, kBinLarge);
            slotrec[slot] = sb;
        }
        __syncwarp();   // the stage is rewritten by the next group
    }
}

// Dynamic shared memory of the aggregated count and scatter kernels: one PairStage per
// warp, then the view's tile histogram.
constexpr int kAggWarps = kAggThreads / 32;
constexpr size_t kStageBytes = sizeof(PairStage) * kAggWarps;

__global__ void __launch_bounds__(kAggThreads, kAggMinBlocks)
k_count_agg(const float4 *__restrict__ rec, int64_t n, int chunk, Grid g, uint32_t *__restrict__ count,
            uint32_t *__restrict__ bcount, uint4 *__restrict__ slotrec)
{
    extern __shared__ float4 smem_agg[];
    PairStage *stage = reinterpret_cast<PairStage *>(smem_agg);
    uint32_t *hist = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(smem_agg) + kStageBytes);
    const int view = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    __shared__ uint32_t next;
    for (int t = threadIdx.x; t < g.Tv; t += blockDim.x) hist[t] = 0;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    for_each_tile_pair<true>(rec, n, view, s0, s1, g, &next, stage[threadIdx.x >> 5], slotrec,
                             [&](int t, uint64_t) { atomicAdd(&hist[t], 1u); });
    __syncthreads();
    uint32_t *base = count + (int64_t)view * g.Tv;
    uint32_t *mine = bcount + ((int64_t)view * gridDim.x + blockIdx.x) * g.Tv;
    for (int t = threadIdx.x; t < g.Tv; t += blockDim.x) {
        const uint32_t c = hist[t];
        mine[t] = c;
        if (c) atomicAdd(base + t, c);
    }
}

// Multi-block scan of the per-tile counts and the raster work order (tiles by
// decreasing list length, bucketed by floor(log2(len)), longest bucket first; tile order
// inside a bucket is arbitrary), in two launches over blocks of kScanSpan tiles.
// k_scan_part: each block's instance total and its histogram of length buckets.
__device__ __forceinline__ uint32_t len_bucket(uint32_t len) { return len ? 32 - __clz(len) : 0; }

__global__ void __launch_bounds__(kScanThreads)
k_scan_part(const uint32_t *__restrict__ count, int64_t Ttot, unsigned long long *__restrict__ part,
            uint32_t *__restrict__ bhist)
{
    __shared__ unsigned long long wsum[kScanThreads / 32];
    __shared__ uint32_t hist[kLenBuckets];
    if (threadIdx.x < kLenBuckets) hist[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * kScanSpan;
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        const int64_t t = b0 + k * kScanThreads + threadIdx.x;
        if (t < Ttot) {
            const uint32_t c = count[t];
            sum += c;
            atomicAdd(&hist[len_bucket(c)], 1u);
        }
    }
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int i = 0; i < kScanThreads / 32; i++) tot += wsum[i];
        part[blockIdx.x] = tot;
    }
    if (threadIdx.x < kLenBuckets) bhist[(int64_t)blockIdx.x * kLenBuckets + threadIdx.x] = hist[threadIdx.x];
}

// k_scan_out: each block adds the earlier blocks' totals, scans its counts into bucket
// starts (written over the counts, for the scatter) and ranges, both clamped to the
// capacity, and places its tiles in the work order after every longer bucket's tiles and
// the earlier blocks' tiles of the same bucket.  Block 0 writes the instance total, the
// capacity status, and clears the long-tile list.
__global__ void __launch_bounds__(kScanThreads)
k_scan_out(uint32_t *__restrict__ count, int64_t Ttot, int64_t capacity, const unsigned long long *__restrict__ part,
           const uint32_t *__restrict__ bhist, int nblocks, uint32_t *__restrict__ ranges,
           uint32_t *__restrict__ order, int64_t *__restrict__ n_inst, uint32_t *__restrict__ nbig,
           int32_t *__restrict__ status)
{
    __shared__ unsigned long long wtot[kScanThreads / 32];
    __shared__ unsigned long long s_pre;
    __shared__ uint32_t btot[kLenBuckets], offs[kLenBuckets];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long cap = (unsigned long long)capacity;
    if (threadIdx.x == 0) {
        unsigned long long pre = 0, tot = 0;
        for (int b = 0; b < nblocks; b++) {
            const unsigned long long x = part[b];
            pre += b < (int)blockIdx.x ? x : 0ull;
            tot += x;
        }
        s_pre = pre;
        if (blockIdx.x == 0) {
            *nbig = 0u;   // the long-tile list of k_sort_tiles starts empty
            *n_inst = (int64_t)tot;
            count[Ttot] = (uint32_t)min(tot, cap);
            if (tot > cap) set_status(status, CGS_ERR_CAPACITY);
        }
    }
    if (order && threadIdx.x < kLenBuckets) {
        uint32_t all = 0, before = 0;
        for (int b = 0; b < nblocks; b++) {
            const uint32_t x = bhist[(int64_t)b * kLenBuckets + threadIdx.x];
            all += x;
            before += b < (int)blockIdx.x ? x : 0u;
        }
        btot[threadIdx.x] = all;
        offs[threadIdx.x] = before;
    }
    __syncthreads();
    if (order && threadIdx.x < kLenBuckets) {
        uint32_t longer = 0;
        for (int b = threadIdx.x + 1; b < kLenBuckets; b++) longer += btot[b];
        offs[threadIdx.x] += longer;
    }
    const int64_t b0 = (int64_t)blockIdx.x * kScanSpan;
    uint32_t c[kScanPer];
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        const int64_t t = b0 + k * kScanThreads + threadIdx.x;
        c[k] = t < Ttot ? count[t] : 0u;
    }
    unsigned long long run = s_pre;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {   // 1024 entries at a time, in tile order
        unsigned long long incl = c[k];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wtot[w] = incl;
        __syncthreads();
        unsigned long long wpre = 0, btot_k = 0;
        for (int i = 0; i < kScanThreads / 32; i++) {
            const unsigned long long x = wtot[i];
            wpre += i < w ? x : 0ull;
            btot_k += x;
        }
        const int64_t t = b0 + k * kScanThreads + threadIdx.x;
        if (t < Ttot) {
            const unsigned long long st = run + wpre + incl - c[k], en = run + wpre + incl;
            count[t] = (uint32_t)min(st, cap);
            ranges[2 * t] = (uint32_t)min(st, cap);
            ranges[2 * t + 1] = (uint32_t)min(en, cap);
        }
        run += btot_k;
        __syncthreads();   // wtot is rewritten by the next round
    }
    if (order) {
#pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            const int64_t t = b0 + k * kScanThreads + threadIdx.x;
            if (t < Ttot) order[atomicAdd(&offs[len_bucket(c[k])], 1u)] = (uint32_t)t;
        }
    }
}

__global__ void k_scatter(const float4 *__restrict__ rec, int64_t n, int V, Grid g,
                          const uint32_t *__restrict__ start, uint32_t *__restrict__ cursor,
                          uint64_t *__restrict__ keys, int64_t capacity)
{
    const int64_t total = (int64_t)V * n;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < total; s += (int64_t)gridDim.x * blockDim.x) {
        float u, v, z;
        int r;
        if (!load_slot(rec, s, u, v, z, r)) continue;
        const int64_t view = s / n;
        Rect R = tile_rect(u, v, r, g);
        const uint64_t key = ((uint64_t)__float_as_uint(z) << 32) | (uint64_t)(uint32_t)s;
        const ReachPre e = load_reach(rec, s, g);
        for (int ty = R.y0; ty < R.y1; ty++)
            for (int tx = R.x0; tx < R.x1; tx++) {
                if (!in_tile(e, u, v, tx, ty, g)) continue;
                const int64_t t = view * g.Tv + ty * g.Tx + tx;
                const uint64_t pos = (uint64_t)start[t] + atomicAdd(cursor + t, 1u);
                if (pos < (uint64_t)capacity) keys[pos] = key;
            }
    }
}

// Aggregated scatter (same block decomposition as k_count_agg): the block counts its
// instances per tile again, reserves one contiguous run per tile in each bucket with a
// single global atomic, then places its instances with shared-memory atomics.
__global__ void __launch_bounds__(kAggThreads, kAggMinBlocks)
k_scatter_agg(const float4 *__restrict__ rec, int64_t n, int chunk, Grid g, const uint32_t *__restrict__ start,
              uint32_t *__restrict__ cursor, const uint32_t *__restrict__ bcount, uint4 *__restrict__ slotrec,
              uint64_t *__restrict__ keys, int64_t capacity)
{
    extern __shared__ float4 smem_agg[];
    PairStage *stage = reinterpret_cast<PairStage *>(smem_agg);
    uint32_t *hist = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(smem_agg) + kStageBytes);  // run positions
    const int view = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    // this chunk's per-tile counts (from the count pass): reserve one run per tile
    const int64_t tbase = (int64_t)view * g.Tv;
    const uint32_t *mine = bcount + ((int64_t)view * gridDim.x + blockIdx.x) * g.Tv;
    __shared__ uint32_t next;
    if (threadIdx.x == 0) next = 0;
    for (int t0 = threadIdx.x; t0 < g.Tv; t0 += 4 * blockDim.x) {   // four tiles in flight
        uint32_t c[4], st4[4], r[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int t = t0 + q * (int)blockDim.x;
            c[q] = t < g.Tv ? mine[t] : 0u;
            st4[q] = t < g.Tv ? start[tbase + t] : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int t = t0 + q * (int)blockDim.x;
            r[q] = c[q] ? atomicAdd(cursor + tbase + t, c[q]) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int t = t0 + q * (int)blockDim.x;
            if (t < g.Tv) hist[t] = c[q] ? st4[q] + r[q] : 0u;
        }
    }
    __syncthreads();
    for_each_tile_pair<false>(rec, n, view, s0, s1, g, &next, stage[threadIdx.x >> 5], slotrec,
                              [&](int t, uint64_t key) {
                                  const uint64_t pos = atomicAdd(&hist[t], 1u);
                                  if (pos < (uint64_t)capacity) keys[pos] = key;
                              });
}

// Compare-exchange network of an ascending bitonic sort in which every comparator
// puts the smaller key at the lower index (the first stage of each merge compares
// mirrored pairs), so padding with the largest key at the end is never moved.
// k (merge size) and d (comparator distance) are powers of two: index arithmetic is
// shifts and masks (lk = log2 k, ld = log2 d).
__device__ __forceinline__ void bitonic_pair(uint32_t i, uint32_t lk, uint32_t ld, bool flip, uint32_t &a,
                                             uint32_t &b)
{
    if (flip) {
        const uint32_t blk = i >> (lk - 1), off = i & ((1u << (lk - 1)) - 1u);
        a = (blk << lk) + off;
        b = (blk << lk) + (1u << lk) - 1u - off;
    } else {
        const uint32_t blk = i >> ld, off = i & ((1u << ld) - 1u);
        a = (blk << (ld + 1)) + off;
        b = a + (1u << ld);
    }
}

__device__ __forceinline__ void smem_bitonic(uint64_t *s, uint32_t P)
{
    const uint32_t lp = 31 - __clz(P);
    for (uint32_t lk = 1; lk <= lp; lk++) {
        for (int ld = (int)lk - 1; ld >= 0; ld--) {
            const bool flip = (ld == (int)lk - 1);
            for (uint32_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
                uint32_t a, b;
                bitonic_pair(i, lk, (uint32_t)ld, flip, a, b);
                const uint64_t x = s[a], y = s[b];
                if (y < x) {
                    s[a] = y;
                    s[b] = x;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ uint32_t next_pow2(uint32_t x)
{
    return x <= 1 ? 1u : 1u << (32 - __clz(x - 1));
}

// Per-tile sort in shared memory (lists of up to kSmallCap keys).  The key is (depth bits
// << 32 | slot) and is unique in a tile.  Most tiles take a one-pass bucket sort (below);
// a tile whose depths crowd into a few buckets takes a stable LSD radix sort: sorting by
// the depth bits (8-bit digits; a pass whose digit is the same for every key of the tile
// is skipped) and then ordering each run of equal depths by slot gives exactly the
// (depth, slot) order.  Stability: warp w owns a contiguous segment of the list and
// walks it 32 keys at a time; a ballot multisplit ranks equal digits within a step, and
// per-warp digit histograms scanned digit-major give each (digit, warp) its start.
constexpr int kTieRun = 32;   // longest run of equal 16-bit depth prefixes fixed by insertion
// Lists of at most kSortCapS keys are sorted by blocks of kSortThreadsS threads (most tiles);
// longer ones, up to kSmallCap, by blocks of kSortThreadsL threads taking them from a list.
// Per-tile work that every warp repeats (digit histograms, the digit scan, partial 32-key
// steps) dominated with eight warps on lists of a few hundred keys: on the 16-view window
// (lists of 65 to 1.6k keys, 93% of keys in lists of 257 to 1024) four warps and a
// 1024-key cap took the whole sort from 0.986 to 0.863 ms (eight warps with that cap 0.965,
// two warps with a 512-key cap 0.886).
constexpr int kSortThreadsS = 128, kSortCapS = 1024, kSortThreadsL = 256;

// Lanes of the warp whose 8-bit digit equals this lane's (restricted to `valid` lanes),
// from eight ballots, one per digit bit (a ballot-based multisplit: __match_any_sync
// runs on a low-throughput pipe).
__device__ __forceinline__ unsigned same_digit_lanes(uint32_t d, unsigned valid)
{
    unsigned peers = valid;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(kFull, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// Exclusive scan over the 32 NW threads of a block.
template <int NW>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t pre = 0;
    for (int i = 0; i < w; i++) pre += wsum[i];
    __syncthreads();
    return pre + incl - x;
}

// Buckets of the one-pass sort: the top 11 bits of a tile's depth range (the bucket array
// shares the radix sort's digit histograms and ranks, which the long-list kernel's 2048
// buckets fit).  A tile is bucket-sorted when its rank work, the sum over buckets of the
// squared bucket size, is at most kRankWork per key; else it takes the radix sort.  On the
// 16-view window the bucket sort took the whole bin sort from 0.803 to 0.755 ms, lists
// identical (a bound of 16 per key: 0.769 ms; 64 as fast as 32).
constexpr int kBucketBits = 11, kBuckets = 1 << kBucketBits;
constexpr uint32_t kRankWork = 32;

template <int NTH, int CAP>
struct SortSmem {
    uint64_t bufA[CAP], bufB[CAP];
    union {
        struct {
            uint32_t hist[NTH / 32][256];
            uint16_t lrank[CAP];
        } r;                         // radix sort: per-warp digit histograms, ranks
        uint32_t bins[kBuckets];     // bucket sort: counts, then bucket starts, then ends
    } u;
    uint32_t wsum[NTH / 32], wmin[NTH / 32], wmax[NTH / 32];
    int s_long;   // a run of equal 16-bit prefixes longer than kTieRun
};

// One-pass bucket sort of a tile's keys (in bufA; depth bits in [dmin, dmax]; bins
// already zero).  Bucket = the top kBucketBits of the depth bits less dmin: a
// shared-memory histogram, its scan, a scatter into bucket order (bufB, any order inside
// a bucket), then each key's place is its bucket's start plus the number of smaller keys
// in its bucket.  Buckets are monotone in the key and the keys are unique, so the result
// is the (depth, slot) order whatever the order of the atomics.  Returns false, with bufA
// unchanged, when the rank work would exceed kRankWork per key.
template <int NTH, int CAP>
__device__ __forceinline__ bool bucket_sort_tile(SortSmem<NTH, CAP> &sm, uint32_t *__restrict__ vals, uint32_t st,
                                                 uint32_t len, uint32_t dmin, uint32_t dmax)
{
    constexpr int NW = NTH / 32;
    constexpr int BPT = kBuckets / NTH;   // buckets per thread in the scan
    static_assert(BPT * NTH == kBuckets, "a block covers the buckets evenly");
    uint64_t *bufA = sm.bufA, *bufB = sm.bufB;
    uint32_t *bins = sm.u.bins;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int hb = 32 - __clz(dmax - dmin);   // bit length of the depth range
    const int sh = max(0, hb - kBucketBits);
    auto bucket = [&](uint64_t k) { return ((uint32_t)(k >> 32) - dmin) >> sh; };   // < kBuckets
    for (uint32_t i = threadIdx.x; i < len; i += NTH) atomicAdd(&bins[bucket(bufA[i])], 1u);
    __syncthreads();
    // exclusive scan of the buckets (BPT consecutive ones per thread) and the rank work
    uint32_t c[BPT], tot = 0u, sq = 0u;
#pragma unroll
    for (int b = 0; b < BPT; b++) {
        c[b] = bins[threadIdx.x * BPT + b];
        tot += c[b];
        sq += c[b] * c[b];
    }
    uint32_t incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(kFull, sq, off);
    if (lane == 31) sm.wsum[w] = incl;
    if (lane == 0) sm.wmax[w] = sq;
    __syncthreads();
    uint32_t pre = 0u, sqt = 0u;
    for (int i = 0; i < NW; i++) {
        pre += i < w ? sm.wsum[i] : 0u;
        sqt += sm.wmax[i];
    }
    uint32_t off = pre + incl - tot;
#pragma unroll
    for (int b = 0; b < BPT; b++) {
        bins[threadIdx.x * BPT + b] = off;   // start of the bucket
        off += c[b];
    }
    __syncthreads();
    if (sqt > kRankWork * len) return false;   // block-uniform
    for (uint32_t i = threadIdx.x; i < len; i += NTH) {
        const uint64_t k = bufA[i];
        bufB[atomicAdd(&bins[bucket(k)], 1u)] = k;
    }
    __syncthreads();
    // bins[b] is now the end of bucket b, which is the start of bucket b + 1
    for (uint32_t j = threadIdx.x; j < len; j += NTH) {
        const uint64_t k = bufB[j];
        const uint32_t b = bucket(k);
        const uint32_t s0 = b ? bins[b - 1] : 0u, s1 = bins[b];
        uint32_t r = 0u;
        for (uint32_t i = s0; i < s1; i++) r += bufB[i] < k ? 1u : 0u;
        vals[st + s0 + r] = (uint32_t)k;
    }
    return true;
}

// Sort of one tile's list (2 <= len <= CAP keys) in shared memory by a block of NTH
// threads, written to vals as slot ids: the bucket sort, else the stable LSD radix sort.
template <int NTH, int CAP>
__device__ __forceinline__ void sort_tile(SortSmem<NTH, CAP> &sm, const uint64_t *__restrict__ keys,
                                          uint32_t *__restrict__ vals, uint32_t st, uint32_t len)
{
    constexpr int NW = NTH / 32;
    constexpr int DPT = 256 / NTH;   // digits per thread in the digit scan
    static_assert(DPT >= 1 && DPT * NTH == 256, "a block covers the 256 digits evenly");
    uint64_t *bufA = sm.bufA, *bufB = sm.bufB;
    uint32_t (*hist)[256] = sm.u.r.hist;
    uint16_t *lrank = sm.u.r.lrank;
    uint32_t *wsum = sm.wsum, *wmin = sm.wmin, *wmax = sm.wmax;
    int &s_long = sm.s_long;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // load, and find the range of the depth bits over the tile (positive floats: the bits
    // order like the values)
    uint32_t dmin = ~0u, dmax = 0u;
    for (uint32_t i0 = threadIdx.x; i0 < len; i0 += 4 * NTH) {   // four keys in flight
        uint64_t kk[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = i0 + q * NTH;
            kk[q] = i < len ? keys[st + i] : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = i0 + q * NTH;
            if (i < len) {
                bufA[i] = kk[q];
                const uint32_t dd = (uint32_t)(kk[q] >> 32);
                dmin = min(dmin, dd);
                dmax = max(dmax, dd);
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        dmin = min(dmin, __shfl_xor_sync(kFull, dmin, off));
        dmax = max(dmax, __shfl_xor_sync(kFull, dmax, off));
    }
    if (lane == 0) {
        wmin[w] = dmin;
        wmax[w] = dmax;
    }
    if (threadIdx.x == 0) s_long = 0;
    for (int i = threadIdx.x; i < kBuckets; i += NTH) sm.u.bins[i] = 0u;   // for the bucket sort
    __syncthreads();
    dmin = ~0u;
    dmax = 0u;
    for (int i = 0; i < NW; i++) {
        dmin = min(dmin, wmin[i]);
        dmax = max(dmax, wmax[i]);
    }
    if (bucket_sort_tile<NTH, CAP>(sm, vals, st, len, dmin, dmax)) return;
    uint64_t *src = bufA, *dst = bufB;
    const uint32_t per = (len + NW - 1) / NW;
    const uint32_t seg0 = min(len, (uint32_t)w * per), seg1 = min(len, seg0 + per);
    // The digits are taken from the depth bits less the tile's smallest, r = d - dmin.
    // First attempt: radix passes over the 16 highest bits of r's range [lo, hb) (two
    // passes instead of up to four); keys equal in r >> lo are then ordered by the full key
    // (depth, slot), run by run.  A tile with such a run longer than kTieRun is sorted again
    // over every bit (lo = 0), which leaves only runs of equal depth.
    const int hb = 32 - __clz(dmax - dmin);   // bit length of the range
    int lo = max(0, hb - 16);
    for (int attempt = 0; attempt < 2; attempt++) {
        for (int shift = lo; shift < hb; shift += 8) {
            for (int i = lane; i < 256; i += 32) hist[w][i] = 0u;
            __syncwarp();
            // count, and keep each key's rank among the equal digits of this warp's segment
            // (earlier 32-key groups first, then lanes in order): the scatter below needs no
            // ranking of its own
            for (uint32_t c = seg0; c < seg1; c += 32) {
                const uint32_t e = c + lane;
                const bool valid = e < seg1;
                const uint32_t d = valid ? ((((uint32_t)(src[e] >> 32) - dmin) >> shift) & 0xffu) : 0u;
                const unsigned peers = same_digit_lanes(d, __ballot_sync(kFull, valid));
                const uint32_t before = valid ? hist[w][d] : 0u;
                __syncwarp();
                if (valid) {
                    lrank[e] = (uint16_t)(before + __popc(peers & ((1u << lane) - 1u)));
                    if (lane == __ffs(peers) - 1) hist[w][d] = before + __popc(peers);
                }
                __syncwarp();
            }
            __syncthreads();
            {   // start of each (digit, warp) run: digit-major exclusive scan (DPT consecutive
                // digits per thread)
                uint32_t cnts[DPT][NW], tot = 0u;
#pragma unroll
                for (int d = 0; d < DPT; d++)
#pragma unroll
                    for (int i = 0; i < NW; i++) {
                        cnts[d][i] = hist[i][threadIdx.x * DPT + d];
                        tot += cnts[d][i];
                    }
                uint32_t off = block_excl_scan<NW>(tot, wsum);
#pragma unroll
                for (int d = 0; d < DPT; d++)
#pragma unroll
                    for (int i = 0; i < NW; i++) {
                        hist[i][threadIdx.x * DPT + d] = off;
                        off += cnts[d][i];
                    }
            }
            __syncthreads();
            for (uint32_t e = seg0 + lane; e < seg1; e += 32) {
                const uint64_t k = src[e];
                const uint32_t d = (((uint32_t)(k >> 32) - dmin) >> shift) & 0xffu;
                dst[hist[w][d] + lrank[e]] = k;
            }
            __syncthreads();
            uint64_t *tmp = src;
            src = dst;
            dst = tmp;
        }
        // runs of keys equal in depth bits lo..31: order by the full key (depth, slot);
        // insertion sort by the run's first thread (runs are rare and short)
        const bool check = lo > 0;
        auto rkey = [&](uint32_t i) { return ((uint32_t)(src[i] >> 32) - dmin) >> lo; };
        for (uint32_t i = threadIdx.x; i + 1 < len; i += NTH) {
            const uint32_t di = rkey(i);
            const bool starts = (i == 0 || rkey(i - 1) != di) && rkey(i + 1) == di;
            if (!starts) continue;
            uint32_t e = i + 1;
            while (e < len && rkey(e) == di) e++;
            if (check && e - i > (uint32_t)kTieRun) {
                s_long = 1;
                continue;
            }
            for (uint32_t a = i + 1; a < e; a++) {
                const uint64_t k = src[a];
                uint32_t b = a;
                while (b > i && src[b - 1] > k) {
                    src[b] = src[b - 1];
                    b--;
                }
                src[b] = k;
            }
        }
        __syncthreads();
        if (!s_long) break;      // block-uniform
        // a long run: sort the tile again over every bit of the range
        for (uint32_t i = threadIdx.x; i < len; i += NTH) bufA[i] = keys[st + i];
        src = bufA;
        dst = bufB;
        lo = 0;
        __syncthreads();
        if (threadIdx.x == 0) s_long = 0;
    }
    for (uint32_t i = threadIdx.x; i < len; i += NTH) vals[st + i] = (uint32_t)src[i];
}

static_assert(sizeof(SortSmem<kSortThreadsL, kSmallCap>) <= 48 * 1024, "static shared memory of k_sort_tiles_l");

// Tiles of at most kSortCapS keys; longer ones are listed (mid) for k_sort_tiles_l.
__global__ void __launch_bounds__(kSortThreadsS)
k_sort_tiles(const uint32_t *__restrict__ ranges, const uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
             uint32_t *__restrict__ mid, uint32_t *__restrict__ nmid)
{
    __shared__ SortSmem<kSortThreadsS, kSortCapS> sm;
    const int64_t t = blockIdx.x;
    const uint32_t st = ranges[2 * t], en = ranges[2 * t + 1];
    const uint32_t len = en - st;
    if (len == 0) return;
    if (len > (uint32_t)kSortCapS) {
        if (threadIdx.x == 0) mid[atomicAdd(nmid, 1u)] = (uint32_t)t;
        return;
    }
    if (len == 1) {
        if (threadIdx.x == 0) vals[st] = (uint32_t)keys[st];
        return;
    }
    sort_tile<kSortThreadsS, kSortCapS>(sm, keys, vals, st, len);
}

// The listed longer tiles (persistent blocks); those above kSmallCap go to k_sort_big.
__global__ void __launch_bounds__(kSortThreadsL)
k_sort_tiles_l(const uint32_t *__restrict__ ranges, const uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
               const uint32_t *__restrict__ mid, const uint32_t *__restrict__ nmid, uint32_t *__restrict__ big,
               uint32_t *__restrict__ nbig)
{
    __shared__ SortSmem<kSortThreadsL, kSmallCap> sm;
    const uint32_t nm = *nmid;
    for (uint32_t mi = blockIdx.x; mi < nm; mi += gridDim.x) {   // block-uniform
        const uint32_t t = mid[mi];
        const uint32_t st = ranges[2 * t], len = ranges[2 * t + 1] - st;
        if (len > (uint32_t)kSmallCap) {
            if (threadIdx.x == 0) big[atomicAdd(nbig, 1u)] = t;
        } else {
            sort_tile<kSortThreadsL, kSmallCap>(sm, keys, vals, st, len);
        }
        __syncthreads();   // the shared buffers are reused by the next tile
    }
}

__global__ void __launch_bounds__(kBigThreads)
k_sort_big(const uint32_t *__restrict__ ranges, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
           const uint32_t *__restrict__ big, const uint32_t *__restrict__ nbig)
{
    extern __shared__ uint64_t sbig[];
    const uint32_t nb = *nbig;
    for (uint32_t bi = blockIdx.x; bi < nb; bi += gridDim.x) {
        const uint32_t t = big[bi];
        const uint32_t st = ranges[2 * t], en = ranges[2 * t + 1];
        const uint32_t len = en - st;
        const uint32_t P = next_pow2(len);
        if (len <= (uint32_t)kBigCap) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) sbig[i] = i < len ? keys[st + i] : kPadKey;
            __syncthreads();
            smem_bitonic(sbig, P);
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) vals[st + i] = (uint32_t)sbig[i];
        } else {
            // in place in global memory; comparators reaching past the list compare
            // against the implicit padding and leave both sides unchanged
            uint64_t *k0 = keys + st;
            const uint32_t lp = 31 - __clz(P);
            for (uint32_t lk = 1; lk <= lp; lk++) {
                for (int ld = (int)lk - 1; ld >= 0; ld--) {
                    const bool flip = (ld == (int)lk - 1);
                    for (uint32_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
                        uint32_t a, b;
                        bitonic_pair(i, lk, (uint32_t)ld, flip, a, b);
                        if (b >= len) continue;
                        uint64_t x = k0[a], y = k0[b];
                        if (y < x) {
                            k0[a] = y;
                            k0[b] = x;
                        }
                    }
                    __syncthreads();
                }
            }
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) vals[st + i] = (uint32_t)k0[i];
        }
        __syncthreads();
    }
}

cudaError_t bin_sort(const float *rec, int64_t n, int V, const Grid &g, void *ws, int64_t capacity,
                     uint32_t *vals, uint32_t *ranges, uint32_t *order, int64_t *n_inst, int32_t *status,
                     int num_sms, cudaStream_t s)
{
    const int64_t Ttot = g.Tv * V;
    BinWs w{};
    const int chunk = chunk_for(n, V, num_sms);
    ws_layout(capacity, Ttot, chunk_count_entries(n, V, g.Tv, chunk), (int64_t)V * n, &w, ws);
    const float4 *r4 = reinterpret_cast<const float4 *>(rec);
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * (2 * (size_t)Ttot + 3), s);
    if (e != cudaSuccess) return e;
    const int64_t slots = (int64_t)V * n;
    const size_t hist_bytes = sizeof(uint32_t) * (size_t)g.Tv;
    const bool agg = hist_bytes <= kAggMaxSmem;
    const size_t agg_smem = kStageBytes + hist_bytes;
    if (agg) {
        e = cudaFuncSetAttribute(k_count_agg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)agg_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_scatter_agg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)agg_smem);
        if (e != cudaSuccess) return e;
    }
    const dim3 agrid((unsigned)((n + chunk - 1) / chunk), (unsigned)V);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((slots + threads - 1) / threads, (int64_t)num_sms * 16);
    if (agg)
        k_count_agg<<<agrid, kAggThreads, agg_smem, s>>>(r4, n, chunk, g, w.count, w.bcount, w.slotrec);
    else
        k_count<<<blocks, threads, 0, s>>>(r4, n, V, g, w.count);
    const int nsb = (int)((Ttot + kScanSpan - 1) / kScanSpan);
    k_scan_part<<<nsb, kScanThreads, 0, s>>>(w.count, Ttot, w.part, w.bhist);
    k_scan_out<<<nsb, kScanThreads, 0, s>>>(w.count, Ttot, capacity, w.part, w.bhist, nsb, ranges, order, n_inst,
                                            w.nbig, status);
    if (agg)
        k_scatter_agg<<<agrid, kAggThreads, agg_smem, s>>>(r4, n, chunk, g, w.count, w.cursor, w.bcount, w.slotrec,
                                                             w.keys, capacity);
    else
        k_scatter<<<blocks, threads, 0, s>>>(r4, n, V, g, w.count, w.cursor, w.keys, capacity);
    k_sort_tiles<<<(unsigned)Ttot, kSortThreadsS, 0, s>>>(ranges, w.keys, vals, w.mid, w.nmid);
    k_sort_tiles_l<<<(unsigned)std::min<int64_t>(Ttot, (int64_t)num_sms * 4), kSortThreadsL, 0, s>>>(
        ranges, w.keys, vals, w.mid, w.nmid, w.big, w.nbig);
    const size_t big_smem = sizeof(uint64_t) * kBigCap;
    e = cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
    if (e != cudaSuccess) return e;
    k_sort_big<<<num_sms, kBigThreads, big_smem, s>>>(ranges, w.keys, vals, w.big, w.nbig);
    return cudaGetLastError();
}

}  // namespace cgs
