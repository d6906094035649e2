// Tile binning of the window's projected splats (one shared sort for all views).
//
// The blending order of Eq. 1 (Sec. III-B, CaRtGS) is depth order within each
// tile.  Instead of a global LSD radix sort over 64-bit (tile, depth) keys, which
// reads and writes every instance once per digit pass, the sort here is
// most-significant-digit first with the tile id as one full-width digit:
//   1. k_count_agg   : per (4096-slot chunk, tile) instance counts in shared memory; a
//                      slot is counted in the tiles of its rect its alpha >= 1/255 ellipse
//                      reaches (reach_box), and a slot with at most 64 rect tiles keeps
//                      the decisions as a bit mask for step 3
//   2. k_scan        : exclusive scan -> tile ranges (the digit's bucket offsets)
//   3. k_scatter_agg : every instance is written once into its tile's bucket as the
//                      64-bit key (depth bits << 32 | slot), in one reserved run per
//                      (chunk, tile); the order inside a bucket is arbitrary
//   4. k_sort_*      : each bucket is sorted in shared memory.  The keys within a tile
//                      are unique (a slot appears once per tile), so the result is one
//                      well-defined order, (depth, slot) ascending, whatever order the
//                      scatter produced.  Depth is positive, so its IEEE bits order
//                      like its values.
// Buckets longer than kSmallCap go to a second kernel with a larger shared-memory
// buffer; buckets beyond that are sorted in place in global memory by one block.  When a
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
// Slots of a view per block of the count and scatter passes: 8192 measured 1% faster on the
// 16-view window but 9% slower for one view at a time (half the blocks).
constexpr int kChunk = 4096;

struct BinWs {
    uint32_t *count;     // [Ttot + 1]
    uint32_t *cursor;    // [Ttot]
    uint32_t *nbig;      // [1]
    uint32_t *big;       // [Ttot]
    uint32_t *bcount;    // [chunks x Ttot]: per (slot chunk, tile) instance counts
    uint64_t *masks;     // [V n]: per slot, the tiles of its rect that passed the reach test
    uint64_t *keys;      // [capacity]
};

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Sections: counters (one memset), big-tile list, per-chunk counts and per-slot tile
// masks (shared-memory path only), keys.
static size_t ws_layout(int64_t capacity, int64_t Ttot, int64_t chunk_counts, int64_t slots, BinWs *w, void *base)
{
    size_t head = align256(sizeof(uint32_t) * (2 * (size_t)Ttot + 2));
    size_t bigb = align256(sizeof(uint32_t) * (size_t)Ttot);
    size_t chb = align256(sizeof(uint32_t) * (size_t)chunk_counts);
    size_t mkb = chunk_counts > 0 ? align256(sizeof(uint64_t) * (size_t)slots) : 0;
    size_t keyb = align256(sizeof(uint64_t) * (size_t)(capacity > 0 ? capacity : 1));
    if (w && base) {
        char *b = static_cast<char *>(base);
        w->count = reinterpret_cast<uint32_t *>(b);
        w->cursor = w->count + Ttot + 1;
        w->nbig = w->cursor + Ttot;
        w->big = reinterpret_cast<uint32_t *>(b + head);
        w->bcount = reinterpret_cast<uint32_t *>(b + head + bigb);
        w->masks = reinterpret_cast<uint64_t *>(b + head + bigb + chb);
        w->keys = reinterpret_cast<uint64_t *>(b + head + bigb + chb + mkb);
    }
    return head + bigb + chb + mkb + keyb;
}

// Per-(chunk, tile) counts kept between the count and scatter passes when a view's tile
// histogram fits in shared memory.
static int64_t chunk_count_entries(int64_t n, int64_t V, int64_t Tv)
{
    if (sizeof(uint32_t) * (size_t)Tv > kAggMaxSmem) return 0;
    return (n + kChunk - 1) / kChunk * V * Tv;
}

size_t bin_ws_bytes(int64_t capacity, int64_t n, int64_t V, int64_t Tv)
{
    return ws_layout(capacity, Tv * V, chunk_count_entries(n, V, Tv), V * n, nullptr, nullptr);
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
// memory: block (c, v) owns slots [c*kChunk, (c+1)*kChunk) of view v, counts its
// instances per tile in shared memory and touches each global counter once.
constexpr int kAggThreads = 512;

// Calls f(tile in view, key) for every tile of the rectangles of the visible slots [s0, s1)
// of a view that the slot can reach (in_tile), row by row, load-balanced over the lanes of
// each warp: a warp takes the next group of 32 slots from the shared counter `next`
// (groups differ widely in work), forms the prefix sum of their row counts, and hands out
// rows round-robin; a lane finds the slot owning row j by a 5-step binary search over the
// prefix (shuffles).
// Tile masks: a slot whose rect has at most 64 tiles keeps one bit per tile (row-major over
// the rect) saying whether it passed the reach test.  The count pass (RECORD) sets them
// (wm: this warp's 32 shared words) and stores them per slot; the scatter pass (!RECORD)
// reads them back instead of testing again, and tests only the slots with larger rects.
constexpr int kMaskTiles = 64;

template <bool RECORD, class F>
__device__ __forceinline__ void for_each_tile_row(const float4 *__restrict__ rec, int64_t n, int view, int64_t s0,
                                                  int64_t s1, const Grid &g, uint32_t *next,
                                                  unsigned long long *wm, uint64_t *__restrict__ masks, F f)
{
    const int lane = threadIdx.x & 31;
    // warps take 32-slot groups from a shared counter (groups differ in work)
    for (;;) {
        uint32_t grp = 0;
        if (lane == 0) grp = atomicAdd(next, 1u);
        grp = __shfl_sync(kFull, grp, 0);
        const int64_t wb = s0 + 32 * (int64_t)grp;
        if (wb >= s1) break;
        const int64_t gi = wb + lane;
        int h = 0, x0 = 0, x1 = 0, y0 = 0;
        uint32_t zb = 0;
        float u = 0.f, v = 0.f, z;
        ReachPre e{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
        int r;
        if (gi < s1 && load_slot(rec, (int64_t)view * n + gi, u, v, z, r)) {
            const Rect R = tile_rect(u, v, r, g);
            if (R.x1 > R.x0 && R.y1 > R.y0) {
                h = R.y1 - R.y0;
                x0 = R.x0;
                x1 = R.x1;
                y0 = R.y0;
                zb = __float_as_uint(z);
                e = load_reach(rec, (int64_t)view * n + gi, g);
            }
        }
        const bool small = h * (x1 - x0) <= kMaskTiles;
        unsigned long long mk = 0ull;
        if (RECORD) {
            wm[lane] = 0ull;
            __syncwarp();
        } else if (gi < s1 && h > 0 && small) {
            mk = masks[(int64_t)view * n + gi];
        }
        int incl = h;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        for (int r0 = 0; r0 < total; r0 += 32) {
            const int j = r0 + lane;
            int L = 0;   // owner: the number of lanes whose inclusive prefix is <= j
#pragma unroll
            for (int b = 16; b > 0; b >>= 1)
                if (__shfl_sync(kFull, incl, L + b - 1) <= j) L += b;
            const int oend = __shfl_sync(kFull, incl, L), oh = __shfl_sync(kFull, h, L);
            const int ox0 = __shfl_sync(kFull, x0, L), ox1 = __shfl_sync(kFull, x1, L);
            const int oy0 = __shfl_sync(kFull, y0, L);
            const uint32_t ozb = __shfl_sync(kFull, zb, L);
            const float ou = __shfl_sync(kFull, u, L), ov = __shfl_sync(kFull, v, L);
            const bool osmall = __shfl_sync(kFull, small, L);
            const unsigned long long omk = RECORD ? 0ull : __shfl_sync(kFull, mk, L);
            const bool test = j < total && (RECORD || !osmall);
            ReachPre oe{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
            if (__any_sync(kFull, test))
                oe = ReachPre{__shfl_sync(kFull, e.A, L),  __shfl_sync(kFull, e.B2, L), __shfl_sync(kFull, e.C, L),
                              __shfl_sync(kFull, e.t2, L), __shfl_sync(kFull, e.ex, L), __shfl_sync(kFull, e.ey, L),
                              __shfl_sync(kFull, e.bc, L), __shfl_sync(kFull, e.ba, L), __shfl_sync(kFull, e.mode, L)};
            if (j < total) {
                const uint32_t slot = (uint32_t)((int64_t)view * n + wb + L);
                const uint64_t key = ((uint64_t)ozb << 32) | (uint64_t)slot;
                const int row = j - (oend - oh), ty = oy0 + row, ow = ox1 - ox0;
                if (!RECORD && osmall) {
                    // the count pass's decisions for this row
                    unsigned long long bits = (omk >> (row * ow)) & (ow >= 64 ? ~0ull : ((1ull << ow) - 1ull));
                    while (bits) {
                        const int b = __ffsll((long long)bits) - 1;
                        bits &= bits - 1ull;
                        f(ty * g.Tx + ox0 + b, key);
                    }
                } else {
                    unsigned long long rowbits = 0ull;
                    for (int tx = ox0; tx < ox1; tx++)
                        if (in_tile(oe, ou, ov, tx, ty, g)) {
                            f(ty * g.Tx + tx, key);
                            if (RECORD && osmall) rowbits |= 1ull << (tx - ox0);   // tx - ox0 < 64
                        }
                    if (RECORD && osmall && rowbits) atomicOr(&wm[L], rowbits << (row * ow));
                }
            }
        }
        if (RECORD) {
            __syncwarp();
            if (gi < s1 && h > 0 && small) masks[(int64_t)view * n + gi] = wm[lane];
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kAggThreads)
k_count_agg(const float4 *__restrict__ rec, int64_t n, Grid g, uint32_t *__restrict__ count,
            uint32_t *__restrict__ bcount, uint64_t *__restrict__ masks)
{
    __shared__ unsigned long long wmask[kAggThreads / 32][32];
    extern __shared__ uint32_t hist[];
    const int view = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * kChunk;
    const int64_t s1 = min(n, s0 + kChunk);
    __shared__ uint32_t next;
    for (int t = threadIdx.x; t < g.Tv; t += blockDim.x) hist[t] = 0;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    for_each_tile_row<true>(rec, n, view, s0, s1, g, &next, wmask[threadIdx.x >> 5], masks,
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

// Single-block exclusive scan of the per-tile counts; writes ranges (clamped to the
// capacity), the total instance count and the capacity status.  Each of the 32 warps
// owns a contiguous chunk and walks it 32 entries at a time (coalesced loads, warp
// shuffle scans); a first pass forms the chunk totals.
__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x += y;
    }
    return x;
}

__global__ void __launch_bounds__(1024)
k_scan(uint32_t *__restrict__ count, int64_t Ttot, int64_t capacity, uint32_t *__restrict__ ranges,
       int64_t *__restrict__ n_inst, int32_t *__restrict__ status)
{
    __shared__ unsigned long long wtot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (Ttot + 31) / 32;
    const int64_t lo = (int64_t)w * per, hi = min(Ttot, lo + per);
    unsigned long long s = 0;
    for (int64_t t = lo + lane; t < hi; t += 32) s += count[t];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if (lane == 0) wtot[w] = s;
    __syncthreads();
    unsigned long long run = 0, total = 0;
    for (int i = 0; i < 32; i++) {
        run += (i < w) ? wtot[i] : 0ull;
        total += wtot[i];
    }
    const unsigned long long cap = (unsigned long long)capacity;
    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t t = base + lane;
        const unsigned long long c = t < hi ? count[t] : 0ull;
        const unsigned long long incl = warp_incl_scan(c);
        const unsigned long long st = run + incl - c, en = run + incl;
        if (t < hi) {
            count[t] = (uint32_t)min(st, cap);      // bucket start (clamped) for the scatter
            ranges[2 * t] = (uint32_t)min(st, cap);
            ranges[2 * t + 1] = (uint32_t)min(en, cap);
        }
        run += __shfl_sync(kFull, incl, 31);
    }
    if (threadIdx.x == 0) {
        *n_inst = (int64_t)total;
        count[Ttot] = (uint32_t)min(total, cap);
        if (total > cap) set_status(status, CGS_ERR_CAPACITY);
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
__global__ void __launch_bounds__(kAggThreads)
k_scatter_agg(const float4 *__restrict__ rec, int64_t n, Grid g, const uint32_t *__restrict__ start,
              uint32_t *__restrict__ cursor, const uint32_t *__restrict__ bcount, uint64_t *__restrict__ masks,
              uint64_t *__restrict__ keys, int64_t capacity)
{
    extern __shared__ uint32_t hist[];     // [Tv] counts, then run positions
    const int view = blockIdx.y;
    const int64_t s0 = (int64_t)blockIdx.x * kChunk;
    const int64_t s1 = min(n, s0 + kChunk);
    // this chunk's per-tile counts (from the count pass): reserve one run per tile
    const int64_t tbase = (int64_t)view * g.Tv;
    const uint32_t *mine = bcount + ((int64_t)view * gridDim.x + blockIdx.x) * g.Tv;
    __shared__ uint32_t next;
    if (threadIdx.x == 0) next = 0;
    for (int t = threadIdx.x; t < g.Tv; t += blockDim.x) {
        const uint32_t c = mine[t];
        hist[t] = c ? start[tbase + t] + atomicAdd(cursor + tbase + t, c) : 0u;
    }
    __syncthreads();
    for_each_tile_row<false>(rec, n, view, s0, s1, g, &next, nullptr, masks, [&](int t, uint64_t key) {
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

// Per-tile stable LSD radix sort in shared memory (lists of up to kSmallCap keys).
// The key is (depth bits << 32 | slot) and is unique in a tile, so sorting by the depth
// bits (8-bit digits; a pass whose digit is the same for every key of the tile is
// skipped) and then ordering each run of equal depths by slot gives exactly the
// (depth, slot) order.  Stability: warp w owns a contiguous segment of the list and
// walks it 32 keys at a time; a ballot multisplit ranks equal digits within a step, and
// per-warp digit histograms scanned digit-major give each (digit, warp) its start.
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kTieRun = 32;   // longest run of equal 16-bit depth prefixes fixed by insertion

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

__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t x, uint32_t *wsum)
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

__global__ void __launch_bounds__(kRsThreads)
k_sort_tiles(const uint32_t *__restrict__ ranges, const uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
             uint32_t *__restrict__ big, uint32_t *__restrict__ nbig)
{
    __shared__ uint64_t bufA[kSmallCap], bufB[kSmallCap];
    __shared__ uint32_t hist[kRsWarps][256];
    __shared__ uint16_t lrank[kSmallCap];
    __shared__ uint32_t wsum[kRsWarps], wmin[kRsWarps], wmax[kRsWarps];
    __shared__ int s_long;   // a run of equal 16-bit prefixes longer than kTieRun
    const int64_t t = blockIdx.x;
    const uint32_t st = ranges[2 * t], en = ranges[2 * t + 1];
    const uint32_t len = en - st;
    if (len == 0) return;
    if (len > (uint32_t)kSmallCap) {
        if (threadIdx.x == 0) big[atomicAdd(nbig, 1u)] = (uint32_t)t;
        return;
    }
    if (len == 1) {
        if (threadIdx.x == 0) vals[st] = (uint32_t)keys[st];
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // load, and find the range of the depth bits over the tile (positive floats: the bits
    // order like the values)
    uint32_t dmin = ~0u, dmax = 0u;
    for (uint32_t i = threadIdx.x; i < len; i += kRsThreads) {
        const uint64_t k = keys[st + i];
        bufA[i] = k;
        const uint32_t d = (uint32_t)(k >> 32);
        dmin = min(dmin, d);
        dmax = max(dmax, d);
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
    __syncthreads();
    dmin = ~0u;
    dmax = 0u;
    for (int i = 0; i < kRsWarps; i++) {
        dmin = min(dmin, wmin[i]);
        dmax = max(dmax, wmax[i]);
    }
    uint64_t *src = bufA, *dst = bufB;
    const uint32_t per = (len + kRsWarps - 1) / kRsWarps;
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
            {   // start of each (digit, warp) run: digit-major exclusive scan
                const uint32_t dg = threadIdx.x;       // 256 threads = 256 digits
                uint32_t cnts[kRsWarps], tot = 0u;
#pragma unroll
                for (int i = 0; i < kRsWarps; i++) {
                    cnts[i] = hist[i][dg];
                    tot += cnts[i];
                }
                uint32_t off = block_excl_scan256(tot, wsum);
#pragma unroll
                for (int i = 0; i < kRsWarps; i++) {
                    hist[i][dg] = off;
                    off += cnts[i];
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
        for (uint32_t i = threadIdx.x; i + 1 < len; i += kRsThreads) {
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
        for (uint32_t i = threadIdx.x; i < len; i += kRsThreads) bufA[i] = keys[st + i];
        src = bufA;
        dst = bufB;
        lo = 0;
        __syncthreads();
        if (threadIdx.x == 0) s_long = 0;
    }
    for (uint32_t i = threadIdx.x; i < len; i += kRsThreads) vals[st + i] = (uint32_t)src[i];
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

// Work order for the raster kernels: tiles by decreasing list length (bucketed by
// floor(log2(len)), longest bucket first; tile order inside a bucket is arbitrary).
__global__ void __launch_bounds__(1024)
k_tile_order(const uint32_t *__restrict__ ranges, int64_t Ttot, uint32_t *__restrict__ order)
{
    __shared__ uint32_t hist[33], offs[33];
    if (threadIdx.x < 33) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < Ttot; t += blockDim.x) {
        uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        uint32_t b = len ? 32 - __clz(len) : 0;     // 0 for empty, 1..32 otherwise
        atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 32; b >= 0; b--) {
            offs[b] = run;
            run += hist[b];
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < Ttot; t += blockDim.x) {
        uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
        uint32_t b = len ? 32 - __clz(len) : 0;
        order[atomicAdd(&offs[b], 1u)] = (uint32_t)t;
    }
}

cudaError_t bin_sort(const float *rec, int64_t n, int V, const Grid &g, void *ws, int64_t capacity,
                     uint32_t *vals, uint32_t *ranges, uint32_t *order, int64_t *n_inst, int32_t *status,
                     int num_sms, cudaStream_t s)
{
    const int64_t Ttot = g.Tv * V;
    BinWs w{};
    ws_layout(capacity, Ttot, chunk_count_entries(n, V, g.Tv), (int64_t)V * n, &w, ws);
    const float4 *r4 = reinterpret_cast<const float4 *>(rec);
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * (2 * (size_t)Ttot + 2), s);
    if (e != cudaSuccess) return e;
    const int64_t slots = (int64_t)V * n;
    const size_t hist_bytes = sizeof(uint32_t) * (size_t)g.Tv;
    const bool agg = hist_bytes <= kAggMaxSmem;
    if (agg) {
        e = cudaFuncSetAttribute(k_count_agg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_scatter_agg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_bytes);
        if (e != cudaSuccess) return e;
    }
    const dim3 agrid((unsigned)((n + kChunk - 1) / kChunk), (unsigned)V);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((slots + threads - 1) / threads, (int64_t)num_sms * 16);
    if (agg)
        k_count_agg<<<agrid, kAggThreads, hist_bytes, s>>>(r4, n, g, w.count, w.bcount, w.masks);
    else
        k_count<<<blocks, threads, 0, s>>>(r4, n, V, g, w.count);
    k_scan<<<1, 1024, 0, s>>>(w.count, Ttot, capacity, ranges, n_inst, status);
    if (agg)
        k_scatter_agg<<<agrid, kAggThreads, hist_bytes, s>>>(r4, n, g, w.count, w.cursor, w.bcount, w.masks,
                                                             w.keys, capacity);
    else
        k_scatter<<<blocks, threads, 0, s>>>(r4, n, V, g, w.count, w.cursor, w.keys, capacity);
    k_sort_tiles<<<(unsigned)Ttot, kRsThreads, 0, s>>>(ranges, w.keys, vals, w.big, w.nbig);
    const size_t big_smem = sizeof(uint64_t) * kBigCap;
    e = cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
    if (e != cudaSuccess) return e;
    k_sort_big<<<num_sms, kBigThreads, big_smem, s>>>(ranges, w.keys, vals, w.big, w.nbig);
    if (order) k_tile_order<<<1, 1024, 0, s>>>(ranges, Ttot, order);
    return cudaGetLastError();
}

}  // namespace cgs
