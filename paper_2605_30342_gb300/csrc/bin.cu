// bin.cu -- stage B of the two-level binning without a sort: every tile's
// list of a batch, its records in stage-A order (depth, ties by index),
// counted and placed from the records' tile rectangles.
//
// Stage A leaves each view's visible records in depth order.  The
// composites need, per (view, tile), the records whose rectangle covers the
// tile in that order: the lists a stable sort of the records' tile entries
// by tile gives (the per-pixel depth order of the uncertainty and the
// single-view visibility algorithms).  Here each view's records are cut into
// chunks of kBinChunk consecutive records, one warp per chunk:
//   k_bin_chunks   the chunks of every view (a prefix over the views)
//   k_bin_count    per chunk and tile: how many of the chunk's records cover
//                  the tile (shared-memory counters; table rows chunk-major)
//   k_bin_columns  each (view, tile) column of the table becomes the
//                  exclusive prefix over the view's chunks; the column's sum
//                  is the tile's list length
//   an exclusive scan of the lengths in (view, tile) order gives each list's
//   start, k_bin_ranges the composites' ranges
//   k_bin_place    writes each chunk's entries at list start + column prefix
//                  + the number of the chunk's earlier entries for the tile
//                  (a running position per tile in shared memory; within a
//                  round of 32 entries, which the lanes hold in record order,
//                  the rank among equal tiles comes from match_any)
// Within a (chunk, tile) the entries land in record order and the chunks of
// a view follow one another, so every list equals the stable sort's.
#include "gavis_internal.cuh"

namespace gavis {

namespace {

constexpr int kBinWarps = 4;   // warps per CTA of the count and place kernels

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// the view of chunk gc: the largest v < nv with chunk_off[v] <= gc (views
// without records have no chunks: equal neighbouring offsets)
__device__ __forceinline__ int view_of_chunk(const uint32_t *chunk_off, int nv, uint32_t gc)
{
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk_off[mid] <= gc) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The tile entries of records [r0, r1) in stage-A order, 32 per round: the
// warp takes 32 records at a time (a visible record has at least one tile),
// and lane j of a round holds entry j of the records' concatenated
// row-major rectangles.  Its record is the last lane whose first entry is at
// or before j: the lanes that start before the round plus those whose start
// lies in the round at or before j.  next() yields the rounds one by one
// (warp-converged); the payload is recs[r] - vrow of the entry's record.
struct EntryRounds {
    const uint2 *rect_sorted;
    const uint32_t *recs;
    uint32_t r1, TW, vrow, rb;   // rb: first record of the next batch
    int lane;
    unsigned upto;               // lanes 0..lane
    // the current batch (one record per lane) and the prefetched next one
    uint32_t excl, w, first, pay, total, j0;
    float rw;
    uint2 nrc;
    uint32_t npay;

    __device__ __forceinline__ EntryRounds(const uint2 *rs, const uint32_t *rc, uint32_t r0, uint32_t r1_,
                                           uint32_t TW_, uint32_t vrow_, int lane_)
        : rect_sorted(rs), recs(rc), r1(r1_), TW(TW_), vrow(vrow_), rb(r0), lane(lane_),
          upto(0xffffffffu >> (31 - lane_)), excl(0), w(1), first(0), pay(0), total(0), j0(0), rw(1.0f),
          nrc(make_uint2(0u, 0u)), npay(0u)
    {
        if (r0 + (uint32_t)lane < r1) {
            nrc = rect_sorted[r0 + (uint32_t)lane];
            npay = recs[r0 + (uint32_t)lane];
        }
    }

    // the next batch of 32 records: decode the prefetched rectangles, load
    // the following batch's, scan the tile counts
    __device__ __forceinline__ void refill()
    {
        const uint32_t r = rb + (uint32_t)lane;
        const uint2 rc = nrc;
        const uint32_t rpay = npay;
        if (r + 32u < r1) {
            nrc = rect_sorted[r + 32u];
            npay = recs[r + 32u];
        }
        first = 0u;
        w = 1u;
        pay = 0u;
        uint32_t cnt = 0u;
        if (r < r1) {
            const uint32_t x0 = rc.x & 0xffffu, y0 = rc.y & 0xffffu;
            w = (rc.x >> 16) - x0 + 1u;
            cnt = w * ((rc.y >> 16) - y0 + 1u);
            first = y0 * TW + x0;
            pay = rpay - vrow;
        }
        rw = rcp_approx((float)w);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        excl = inc - cnt;   // lanes past r1: excl = total, which no valid j reaches
        total = __shfl_sync(0xffffffffu, inc, 31);
        j0 = 0u;
        rb += 32u;
    }

    // false when the records are exhausted
    __device__ __forceinline__ bool next(bool &valid, uint32_t &t, uint32_t &g)
    {
        if (j0 >= total) {   // warp-uniform
            if (rb >= r1) return false;
            refill();
        }
        const uint32_t j = j0 + (uint32_t)lane;
        const uint32_t before = (uint32_t)__popc(__ballot_sync(0xffffffffu, excl < j0));
        const uint32_t starts =
            __reduce_or_sync(0xffffffffu, (excl >= j0 && excl - j0 < 32u) ? 1u << (excl - j0) : 0u);
        const int k = (int)(before + (uint32_t)__popc(starts & upto)) - 1;
        const uint32_t ek = __shfl_sync(0xffffffffu, excl, k), wk = __shfl_sync(0xffffffffu, w, k);
        const uint32_t fk = __shfl_sync(0xffffffffu, first, k);
        const float rk = __shfl_sync(0xffffffffu, rw, k);
        g = __shfl_sync(0xffffffffu, pay, k);
        // row and column of entry m of the rectangle: m < 2^16 tiles, so
        // m * (1/wk) with the approximate reciprocal (relative error below
        // 2^-21 after the product's rounding) is within one of m / wk, and
        // one correction step each way makes the quotient exact
        const uint32_t m = j - ek;
        uint32_t ty = (uint32_t)((float)m * rk);
        int d = (int)(m - ty * wk);
        if (d < 0) { --ty; d += (int)wk; }
        else if (d >= (int)wk) { ++ty; d -= (int)wk; }
        t = fk + ty * TW + (uint32_t)d;
        valid = j < total;
        j0 += 32u;
        return true;
    }
};

// chunk_off[v] (v = 0..nv) = chunks of the views before v, roff[v] = their
// records (voff clamped to the live records); one warp
__global__ void k_bin_chunks(const uint32_t *voff, int nv, size_t nrec, const unsigned long long *d_nrec,
                             uint32_t *roff, uint32_t *chunk_off)
{
    size_t live = nrec;
    if (d_nrec && (size_t)*d_nrec < live) live = (size_t)*d_nrec;
    const uint32_t lv = (uint32_t)live;
    const int lane = (int)threadIdx.x;
    const int per = (nv + 31) / 32;
    const int a = min(lane * per, nv), b = min(a + per, nv);
    auto rec_off = [&](int v) { return min(voff[v], lv); };
    auto chunks = [&](int v) { return (rec_off(v + 1) - rec_off(v) + (uint32_t)kBinChunk - 1u) / (uint32_t)kBinChunk; };
    uint32_t sum = 0;
    for (int v = a; v < b; ++v) sum += chunks(v);
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    uint32_t run = inc - sum;
    for (int v = a; v < b; ++v) {
        chunk_off[v] = run;
        roff[v] = rec_off(v);
        run += chunks(v);
    }
    if (lane == 31) {
        chunk_off[nv] = inc;
        roff[nv] = rec_off(nv);
    }
}

// table[gc * TT + t] = records of chunk gc whose rectangle covers tile t,
// from the rectangles' corners: +1 at (x0, y0) and (x1 + 1, y1 + 1), -1 at
// (x1 + 1, y0) and (x0, y1 + 1) in a per-warp difference array (modulo 2^32;
// the prefix sums are the counts), then prefix sums along x (a lane per row)
// and along y (a lane per column).  Rows are TW + 1 words apart (column TW
// takes the x1 + 1 = TW corners, which no tile reads; for an even TW the odd
// stride also puts the lanes of the row pass on different banks), and
// corners on row TH are left out (no tile below).
__global__ void __launch_bounds__(kBinWarps * 32) k_bin_count(const uint2 *rect_sorted, const uint32_t *roff,
                                                              const uint32_t *chunk_off, int nv, int TW, int TH,
                                                              uint32_t *table)
{
    extern __shared__ uint32_t s_bin[];
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    const uint32_t gc = blockIdx.x * kBinWarps + (uint32_t)warp;
    if (gc >= chunk_off[nv]) return;   // the whole warp
    const int v = view_of_chunk(chunk_off, nv, gc);
    const uint32_t r0 = roff[v] + (gc - chunk_off[v]) * (uint32_t)kBinChunk;
    const uint32_t r1 = min(r0 + (uint32_t)kBinChunk, roff[v + 1]);
    const int RS = TW + 1;   // row stride of the difference array
    uint32_t *D = s_bin + (size_t)warp * (size_t)(RS * TH);
    for (int i = lane; i < RS * TH; i += 32) D[i] = 0u;
    __syncwarp();
    for (uint32_t r = r0 + (uint32_t)lane; r < r1; r += 32) {
        const uint2 rc = rect_sorted[r];
        const int x0 = (int)(rc.x & 0xffffu), x1 = (int)(rc.x >> 16) + 1;
        const int y0 = (int)(rc.y & 0xffffu), y1 = (int)(rc.y >> 16) + 1;
        atomicAdd(&D[y0 * RS + x0], 1u);
        atomicAdd(&D[y0 * RS + x1], 0xffffffffu);
        if (y1 < TH) {
            atomicAdd(&D[y1 * RS + x0], 0xffffffffu);
            atomicAdd(&D[y1 * RS + x1], 1u);
        }
    }
    __syncwarp();
    for (int y = lane; y < TH; y += 32) {   // along x
        uint32_t run = 0u;
        uint32_t *row = D + y * RS;
        for (int x = 0; x < TW; ++x) {
            run += row[x];
            row[x] = run;
        }
    }
    __syncwarp();
    for (int x = lane; x < TW; x += 32) {   // along y
        uint32_t run = 0u;
        for (int y = 0; y < TH; ++y) {
            run += D[y * RS + x];
            D[y * RS + x] = run;
        }
    }
    __syncwarp();
    uint32_t *out = table + (size_t)gc * (size_t)(TW * TH);
    for (int y = 0; y < TH; ++y)
        for (int x = lane; x < TW; x += 32) out[y * TW + x] = D[y * RS + x];
}

// per (view, tile): the column of the view's chunks becomes its exclusive
// prefix, in place; tile_tot = the column's sum.  A CTA takes 32 tiles of a
// view (a lane each) and its kColWarps warps split the view's chunks into
// consecutive segments: each warp sums its segment, the segment sums are
// prefixed across the warps in shared memory, and each warp rewrites its
// segment from its offset.  A thread keeps kBinColBatch loads in flight
// before the stores (a store may alias a later load as far as the compiler
// knows).
constexpr int kColWarps = 8;
constexpr int kBinColBatch = 8;
__global__ void __launch_bounds__(kColWarps * 32) k_bin_columns(uint32_t *table, const uint32_t *chunk_off, int TT,
                                                               uint32_t *tile_tot)
{
    __shared__ uint32_t s_part[kColWarps][32];
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    const int t = (int)blockIdx.x * 32 + lane;
    const int v = (int)blockIdx.y;
    const uint32_t c0 = chunk_off[v], c1 = chunk_off[v + 1];
    const uint32_t per = (c1 - c0 + kColWarps - 1) / kColWarps;
    const uint32_t s0 = min(c0 + (uint32_t)warp * per, c1), s1 = min(s0 + per, c1);
    const size_t st = (size_t)TT;
    const bool live = t < TT;
    uint32_t sum = 0u;
    if (live) {
        const uint32_t *p = table + (size_t)s0 * st + (size_t)t;
        for (uint32_t c = s0; c < s1; c += kBinColBatch, p += kBinColBatch * st) {
            const uint32_t k = s1 - c < (uint32_t)kBinColBatch ? s1 - c : (uint32_t)kBinColBatch;
#pragma unroll
            for (int i = 0; i < kBinColBatch; ++i) sum += (uint32_t)i < k ? p[i * st] : 0u;
        }
    }
    s_part[warp][lane] = sum;
    __syncthreads();
    uint32_t run = 0u, tot = 0u;
#pragma unroll
    for (int w = 0; w < kColWarps; ++w) {
        const uint32_t x = s_part[w][lane];
        if (w < warp) run += x;
        tot += x;
    }
    if (!live) return;
    if (warp == 0) tile_tot[(size_t)v * st + (size_t)t] = tot;
    uint32_t *p = table + (size_t)s0 * st + (size_t)t;
    for (uint32_t c = s0; c < s1; c += kBinColBatch, p += kBinColBatch * st) {
        const uint32_t k = s1 - c < (uint32_t)kBinColBatch ? s1 - c : (uint32_t)kBinColBatch;
        uint32_t x[kBinColBatch];
#pragma unroll
        for (int i = 0; i < kBinColBatch; ++i) x[i] = (uint32_t)i < k ? p[i * st] : 0u;
#pragma unroll
        for (int i = 0; i < kBinColBatch; ++i) {
            if ((uint32_t)i < k) p[i * st] = run;
            run += x[i];
        }
    }
}

// ranges of the lists, cut off at the entry capacity (entries past it are
// not written); an empty list is (0, 0), as the sorted path leaves it
__global__ void k_bin_ranges(const uint32_t *start, const uint32_t *tot, size_t nvt, size_t cap_M, uint2 *ranges)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvt) return;
    const uint32_t len = tot[i];
    const size_t s = len ? start[i] : 0u, e = s + len;
    ranges[i] = make_uint2((uint32_t)(s < cap_M ? s : cap_M), (uint32_t)(e < cap_M ? e : cap_M));
}

// vals[p] = Gaussian index of each tile entry at its list position p: the
// warp's running positions per tile start at list start + column prefix
__global__ void __launch_bounds__(kBinWarps * 32) k_bin_place(const uint2 *rect_sorted, const uint32_t *recs,
                                                              const uint32_t *roff, const uint32_t *chunk_off, int nv,
                                                              int64_t n, int TW, int TT, const uint32_t *table,
                                                              const uint32_t *tile_start, uint32_t *vals,
                                                              size_t cap_M, uint32_t *overflow)
{
    extern __shared__ uint32_t s_bin[];
    const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
    const uint32_t gc = blockIdx.x * kBinWarps + (uint32_t)warp;
    if (gc >= chunk_off[nv]) return;   // the whole warp
    const int v = view_of_chunk(chunk_off, nv, gc);
    const uint32_t r0 = roff[v] + (gc - chunk_off[v]) * (uint32_t)kBinChunk;
    const uint32_t r1 = min(r0 + (uint32_t)kBinChunk, roff[v + 1]);
    uint32_t *pos_t = s_bin + (size_t)warp * (size_t)TT;
    const uint32_t *row = table + (size_t)gc * (size_t)TT;
    const uint32_t *st = tile_start + (size_t)v * (size_t)TT;
    // eight of the lane's tiles per step, their loads in flight together
    for (int t0 = 0; t0 < TT; t0 += 8 * 32) {
        uint32_t a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int t = t0 + i * 32 + lane;
            a[i] = t < TT ? st[t] : 0u;
            b[i] = t < TT ? row[t] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int t = t0 + i * 32 + lane;
            if (t < TT) pos_t[t] = a[i] + b[i];
        }
    }
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    bool over = false;
    EntryRounds er(rect_sorted, recs, r0, r1, (uint32_t)TW, (uint32_t)v * (uint32_t)n, lane);
    bool valid = false;
    uint32_t t = 0u, g = 0u;
    while (er.next(valid, t, g)) {
        // tiles are below TT, so the empty lanes' all-ones key matches no entry
        const unsigned peers = __match_any_sync(0xffffffffu, valid ? t : 0xffffffffu);
        uint32_t p = 0u;
        if (valid) p = pos_t[t] + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (valid && (peers >> lane) == 1u) pos_t[t] = p + 1u;   // the last of the peers moves the tile on
        __syncwarp();
        if (valid) {
            if ((size_t)p < cap_M) vals[p] = g;
            else over = true;
        }
    }
    if (over && overflow) *overflow = 1u;
}

// canonical keys ((view * TT + tile) << 32) | depth bits from the lists
__global__ void k_keys_from_ranges(const uint2 *ranges, const uint32_t *vals, size_t nvt, int TT, const GeoRec *geo,
                                   int64_t n, size_t cap, uint64_t *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvt) return;
    const uint2 rg = ranges[i];
    const size_t vrow = (i / (size_t)TT) * (size_t)n;
    for (uint32_t e = rg.x; e < rg.y && (size_t)e < cap; ++e)
        out[e] = ((uint64_t)i << 32) | (uint64_t)__float_as_uint(geo[vrow + vals[e]].b.z);
}

unsigned nblk(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

size_t place_smem(int TT) { return (size_t)kBinWarps * (size_t)TT * sizeof(uint32_t); }
size_t count_smem(int TW, int TH) { return (size_t)kBinWarps * (size_t)((TW + 1) * TH) * sizeof(uint32_t); }
size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t bin_chunks_max(size_t cap_R, int nv) { return (cap_R + kBinChunk - 1) / kBinChunk + (size_t)nv; }

BinLayout bin_layout(void *base, size_t cap_R, int nv, int TT)
{
    BinLayout L;
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t b) { char *q = p ? p + off : nullptr; off += a256(b ? b : 1); return q; };
    const size_t nvt = (size_t)nv * (size_t)TT;
    L.roff = reinterpret_cast<uint32_t *>(take(((size_t)nv + 1) * 4));
    L.chunk_off = reinterpret_cast<uint32_t *>(take(((size_t)nv + 1) * 4));
    L.table = reinterpret_cast<uint32_t *>(take(bin_chunks_max(cap_R, nv) * (size_t)TT * 4));
    L.tile_tot = reinterpret_cast<uint32_t *>(take(nvt * 4));
    L.tile_start = reinterpret_cast<uint32_t *>(take(nvt * 4));
    L.scan_tmp = take(scan_tmp_bytes(nvt) + 64);
    L.bytes = off;
    return L;
}

void bin_prepare()
{
    static bool done = false;
    if (done) return;
    const int most = (int)place_smem(kBinMaxTiles);
    cudaFuncSetAttribute(k_bin_place, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    // (TW + 1) TH <= 2 TT words for TW >= 1
    cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * most);
    done = true;
}

cudaError_t launch_bin_tiles(const uint32_t *recs, const uint2 *rect_sorted, const uint32_t *voff, int nv, int64_t n,
                             int TW, int TT, size_t cap_R, const unsigned long long *d_nrec, const BinLayout &B,
                             uint2 *ranges, uint32_t *vals, size_t cap_M, uint32_t *overflow, cudaStream_t s)
{
    if (nv < 1 || TT < 1 || TT > kBinMaxTiles || nv > kMaxBatchViews || TW < 1 || TT % TW != 0)
        return cudaErrorInvalidValue;
    bin_prepare();
    const size_t nvt = (size_t)nv * (size_t)TT;
    const unsigned grid = nblk(bin_chunks_max(cap_R, nv), kBinWarps);
    k_bin_chunks<<<1, 32, 0, s>>>(voff, nv, cap_R, d_nrec, B.roff, B.chunk_off);
    count_launch();
    const int TH = TT / TW;
    k_bin_count<<<grid, kBinWarps * 32, count_smem(TW, TH), s>>>(rect_sorted, B.roff, B.chunk_off, nv, TW,
                                                                 TH, B.table);
    count_launch();
    k_bin_columns<<<dim3(nblk((size_t)TT, 32), (unsigned)nv), kColWarps * 32, 0, s>>>(B.table, B.chunk_off, TT,
                                                                                   B.tile_tot);
    count_launch();
    cudaError_t e = exclusive_scan_u32(B.tile_tot, B.tile_start, nvt, B.scan_tmp, nullptr, s);
    if (e != cudaSuccess) return e;
    k_bin_ranges<<<nblk(nvt, 256), 256, 0, s>>>(B.tile_start, B.tile_tot, nvt, cap_M, ranges);
    count_launch();
    k_bin_place<<<grid, kBinWarps * 32, place_smem(TT), s>>>(rect_sorted, recs, B.roff, B.chunk_off, nv, n, TW, TT,
                                                            B.table, B.tile_start, vals, cap_M, overflow);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_keys_from_ranges(const uint2 *ranges, const uint32_t *vals, int nv, int TT, const GeoRec *geo,
                                    int64_t n, size_t cap, uint64_t *out, cudaStream_t s)
{
    const size_t nvt = (size_t)nv * (size_t)TT;
    if (nvt == 0) return cudaSuccess;
    k_keys_from_ranges<<<nblk(nvt, 256), 256, 0, s>>>(ranges, vals, nvt, TT, geo, n, cap, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace gavis
