// sort.cu -- device-wide exclusive scan, stable LSD radix sort of
// (uint32 or uint64 key, uint32 value) pairs, and the stage-A key emission
// from visibility words.
//
// Radix sort: 8-bit digits, one pass per digit over [0, end_bit).  Each pass
// is (1) a per-block digit histogram over a tile of 4096 keys (read as
// 16-byte words), (2) an exclusive scan of the histograms in digit-major
// order, which gives every (digit, block) its output offset, and (3) a
// stable scatter: items are ranked within a warp (lanes with equal digits
// found by __match_any_sync or by per-bit ballots), warps are ordered by a
// shared prefix, rounds of 256 items in input order, so equal digits keep
// their input order; the block's items are placed in shared memory in sorted
// order and written out in digit runs.  Items past a block's end rank as
// digit 255 and are never written.  A segmented sort runs the passes over
// several independent ranges at once (a table of blocks, each within one
// range, and one scan over all their histograms).  Starting from
// index-ascending input this yields the canonical (key, index) order.
#include "gavis_internal.cuh"

namespace gavis {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;   // 8192 elements per block

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// d_n (optional): the actual item count in device memory, <= n (graph
// replays); blocks past it only write a zero partial.
template <bool FLAGS>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *in, size_t n,
                                                              unsigned long long *partials,
                                                              const unsigned long long *d_n)
{
    __shared__ unsigned long long s_warp[32];
    if (d_n && *d_n < n) n = (size_t)*d_n;
    const size_t base = (size_t)blockIdx.x * kScanChunk;
    if (base >= n) {
        if (threadIdx.x == 0) partials[blockIdx.x] = 0ull;
        return;
    }
    unsigned long long v = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        size_t i = base + (size_t)r * kScanThreads + threadIdx.x;
        if (i < n) v += FLAGS ? (in[i] != 0u) : in[i];
    }
    v = block_sum_u64(v, s_warp);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// single block: exclusive scan of nb partials, total -> partials[nb] and *d_total
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(unsigned long long *partials, int nb,
                                                                unsigned long long *d_total)
{
    __shared__ unsigned long long s[kScanThreads];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanThreads) {
        int i = base + threadIdx.x;
        unsigned long long x = i < nb ? partials[i] : 0ull;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < kScanThreads; o <<= 1) {
            unsigned long long y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
            __syncthreads();
            s[threadIdx.x] += y;
            __syncthreads();
        }
        unsigned long long carry = s_carry;
        if (i < nb) partials[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = carry + s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[nb] = s_carry;
        if (d_total) *d_total = s_carry;
    }
}

// self_prefix: partials hold the chunks' plain sums, and each block adds up
// those of the chunks before it (no separate scan of the partials)
template <bool FLAGS>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *in, uint32_t *out, size_t n,
                                                             const unsigned long long *partials,
                                                             const unsigned long long *d_n, bool self_prefix)
{
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_sum[32];
    __shared__ unsigned long long s_pre;
    if (d_n && *d_n < n) n = (size_t)*d_n;
    if ((size_t)blockIdx.x * kScanChunk >= n) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (self_prefix) {
        unsigned long long acc = 0;
        for (unsigned c = threadIdx.x; c < blockIdx.x; c += kScanThreads) acc += partials[c];
        acc = block_sum_u64(acc, s_sum);
        if (threadIdx.x == 0) s_pre = acc;
        __syncthreads();
    }
    const unsigned long long chunk_pre = self_prefix ? s_pre : partials[blockIdx.x];
    const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t x[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        size_t i = base + r;
        x[r] = i < n ? (FLAGS ? (uint32_t)(in[i] != 0u) : in[i]) : 0u;
        sum += x[r];
    }
    // exclusive scan of per-thread sums across the block
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    uint32_t run = (uint32_t)chunk_pre + (warp ? s_warp[warp - 1] : 0u) + inc - sum;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        size_t i = base + r;
        if (i < n) out[i] = run;
        run += x[r];
    }
}

__global__ void k_popc_words(const uint32_t *words, size_t nwords, uint32_t *cnt)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nwords) cnt[i] = (uint32_t)__popc(words[i]);
}

// One thread per visibility word (32 Gaussians of one view); a warp's words
// are consecutive and so are their records, which the warp's lanes write in
// order (coalesced): lane j of a round finds its word by a binary search over
// the warp's prefix popcounts, then its set bit.
// Records at positions >= cap_R are dropped and set *overflow.
template <typename KeyT>
__global__ void k_emit_vis_words(const uint32_t *words, const uint32_t *woff, uint32_t nv, uint32_t nw, uint32_t n,
                                 const GeoRec *geo, const float *zrec, int zb, uint32_t zmin, uint32_t vmask, KeyT *keyA,
                                 uint32_t *valA, uint32_t *voff, size_t cap_R, uint32_t *overflow,
                                 const KeyParams *kp)
{
    if (kp) {   // key parameters computed on the device (graph replays)
        zb = kp->zb;
        zmin = kp->zmin;
        vmask = kp->vmask;
    }
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(threadIdx.x & 31u);
    const uint32_t total_words = nv * nw;
    uint32_t bits = 0, off = 0, v = 0, wi = 0;
    if (w < total_words) {
        v = w / nw;
        wi = w - v * nw;
        bits = words[w];
        off = woff[w];
        if (voff && wi == 0) voff[v] = off;
        if (voff && w == total_words - 1) voff[nv] = off + (uint32_t)__popc(bits);
    }
    const uint32_t cnt = (uint32_t)__popc(bits);
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - cnt;
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t base = __shfl_sync(0xffffffffu, off, 0);   // the valid lanes are a prefix of the warp
    for (uint32_t j0 = 0; j0 < total; j0 += 32) {
        const uint32_t j = j0 + (uint32_t)lane;
        int k = 0;   // last lane whose records start at or before j
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t e = __shfl_sync(0xffffffffu, excl, k + step);
            if (e <= j) k += step;
        }
        const uint32_t ek = __shfl_sync(0xffffffffu, excl, k);
        uint32_t bk = __shfl_sync(0xffffffffu, bits, k);
        const uint32_t vk = __shfl_sync(0xffffffffu, v, k), wik = __shfl_sync(0xffffffffu, wi, k);
        if (j < total) {
            if ((size_t)base + j >= cap_R) {
                if (overflow) *overflow = 1u;
                continue;
            }
            // position of the (j - ek)-th set bit of the word: halve the
            // search range five times by the set bits' counts
            uint32_t m = j - ek, pos = 0;
#pragma unroll
            for (int h = 16; h > 0; h >>= 1) {
                const uint32_t c = (uint32_t)__popc(bk & ((1u << h) - 1u));
                if (m >= c) { m -= c; pos += (uint32_t)h; bk >>= h; }
            }
            const uint32_t r = vk * n + wik * 32u + pos;
            const float z = zrec ? zrec[r] : geo[r].b.z;
            keyA[base + j] = ((KeyT)(vk & vmask) << zb) | (KeyT)(__float_as_uint(z) - zmin);
            valA[base + j] = r;
        }
    }
}

__global__ void k_key_params(const BatchInfo *info, int nv, KeyParams *kp)
{
    if (threadIdx.x != 0) return;
    const unsigned long long vis = info->visible;
    const uint32_t zmin = info->zrange[0];
    const int zb = vis ? depth_bits(zmin, info->zrange[1]) : 0;
    const int vb = bits_of((uint64_t)nv - 1);
    const int gb = vb + zb <= 32 ? vb : 32 - zb;
    KeyParams k;
    k.zmin = vis ? zmin : 0u;
    k.zb = zb;
    k.gsz = 1 << gb;
    k.vmask = (uint32_t)(k.gsz - 1);
    *kp = k;
}

// One block of 1024 threads: the segments' starts and their first blocks in
// shared memory, then every table entry by a binary search over those.
__global__ void __launch_bounds__(1024) k_segment_blocks(const uint32_t *off, int nv, const KeyParams *kp, int gsz,
                                                         uint32_t cap, RsBlock *blk, uint32_t nblk_max)
{
    __shared__ uint32_t s_seg[1025];   // segment starts (clamped to cap); s_seg[nseg] = end of the last
    __shared__ uint32_t s_bst[1025];   // first table block of each segment; s_bst[nseg] = live blocks
    __shared__ uint32_t s_warp[32];
    const int g = kp ? kp->gsz : gsz;
    const int nseg = (nv + g - 1) / g;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int sg = t; sg <= nseg; sg += blockDim.x) {
        const int v = sg * g < nv ? sg * g : nv;
        const uint32_t o = off[v];
        s_seg[sg] = o < cap ? o : cap;
    }
    __syncthreads();
    uint32_t nb = 0;
    if (t < nseg) {
        const uint32_t a = s_seg[t], b = s_seg[t + 1];
        nb = b > a ? (b - a + (uint32_t)kRadixTile - 1) / (uint32_t)kRadixTile : 0u;
    }
    uint32_t x = nb;   // inclusive scan over the block (nseg <= 1024)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t incl = x + (warp ? s_warp[warp - 1] : 0u);
    if (t < nseg) s_bst[t] = incl - nb;
    if (t == (nseg > 0 ? nseg - 1 : 0)) s_bst[nseg] = nseg > 0 ? incl : 0u;
    __syncthreads();
    const uint32_t live = s_bst[nseg];
    for (uint32_t k = (uint32_t)t; k < nblk_max; k += blockDim.x) {
        RsBlock b;
        if (k < live) {
            int lo = 0, hi = nseg - 1;   // the last segment whose first block is <= k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_bst[mid] <= k) lo = mid;
                else hi = mid - 1;
            }
            const uint32_t j = k - s_bst[lo];
            const uint32_t st = s_seg[lo] + j * (uint32_t)kRadixTile;
            const uint32_t en = s_seg[lo + 1];
            b.start = st;
            b.end = st + (uint32_t)kRadixTile < en ? st + (uint32_t)kRadixTile : en;
            b.h0 = 256u * s_bst[lo] + j;
            b.hs = s_bst[lo + 1] - s_bst[lo];
        } else {   // empty: its zero histogram follows the live ones
            b.start = 0u;
            b.end = 0u;
            b.h0 = 256u * k;
            b.hs = 1u;
        }
        blk[k] = b;
    }
}

// record r's first tile entry: its warp's offset (warp_off) plus the tiles
// of the warp's records before it (rect_sorted)
__global__ void k_entry_offsets_dev(const uint32_t *warp_off, const uint2 *rect_sorted, const uint32_t *voff, int nv,
                                    const BatchInfo *info, unsigned long long cap_R, unsigned long long cap_M,
                                    uint32_t *eoff)
{
    const unsigned long long nrec = info->visible < cap_R ? info->visible : cap_R;
    const unsigned long long M = info->total < cap_M ? info->total : cap_M;
    for (int v = threadIdx.x; v <= nv; v += blockDim.x) {
        const uint32_t r = voff[v];
        unsigned long long e = M;
        if (v < nv && (unsigned long long)r < nrec) {
            uint32_t o = warp_off[r >> 5];
            for (uint32_t q = r & ~31u; q < r; ++q) {
                const uint2 rc = rect_sorted[q];
                o += ((rc.x >> 16) - (rc.x & 0xffffu) + 1u) * ((rc.y >> 16) - (rc.y & 0xffffu) + 1u);
            }
            e = o;
        }
        eoff[v] = (uint32_t)(e < M ? e : M);
    }
}

constexpr int kRsThreads = 256;
constexpr int kRsTile = kRadixTile;
constexpr int kRsRounds = kRsTile / kRsThreads;
static_assert(kRsRounds * kRsThreads == kRsTile, "whole rounds of 256 keys per block");
constexpr int kRsWarps = kRsThreads / 32;

// Lanes of the warp holding the same digit d as this lane.  BALLOT builds the
// mask from one ballot per digit bit, which is cheaper than __match_any_sync
// when the 32 digits are mostly distinct (low digits of unsorted keys);
// __match_any_sync wins when they are few (high digits).
template <bool BALLOT>
__device__ __forceinline__ unsigned digit_peers(int d)
{
    if (!BALLOT) return __match_any_sync(0xffffffffu, d);
    unsigned p = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        p &= bit ? bal : ~bal;
    }
    return p;
}

// Per-block digit histogram: warp-private counters with plain shared atomics
// (rounds in which the whole warp holds one digit add 32 once).
// d_n (optional): the actual item count in device memory, <= n (graph replays)
// blk (optional): per-block item ranges and histogram columns of a
// segmented sort (RsBlock); otherwise block b takes items [4096 b, 4096 b +
// 4096) of [0, n) and histogram column b of nblocks.
struct BlockRange {
    size_t base, lim, h0, hs;   // items [base, lim); digit d's count at hist[h0 + d hs]
};
__device__ __forceinline__ BlockRange block_range(const RsBlock *blk, size_t n, int nblocks)
{
    BlockRange b;
    if (blk) {
        const RsBlock r = blk[blockIdx.x];
        b.base = r.start;
        b.lim = r.end;
        b.h0 = r.h0;
        b.hs = r.hs;
    } else {
        b.base = (size_t)blockIdx.x * kRsTile;
        b.lim = b.base + kRsTile < n ? b.base + kRsTile : n;
        b.h0 = blockIdx.x;
        b.hs = (size_t)nblocks;
    }
    return b;
}

template <typename KeyT>
__global__ void __launch_bounds__(kRsThreads) k_radix_hist(const KeyT *keys, size_t n, int shift,
                                                           uint32_t *hist, int nblocks,
                                                           const unsigned long long *d_n, const RsBlock *blk)
{
    if (d_n && *d_n < n) n = (size_t)*d_n;
    __shared__ uint32_t s_h[kRsWarps][257];
    const BlockRange br = block_range(blk, n, nblocks);
    const size_t base = br.base;
    n = br.lim;   // items of this block: [base, lim)
    if (base >= n) {   // whole block past the live items (graph replays)
        hist[br.h0 + (size_t)threadIdx.x * br.hs] = 0u;
        return;
    }
    for (int i = threadIdx.x; i < kRsWarps * 257; i += kRsThreads) (&s_h[0][0])[i] = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    // The block's keys [base, n) are read as the 16-byte words that hold them
    // (key buffers start 16-byte aligned and are padded to 256 bytes, so the
    // word of the last key lies inside the buffer); keys outside are skipped.
    constexpr int E = 16 / (int)sizeof(KeyT);
    const size_t w0 = base / E, w1 = (n + E - 1) / E;
    const uint4 *kw = reinterpret_cast<const uint4 *>(keys);
    constexpr int WR = (kRsTile / E + kRsThreads - 1) / kRsThreads + 1;   // words per thread, at most
#pragma unroll
    for (int r = 0; r < WR; ++r) {
        const size_t w = w0 + (size_t)r * kRsThreads + threadIdx.x;
        if (w < w1) {
            const uint4 q = kw[w];
            KeyT kk[E];
            memcpy(kk, &q, sizeof(q));
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const size_t i = w * E + (size_t)j;
                if (i >= base && i < n) atomicAdd(&s_h[warp][(int)((kk[j] >> shift) & 255u)], 1u);
            }
        }
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) c += s_h[w][threadIdx.x];
    hist[br.h0 + (size_t)threadIdx.x * br.hs] = c;
}

// Stable scatter of one 4096-item tile.  Warp w owns the contiguous items
// [512 w, 512 (w+1)) and ranks them in input order against warp-private digit
// counters (match_any within each 32-item round); the warps' counters are then
// turned into block-local digit offsets, items are placed in shared memory in
// sorted order, and written out so that consecutive threads write consecutive
// addresses of each digit run.
// Each item's digit and rank share one register, so that 32-bit passes fit
// three CTAs per SM (80 registers).
template <typename KeyT>
constexpr size_t rs_smem() { return (size_t)kRsTile * (sizeof(KeyT) + 4) + (size_t)(kRsWarps + 3) * 256 * 4; }

template <typename KeyT, bool BALLOT>
__global__ void __launch_bounds__(kRsThreads, sizeof(KeyT) == 4 ? 3 : 2) k_radix_scatter(const KeyT *kin, const uint32_t *vin,
                                                              KeyT *kout, uint32_t *vout, size_t n, int shift,
                                                              const uint32_t *hist, const uint32_t *offs,
                                                              int nblocks, const unsigned long long *d_n,
                                                              const RsBlock *blk)
{
    if (d_n && *d_n < n) n = (size_t)*d_n;
    const BlockRange br = block_range(blk, n, nblocks);
    n = br.lim;   // items of this block: [base, lim)
    if (br.base >= n) return;   // nothing of this block is live
    extern __shared__ __align__(16) unsigned char smem[];
    KeyT *s_key = reinterpret_cast<KeyT *>(smem);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(smem + (size_t)kRsTile * sizeof(KeyT));
    uint32_t *s_wc = reinterpret_cast<uint32_t *>(smem + (size_t)kRsTile * (sizeof(KeyT) + 4));   // [warps][256]
    uint32_t *s_goff = s_wc + kRsWarps * 256;
    uint32_t *s_lstart = s_goff + 256;
    uint32_t *s_tmp = s_lstart + 256;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const size_t base = br.base;

    // this block's digit counts -> block-local digit starts (exclusive scan)
    const uint32_t mycnt = hist[br.h0 + (size_t)tid * br.hs];
    s_goff[tid] = offs[br.h0 + (size_t)tid * br.hs];
    for (int w = 0; w < kRsWarps; ++w) s_wc[w * 256 + tid] = 0u;
    {
        uint32_t x = mycnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_tmp[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_tmp[w];
        s_lstart[tid] = wpre + x - mycnt;
        s_goff[tid] -= wpre + x - mycnt;   // global start minus block-local start (mod 2^32)
    }

    // phase A: warp-private stable ranks
    constexpr int R = kRsTile / kRsThreads;   // rounds of 32 items per warp
    KeyT k[R];
    uint32_t v[R];
    uint32_t dr[R];   // (digit << 16) | rank in the warp's digit run (ranks < 4096)
    uint32_t *wc = s_wc + warp * 256;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const size_t i = base + (size_t)warp * (32 * R) + (size_t)r * 32 + lane;
        const bool valid = i < n;
        k[r] = valid ? kin[i] : (KeyT)0;
        v[r] = valid ? vin[i] : 0u;
        // an item past the block's end ranks as digit 255: it follows every
        // valid item of the block, so it lands past the valid ones and is not written
        dr[r] = (valid ? (uint32_t)((k[r] >> shift) & 255u) : 255u) << 16;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int d = (int)(dr[r] >> 16);
        const unsigned peers = digit_peers<BALLOT>(d);
        const uint32_t prior = wc[d];
        dr[r] |= prior + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (lane == __ffs(peers) - 1) wc[d] = prior + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps' runs inside the block's digit run
    {
        uint32_t run = s_lstart[tid];
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t c = s_wc[w * 256 + tid];
            s_wc[w * 256 + tid] = run;
            run += c;
        }
    }
    __syncthreads();
    // phase B: place in shared memory in sorted order
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t lp = wc[dr[r] >> 16] + (dr[r] & 0xffffu);
        s_key[lp] = k[r];
        s_val[lp] = v[r];
    }
    __syncthreads();
    // phase C: coalesced write-out
    const int cnt = base < n ? (int)min((size_t)kRsTile, n - base) : 0;
    for (int i = tid; i < cnt; i += kRsThreads) {
        const KeyT kk = s_key[i];
        const int dd = (int)((kk >> shift) & 255u);
        const uint32_t pos = s_goff[dd] + (uint32_t)i;
        kout[pos] = kk;
        vout[pos] = s_val[i];
    }
}

}  // namespace

size_t scan_tmp_bytes(size_t n)
{
    size_t nb = (n + kScanChunk - 1) / kScanChunk;
    return (nb + 1) * sizeof(unsigned long long);
}

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, void *tmp,
                               unsigned long long *d_total, cudaStream_t s, bool flags,
                               const unsigned long long *d_n)
{
    const size_t nb = (n + kScanChunk - 1) / kScanChunk;
    unsigned long long *partials = reinterpret_cast<unsigned long long *>(tmp);
    if (n == 0) {
        if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), s);
        return cudaSuccess;
    }
    if (flags) {
        k_scan_reduce<true><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, partials, d_n); count_launch();
    } else {
        k_scan_reduce<false><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, partials, d_n); count_launch();
    }
    // a requested total takes the separate scan of the partials; otherwise
    // each apply block sums the partials before it
    const bool self_prefix = d_total == nullptr;
    if (!self_prefix) {
        k_scan_partials<<<1, kScanThreads, 0, s>>>(partials, (int)nb, d_total); count_launch();
    }
    if (flags) {
        k_scan_apply<true><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, partials, d_n, self_prefix);
    } else {
        k_scan_apply<false><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, partials, d_n, self_prefix);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t scan_vis_words(const uint32_t *words, size_t nwords, uint32_t *woff, void *tmp, cudaStream_t s)
{
    if (nwords == 0) return cudaSuccess;
    k_popc_words<<<(unsigned)((nwords + 255) / 256), 256, 0, s>>>(words, nwords, woff); count_launch();
    return exclusive_scan_u32(woff, woff, nwords, tmp, nullptr, s);
}

cudaError_t emit_vis_words(const uint32_t *words, const uint32_t *woff, int nv, int64_t n, const GeoRec *geo,
                           const float *zrec, int zb, uint32_t zmin, uint32_t vmask, uint32_t *keyA, uint32_t *valA,
                           uint32_t *voff, cudaStream_t s)
{
    if (nv <= 0 || n <= 0) return cudaSuccess;
    if ((size_t)nv * (size_t)n >= ((size_t)1 << 32) || zb < 0 || zb > 31) return cudaErrorInvalidValue;
    const uint32_t nw = (uint32_t)((n + 31) / 32);
    const size_t total = (size_t)nv * nw;
    k_emit_vis_words<uint32_t><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        words, woff, (uint32_t)nv, nw, (uint32_t)n, geo, zrec, zb, zmin, vmask, keyA, valA, voff, ~(size_t)0, nullptr,
        nullptr);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_key_params(const BatchInfo *info, int nv, KeyParams *kp, cudaStream_t s)
{
    k_key_params<<<1, 32, 0, s>>>(info, nv, kp); count_launch();
    return cudaGetLastError();
}

cudaError_t emit_vis_words_dev(const uint32_t *words, const uint32_t *woff, int nv, int64_t n, const GeoRec *geo,
                               const float *zrec, const KeyParams *kp, uint32_t *keyA, uint32_t *valA, uint32_t *voff,
                               size_t cap_R, uint32_t *overflow, cudaStream_t s)
{
    if (nv <= 0 || n <= 0) return cudaSuccess;
    if ((size_t)nv * (size_t)n >= ((size_t)1 << 32)) return cudaErrorInvalidValue;
    const uint32_t nw = (uint32_t)((n + 31) / 32);
    const size_t total = (size_t)nv * nw;
    k_emit_vis_words<uint32_t><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        words, woff, (uint32_t)nv, nw, (uint32_t)n, geo, zrec, 0, 0u, 0u, keyA, valA, voff, cap_R, overflow, kp);
    count_launch();
    return cudaGetLastError();
}

size_t radix_segment_blocks_max(size_t cap, int nv) { return (cap + kRsTile - 1) / kRsTile + (size_t)(nv > 0 ? nv : 1); }

cudaError_t launch_segment_blocks(const uint32_t *off, int nv, const KeyParams *kp, int gsz, size_t cap,
                                  RsBlock *blk, size_t nblk_max, cudaStream_t s)
{
    if (nv < 1 || nv > 1024 || (!kp && gsz < 1) || nblk_max >= ((size_t)1 << 24) || cap >= ((size_t)1 << 32))
        return cudaErrorInvalidValue;
    k_segment_blocks<<<1, 1024, 0, s>>>(off, nv, kp, gsz, (uint32_t)cap, blk, (uint32_t)nblk_max); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_entry_offsets_dev(const uint32_t *warp_off, const uint2 *rect_sorted, const uint32_t *voff, int nv,
                                     const BatchInfo *info, size_t cap_R, size_t cap_M, uint32_t *eoff, cudaStream_t s)
{
    if (nv <= 0) return cudaSuccess;
    k_entry_offsets_dev<<<1, 256, 0, s>>>(warp_off, rect_sorted, voff, nv, info, cap_R, cap_M, eoff);
    count_launch();
    return cudaGetLastError();
}

size_t radix_tmp_bytes(size_t n)
{
    size_t nblocks = (n + kRsTile - 1) / kRsTile;
    size_t h = 256 * nblocks;
    size_t a = (h * sizeof(uint32_t) + 255) & ~(size_t)255;
    return 2 * a + scan_tmp_bytes(h) + 256;
}

template <typename KeyT>
cudaError_t radix_sort_pairs(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, size_t n, int end_bit,
                             void *tmp, bool *result_in_alt, cudaStream_t s, const unsigned long long *d_n)
{
    *result_in_alt = false;
    if (n <= 1) return cudaSuccess;
    const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
    const size_t h = 256 * (size_t)nblocks;
    const size_t a = (h * sizeof(uint32_t) + 255) & ~(size_t)255;
    uint32_t *hist = reinterpret_cast<uint32_t *>(tmp);
    uint32_t *offs = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(tmp) + a);
    void *stmp = reinterpret_cast<char *>(tmp) + 2 * a;
    constexpr size_t smem = rs_smem<KeyT>();
    if (!d_n) {   // per device, idempotent (done beforehand when capturing)
        cudaFuncSetAttribute(k_radix_scatter<KeyT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_radix_scatter<KeyT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    KeyT *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    bool alt = false;
    for (int shift = 0; shift < end_bit; shift += 8) {
        k_radix_hist<KeyT><<<nblocks, kRsThreads, 0, s>>>(kin, n, shift, hist, nblocks, d_n, nullptr); count_launch();
        cudaError_t e = exclusive_scan_u32(hist, offs, h, stmp, nullptr, s);
        if (e != cudaSuccess) return e;
        // the lowest digit, and those below the top two passes, are close to
        // uniformly distributed
        if (shift == 0 || shift + 8 < end_bit - 8)
            k_radix_scatter<KeyT, true><<<nblocks, kRsThreads, smem, s>>>(kin, vin, kout, vout, n, shift, hist, offs,
                                                                         nblocks, d_n, nullptr);
        else
            k_radix_scatter<KeyT, false><<<nblocks, kRsThreads, smem, s>>>(kin, vin, kout, vout, n, shift, hist,
                                                                          offs, nblocks, d_n, nullptr);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        KeyT *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
        alt = !alt;
    }
    *result_in_alt = alt;
    return cudaSuccess;
}

size_t radix_segment_blocks(const uint64_t *seg, int nseg, RsBlock *tbl)
{
    size_t k = 0, hbase = 0;
    for (int g = 0; g < nseg; ++g) {
        const uint64_t len = seg[g + 1] - seg[g];
        const uint64_t nb = (len + kRsTile - 1) / kRsTile;
        if (tbl) {
            for (uint64_t b = 0; b < nb; ++b) {
                const uint64_t st = seg[g] + b * kRsTile;
                tbl[k + b].start = (uint32_t)st;
                tbl[k + b].end = (uint32_t)(st + kRsTile < seg[g + 1] ? st + kRsTile : seg[g + 1]);
                tbl[k + b].h0 = (uint32_t)(hbase + b);
                tbl[k + b].hs = (uint32_t)nb;
            }
        }
        k += nb;
        hbase += 256 * nb;
    }
    return k;
}

template <typename KeyT>
cudaError_t radix_sort_segments(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, const RsBlock *blk,
                                size_t nblk, int end_bit, void *tmp, bool *result_in_alt, cudaStream_t s,
                                bool prepared)
{
    *result_in_alt = false;
    if (nblk == 0 || end_bit <= 0) return cudaSuccess;
    const size_t h = 256 * nblk;
    const size_t a = (h * sizeof(uint32_t) + 255) & ~(size_t)255;
    uint32_t *hist = reinterpret_cast<uint32_t *>(tmp);
    uint32_t *offs = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(tmp) + a);
    void *stmp = reinterpret_cast<char *>(tmp) + 2 * a;
    constexpr size_t smem = rs_smem<KeyT>();
    if (!prepared) {
        cudaFuncSetAttribute(k_radix_scatter<KeyT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_radix_scatter<KeyT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    KeyT *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    bool alt = false;
    const size_t nmax = ~(size_t)0;   // ranges come from blk
    for (int shift = 0; shift < end_bit; shift += 8) {
        k_radix_hist<KeyT><<<(unsigned)nblk, kRsThreads, 0, s>>>(kin, nmax, shift, hist, 0, nullptr, blk);
        count_launch();
        cudaError_t e = exclusive_scan_u32(hist, offs, h, stmp, nullptr, s);
        if (e != cudaSuccess) return e;
        if (shift == 0 || shift + 8 < end_bit - 8)
            k_radix_scatter<KeyT, true><<<(unsigned)nblk, kRsThreads, smem, s>>>(kin, vin, kout, vout, nmax, shift,
                                                                                hist, offs, 0, nullptr, blk);
        else
            k_radix_scatter<KeyT, false><<<(unsigned)nblk, kRsThreads, smem, s>>>(kin, vin, kout, vout, nmax, shift,
                                                                                 hist, offs, 0, nullptr, blk);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        KeyT *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
        alt = !alt;
    }
    *result_in_alt = alt;
    return cudaSuccess;
}

template cudaError_t radix_sort_segments<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, const RsBlock *,
                                                   size_t, int, void *, bool *, cudaStream_t, bool);

template cudaError_t radix_sort_pairs<uint64_t>(uint64_t *, uint32_t *, uint64_t *, uint32_t *, size_t, int, void *,
                                                bool *, cudaStream_t, const unsigned long long *);
template cudaError_t radix_sort_pairs<uint32_t>(uint32_t *, uint32_t *, uint32_t *, uint32_t *, size_t, int, void *,
                                                bool *, cudaStream_t, const unsigned long long *);

void radix_prepare()
{
    cudaFuncSetAttribute(k_radix_scatter<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rs_smem<uint64_t>());
    cudaFuncSetAttribute(k_radix_scatter<uint64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rs_smem<uint64_t>());
    cudaFuncSetAttribute(k_radix_scatter<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rs_smem<uint32_t>());
    cudaFuncSetAttribute(k_radix_scatter<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rs_smem<uint32_t>());
}

}  // namespace gavis
