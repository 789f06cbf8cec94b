// raster.cu -- tile binning, per-tile front-to-back compositing and the
// reductions of the GAVIS hot path.
//
//   k_emit_records    stage A of binning from per-record counts (the path
//                     without visibility words; the batched path emits stage A
//                     from the projection's visibility words, in sort.cu)
//   k_emit_tiles      stage B: the record's tiles, in stage-A order
//   k_ranges          [start, end) of every (view, tile) in the sorted entries
//   k_order_keys      the scoring tiles' order, longest list first
//   k_composite_ua    Alg. "3DGS Uncertainty Quantification with Visibility
//                     Field" + plain colour (eq:orig_vr): a persistent grid
//                     whose warps take (view, tile, 8x8 block) items
//   k_composite_vis   Alg. "Single-view Particle Visibility": a block per
//                     (view, tile), per-Gaussian sums reduced per warp
//   k_view_reduce     per-view mean of the per-pixel entropy (eq:id)
//   k_argmax          next-best view (eq:i_gain)
//   k_vf_accumulate   gamma_lm += v a_l Y_lm(d_p) (eq:vis_gamma)
//
// Compositing: each warp owns an 8 x 8 pixel block of a tile (two pixels
// per thread, rows j and j + 4) and walks the tile's list on its own, in
// chunks of 32 entries: every lane gathers one entry's record (by Gaussian
// index from the per-view records), drops it if the footprint box
// (half-extents rounded up) or the ellipse itself misses the block's pixel
// centres, and the survivors are compacted in order into warp-private shared
// memory and composited front to back.  The footprint value q of a
// (pixel, Gaussian) pair uses explicit round-to-nearest operations in a fixed
// order, so the overlap decision q <= q_cut is reproducible bit for bit; the
// culling tests are conservative and never change a pixel's result.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>

#include "gavis_internal.cuh"
#include "sh_basis.cuh"

namespace gavis {
namespace {

// footprint box (x0, x1, y0, y1) from the packed half-extents
__device__ __forceinline__ float4 footprint_box(float u, float v, float ext_bits)
{
    const uint32_t e = __float_as_uint(ext_bits);
    const float ex = __half2float(__ushort_as_half((unsigned short)(e & 0xffffu)));
    const float ey = __half2float(__ushort_as_half((unsigned short)(e >> 16)));
    return make_float4(u - ex, u + ex, v - ey, v + ey);
}

__device__ __forceinline__ bool box_misses(const float4 b, float bx0, float bx1, float by0, float by1)
{
    return b.y < bx0 || b.x > bx1 || b.w < by0 || b.z > by1;
}

// True only if q(d) = A dx^2 + B2 dx dy + C dy^2 (d = p - (u, v)) exceeds
// q_cut at every point p of the rectangle [bx0, bx1] x [by0, by1] of a warp's
// pixel centres, so no pixel of the warp can be covered.  The minimum of the
// convex q over the rectangle is 0 if the centre lies inside, else it lies on
// an edge, where q is a parabola in one variable minimised at a clamped
// stationary point.  The decision must never cull a Gaussian that
// footprint_q admits at some pixel: both evaluations err by a few float32
// ulps of S = A dx^2 + |B2 dx dy| + C dy^2 <= 2 (A dx^2 + C dy^2), so the
// test keeps a margin of 2^-16 times that bound over the rectangle
// (8 times the worst-case error) plus 2^-10 q_cut.
__device__ __forceinline__ bool ellipse_misses(float u, float v, float A, float B2, float C, float bx0, float bx1,
                                               float by0, float by1, float qcut)
{
    const float X0 = bx0 - u, X1 = bx1 - u, Y0 = by0 - v, Y1 = by1 - v;
    if (X0 <= 0.0f && X1 >= 0.0f && Y0 <= 0.0f && Y1 >= 0.0f) return false;
    // stationary points per unit offset (any point of an edge gives a valid
    // upper bound on its minimum, so an approximate quotient is enough)
    const float hA = __fdividef(-0.5f * B2, A), hC = __fdividef(-0.5f * B2, C);
    float m = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float X = e ? X1 : X0, Y = e ? Y1 : Y0;
        const float dy = fminf(fmaxf(hC * X, Y0), Y1);    // vertical edge dx = X
        m = fminf(m, fmaf(fmaf(A, X, B2 * dy), X, C * dy * dy));
        const float dx = fminf(fmaxf(hA * Y, X0), X1);    // horizontal edge dy = Y
        m = fminf(m, fmaf(fmaf(A, dx, B2 * Y), dx, C * Y * Y));
    }
    const float Dx = fmaxf(fabsf(X0), fabsf(X1)), Dy = fmaxf(fabsf(Y0), fabsf(Y1));
    const float smax = 2.0f * fmaf(A, Dx * Dx, C * Dy * Dy);
    return m > fmaf(smax, 1.52587890625e-5f, qcut * (1.0f + 9.765625e-4f));
}

// L2 prefetch of the record a chunk will gather next (its address is known
// one chunk ahead; the gather itself then finds it in L2)
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float footprint_q(float px, float py, float u, float v, float A, float B2, float C)
{
    const float dx = __fsub_rn(px, u), dy = __fsub_rn(py, v);
    const float qa = __fmul_rn(A, dx);
    const float qb = __fmaf_rn(B2, dy, qa);
    const float qc = __fmul_rn(C, dy);
    const float qd = __fmul_rn(qc, dy);
    return __fmaf_rn(qb, dx, qd);
}


// stage A: one record key per visible (view, Gaussian), in (view, index) order
__global__ void k_emit_records(const uint32_t *counts, const uint32_t *pos, const GeoRec *geo, int nv, int64_t n,
                               int zb, uint32_t zmin, uint64_t *keyA, uint32_t *valA, size_t cap_R,
                               uint32_t *overflow)
{
    const size_t total = (size_t)nv * (size_t)n;
    const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total || counts[r] == 0u) return;
    const uint64_t v = r / (size_t)n;
    const uint32_t i = pos[r];
    if ((size_t)i >= cap_R) {
        if (overflow) *overflow = 1u;
        return;
    }
    keyA[i] = (v << zb) | (uint64_t)(__float_as_uint(geo[r].b.z) - zmin);
    valA[i] = (uint32_t)r;
}

// eoff[v] = tile entries of the views before v (v = 0..nv): the stage-B
// offset of each view's first record (records are in view order)
__device__ __forceinline__ uint32_t rect_tiles(uint2 rc)
{
    return ((rc.x >> 16) - (rc.x & 0xffffu) + 1u) * ((rc.y >> 16) - (rc.y & 0xffffu) + 1u);
}

// the first tile entry of record r: its warp's offset plus the tiles of the
// warp's records before it
__device__ __forceinline__ uint32_t record_entry_offset(const uint32_t *warp_off, const uint2 *rect_sorted, uint32_t r)
{
    uint32_t o = warp_off[r >> 5];
    for (uint32_t q = r & ~31u; q < r; ++q) o += rect_tiles(rect_sorted[q]);
    return o;
}

__global__ void k_entry_offsets(const uint32_t *warp_off, const uint2 *rect_sorted, const uint32_t *voff, int nv,
                                uint32_t M, uint32_t *eoff)
{
    for (int v = threadIdx.x; v <= nv; v += blockDim.x) {
        const uint32_t r = voff[v];
        eoff[v] = v < nv && r < voff[nv] ? record_entry_offset(warp_off, rect_sorted, r) : M;
    }
}

__global__ void k_gather_counts(const uint32_t *valA, const uint32_t *counts, size_t nrec, uint32_t *cnt_sorted,
                                const unsigned long long *d_nrec)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec || (d_nrec && i >= (size_t)*d_nrec)) return;
    cnt_sorted[i] = counts[valA[i]];
}

// the tile rectangle of each record in stage-A order (one gather), and its
// tile count, which the rectangle gives
// warp_cnt[w] = tiles of the records [32 w, 32 w + 32) (0 past the live
// records), for every warp of the capacity (blocks of whole warps)
__global__ void k_gather_rects(const uint32_t *valA, const uint2 *rect, size_t nrec, uint32_t *warp_cnt,
                               uint2 *rect_sorted, const unsigned long long *d_nrec)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t live = nrec;
    if (d_nrec && (size_t)*d_nrec < live) live = (size_t)*d_nrec;
    uint32_t cnt = 0u;
    if (i < live) {
        const uint2 rc = rect[valA[i]];
        rect_sorted[i] = rc;
        cnt = rect_tiles(rc);
    }
    const uint32_t ws = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31u) == 0u && i < nrec) warp_cnt[i >> 5] = ws;
}


// Tile keys: v * TT + tile (tb < 0), or (v << tb) | tile with 2^tb >= TT, so
// that the keys of a group of 2^g views differ only in their low tb + g bits.
__device__ __forceinline__ uint32_t tile_index(uint32_t key, int tb, uint32_t TT)
{
    return tb < 0 ? key : (key >> tb) * TT + (key & ((1u << tb) - 1u));
}

// approximate reciprocal (PTX rcp.approx)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// stage B: the tiles of each record, in stage-A order.  A warp takes 32
// consecutive records, whose entries are contiguous (from the warp's offset,
// warp_off, or its first record's, off_sorted); its lanes write those
// entries in order, lane j of a round finding its record from a ballot of the
// records that start before the round and an OR of the window positions
// where the others start, so the stores are coalesced.
__global__ void k_emit_tiles(const uint32_t *valA, const uint32_t *off_sorted, size_t nrec, const uint2 *rect, int64_t n,
                             DivU32 div_n, int TW, int TH, uint32_t *keyB, uint32_t *valB,
                             const unsigned long long *d_nrec, size_t cap_M, uint32_t *overflow, int tb,
                             const uint2 *rect_sorted, const uint32_t *warp_off)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(threadIdx.x & 31u);
    size_t live = nrec;
    if (d_nrec && (size_t)*d_nrec < live) live = (size_t)*d_nrec;
    // per record: its Gaussian, the key of its first tile, the rectangle's
    // width and its reciprocal, its tile count and first entry
    uint32_t g = 0, kfirst = 0, w = 1, cnt = 0, off = 0;
    if (i < live) {
        const uint32_t r = valA[i];   // record indices are 32-bit: v = r / n in 32-bit arithmetic
        const uint32_t v = div_u32(r, div_n);
        g = r - v * (uint32_t)n;
        const uint2 rc = rect_sorted ? rect_sorted[i] : rect[r];
        const uint32_t x0 = rc.x & 0xffffu, y0 = rc.y & 0xffffu;
        w = (rc.x >> 16) - x0 + 1u;
        cnt = w * ((rc.y >> 16) - y0 + 1u);
        kfirst = (tb < 0 ? v * (uint32_t)(TW * TH) : v << tb) + y0 * (uint32_t)TW + x0;
        off = warp_off ? warp_off[i >> 5] : off_sorted[i];
    }
    const float rw = rcp_approx((float)w);
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - cnt;
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    const uint32_t base = __shfl_sync(0xffffffffu, off, 0);   // the valid lanes are a prefix of the warp
    if (cnt && (size_t)base + excl + cnt > cap_M && overflow) *overflow = 1u;
    const uint32_t room = cap_M > (size_t)base ? (uint32_t)min(cap_M - (size_t)base, (size_t)0xffffffffu) : 0u;
    for (uint32_t j0 = 0; j0 < total; j0 += 32) {
        const uint32_t j = j0 + (uint32_t)lane;
        // the last lane whose entries start at or before j: the lanes that
        // start before the window, plus those whose start lies in the window
        // at or before j (a visible record has at least one tile, so the
        // valid lanes' starts are distinct; the empty lanes past the last
        // record start at `total`, which no j reaches)
        const uint32_t before = (uint32_t)__popc(__ballot_sync(0xffffffffu, excl < j0));
        const uint32_t starts =
            __reduce_or_sync(0xffffffffu, (excl >= j0 && excl - j0 < 32u) ? 1u << (excl - j0) : 0u);
        const int k = (int)(before + (uint32_t)__popc(starts & (0xffffffffu >> (31 - lane)))) - 1;
        const uint32_t ek = __shfl_sync(0xffffffffu, excl, k), wk = __shfl_sync(0xffffffffu, w, k);
        const uint32_t fk = __shfl_sync(0xffffffffu, kfirst, k), gk = __shfl_sync(0xffffffffu, g, k);
        const float rk = __shfl_sync(0xffffffffu, rw, k);
        if (j < total && j < room) {
            // row and column of entry m of the rectangle: with the
            // approximate reciprocal the float quotient has a relative error
            // below 2^-21, so for m < 2^20 it is within one of m / wk, and one
            // correction step each way makes it exact
            const uint32_t m = j - ek;
            uint32_t ty, tx;
            if (m < (1u << 20)) {
                ty = (uint32_t)((float)m * rk);
                int d = (int)(m - ty * wk);
                if (d < 0) { --ty; d += (int)wk; }
                else if (d >= (int)wk) { ++ty; d -= (int)wk; }
                tx = (uint32_t)d;
            } else {
                ty = m / wk;
                tx = m - ty * wk;
            }
            const size_t pos = (size_t)base + j;
            keyB[pos] = fk + ty * (uint32_t)TW + tx;
            valB[pos] = gk;
        }
    }
}

__global__ void k_ranges(const uint32_t *keys, size_t M, uint2 *ranges, const unsigned long long *d_M, int tb,
                         uint32_t TT)
{
    if (d_M && *d_M < M) M = (size_t)*d_M;
    // one 16-byte word per thread: keys [4w, 4w + 4) (key buffers start 16-byte
    // aligned and are padded, so the word of the last key lies inside them)
    const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t i0 = 4 * w;
    const unsigned lane = threadIdx.x & 31u;
    uint4 q = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    if (i0 < M) q = reinterpret_cast<const uint4 *>(keys)[w];
    // the neighbours across words come from the adjacent lanes; the warp's two edge lanes load theirs
    uint32_t prev = __shfl_up_sync(0xffffffffu, q.w, 1), next = __shfl_down_sync(0xffffffffu, q.x, 1);
    if (i0 >= M) return;
    if (lane == 0 && i0 > 0) prev = keys[i0 - 1];
    if (lane == 31 && i0 + 4 < M) next = keys[i0 + 4];
    const uint32_t k[6] = {prev, q.x, q.y, q.z, q.w, next};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const size_t i = i0 + (size_t)j;
        if (i >= M) break;
        const uint32_t t = k[j + 1];
        const uint32_t ti = tile_index(t, tb, TT);
        if (i == 0 || k[j] != t) ranges[ti].x = (uint32_t)i;
        if (i == M - 1 || k[j + 2] != t) ranges[ti].y = (uint32_t)(i + 1);
    }
}

__global__ void k_order_keys(const uint2 *ranges, size_t nt, uint32_t *keys, uint32_t *vals)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const uint2 rg = ranges[t];
    const uint32_t len = rg.y > rg.x ? rg.y - rg.x : 0u;
    const uint32_t q = len >> 4;
    keys[t] = 255u - (q < 255u ? q : 255u);
    vals[t] = (uint32_t)t;
}

__global__ void k_keys_export(const uint32_t *keyB, const uint32_t *valB, size_t M, const GeoRec *geo, int64_t n,
                              int tiles_per_view, uint64_t *out, int tb)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const uint32_t t = tile_index(keyB[i], tb, (uint32_t)tiles_per_view);
    const size_t r = (size_t)(t / (uint32_t)tiles_per_view) * (size_t)n + valB[i];
    out[i] = ((uint64_t)t << 32) | (uint64_t)__float_as_uint(geo[r].b.z);
}

// 2^x and log2(x) on the special-function unit (PTX ex2/lg2, approximate;
// exp(x) = 2^(x log2 e) and ln(x) = ln2 log2(x))
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kNegHalfLog2e = -0.72134752044448170368f;   // -log2(e) / 2
constexpr float kLn2 = 0.69314718055994530942f;

// Uncertainty + colour compositing.  The work items are the 8 x 8 pixel
// blocks of every (view, tile), in view-major order; a persistent grid of
// 4-warp CTAs runs them, each warp taking the next item from a global counter
// as soon as it has finished the last, so that no warp waits for another
// (the items' lengths differ a lot: list length and early saturation).  For
// an item the warp (each thread two pixels, (x, y) and (x, y + 4)) walks the
// tile's depth-sorted list on its own, 32 entries at a time: every lane loads
// one entry's footprint, the entries whose footprint touches the block are
// compacted (in list order) into the warp's shared-memory slots, and the warp
// composites them.  It stops as soon as all its pixels are saturated.
// Per pixel and overlapping entry: alpha = o 2^(-q log2(e)/2); colour
// w = alpha Tc, Tc -= w; uncertainty alpha* = a1 alpha + a0 (eq:alpha_comp),
// w = alpha* T, wv = w V, T -= w.  The entropy bound (eq:huber) is assembled
// once per pixel from sum(wv), sum(wv log2 wv) and the prior mass
// w0 = (1 - T) - sum(wv); each item writes its pixels' sum to
// tile_sums[item] (summed per view in item order: deterministic).
// KC: the visible components carry per-Gaussian kc (colour variances given);
// otherwise the constant k_c is applied to sum(wv) once per pixel.
// DEPTH: also accumulate the expected depth sum_i alpha_i T_c,i z_i along the
// colour path (into a.depth).
constexpr int kUaWarps = 4;   // warps per CTA of the uncertainty pass

// PAIRS: count the pixel-Gaussian pairs composited (instrumentation; into
// a.pair_counts, one count per 8 x 8 block).
template <int TILE, bool KC, bool DEPTH, bool PAIRS>
__global__ void __launch_bounds__(kUaWarps * 32) k_composite_ua(CompositeArgs a)
{
    constexpr int NW = kUaWarps;
    constexpr int BPT = blocks_per_tile(TILE);
    __shared__ float4 s_g0[NW][32];   // u, v, A, 2B
    __shared__ float2 s_g1[NW][32];   // C, opacity
    __shared__ float4 s_u0[NW][32];   // a1, a0, V, r
    __shared__ float2 s_u1[NW][32];   // g, b
    __shared__ float s_kc[KC ? NW : 1][32];
    __shared__ float s_z[DEPTH ? NW : 1][32];

    const int tiles = a.TW * a.TH;
    const unsigned long long items = (unsigned long long)a.nv * (unsigned long long)tiles * BPT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const RasterConsts rc = a.rc;
    const bool colour = DEPTH || a.rgb != nullptr;   // colour path only when asked for
    float *kcs = s_kc[KC ? warp : 0];
    float *zs = s_z[DEPTH ? warp : 0];
    float4 *g0s = s_g0[warp];
    float2 *g1s = s_g1[warp];
    float4 *u0s = s_u0[warp];
    float2 *u1s = s_u1[warp];
    const size_t plane = (size_t)a.W * a.H;

    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.work, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= items) break;
        const unsigned long long slot = item / BPT;
        const int blk = (int)(item - slot * BPT);
        const uint32_t bt = a.order ? a.order[slot] : (uint32_t)slot;   // (view, tile); nv * tiles < 2^32
        const int vb = (int)div_u32(bt, a.div_tiles);
        const int t = (int)(bt - (uint32_t)vb * (uint32_t)tiles);
        const int ty = (int)div_u32((uint32_t)t, a.div_TW), tx = t - ty * a.TW;
        const int wx = (blk % (TILE / 8)) * 8, wy = (blk / (TILE / 8)) * 8;
        const int i = tx * TILE + wx + (lane & 7);
        const int j0 = ty * TILE + wy + (lane >> 3);
        const float bx0 = (float)(tx * TILE + wx) + 0.5f, bx1 = bx0 + 7.0f;
        const float by0 = (float)(ty * TILE + wy) + 0.5f, by1 = by0 + 7.0f;
        const float px = (float)i + 0.5f;
        const uint2 rg = a.ranges[bt];
        const size_t vrow = (size_t)vb * (size_t)a.n;

        float T[2], Tc[2], sl[2], swv[2], skc[2], cr[2], cg[2], cb[2], py[2], dz[2];
        bool ua_on[2], rgb_on[2], inside[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int j = j0 + 4 * p;
            inside[p] = i < a.W && j < a.H;
            py[p] = (float)j + 0.5f;
            T[p] = 1.0f; Tc[p] = 1.0f; sl[p] = 0.0f; swv[p] = 0.0f; skc[p] = 0.0f; cr[p] = 0.0f; cg[p] = 0.0f; cb[p] = 0.0f;
            dz[p] = 0.0f;
            ua_on[p] = inside[p];
            rgb_on[p] = inside[p] && colour;
        }
        uint32_t npairs = 0;

        uint32_t nval = rg.x + lane < rg.y ? a.vals[rg.x + lane] : 0u;   // this lane's entry of the next chunk
        for (uint32_t base = rg.x; base < rg.y; base += 32) {
            if (!__any_sync(0xffffffffu, ua_on[0] || rgb_on[0] || ua_on[1] || rgb_on[1])) break;
            const uint32_t e = base + lane;
            const uint32_t val = nval;
            const bool more = e + 32 < rg.y;
            if (more) nval = a.vals[e + 32];
            bool mine = false;
            GeoRec gr;
            size_t r = 0;
            if (e < rg.y) {
                r = vrow + val;
                gr = a.geo[r];
                mine = !box_misses(footprint_box(gr.a.x, gr.a.y, gr.b.w), bx0, bx1, by0, by1) &&
                       !ellipse_misses(gr.a.x, gr.a.y, gr.a.z, gr.a.w, gr.b.x, bx0, bx1, by0, by1, rc.q_cut);
            }
            const unsigned m = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                const int slot = __popc(m & lt);
                const UaRec ur = a.ua[r];
                g0s[slot] = gr.a;
                g1s[slot] = make_float2(gr.b.x, gr.b.y);
                u0s[slot] = ur.a;
                u1s[slot] = make_float2(ur.b.x, ur.b.y);
                if (KC) kcs[slot] = ur.b.z;
                if (DEPTH) zs[slot] = gr.b.z;
            }
            __syncwarp();
            if (more) {
                prefetch_l2(a.geo + vrow + nval);
                prefetch_l2(a.ua + vrow + nval);
            }
            const int nk = __popc(m);
            // Straight-line body: a pixel that misses the entry, or whose
            // accumulator has saturated, gets a zero opacity for it, which
            // leaves every sum and transmittance exactly as it was.
            for (int k = 0; k < nk && (ua_on[0] || rgb_on[0] || ua_on[1] || rgb_on[1]); ++k) {
                const float4 g0 = g0s[k];
                const float2 g1 = g1s[k];
                const float4 u0 = u0s[k];
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float q = footprint_q(px, py[p], g0.x, g0.y, g0.z, g0.w, g1.x);
                    const bool hit = q <= rc.q_cut;
                    const bool hc = hit && rgb_on[p], hu = hit && ua_on[p];
                    if (PAIRS) npairs += (uint32_t)(hc || hu);
                    const float alpha = ex2_approx(fmaf(q, kNegHalfLog2e, g1.y));   // o exp(-q/2)
                    if (colour) {   // the same for every thread of the launch
                        const float2 u1 = u1s[k];
                        const float ac = hc ? alpha : 0.0f;
                        const float wc = ac * Tc[p];
                        cr[p] = fmaf(wc, u0.w, cr[p]);
                        cg[p] = fmaf(wc, u1.x, cg[p]);
                        cb[p] = fmaf(wc, u1.y, cb[p]);
                        if (DEPTH) dz[p] = fmaf(wc, zs[k], dz[p]);
                        Tc[p] -= wc;
                        rgb_on[p] = Tc[p] >= rc.eps_T;
                    }
                    const float as = hu ? fmaf(alpha, u0.x, u0.y) : 0.0f;   // eq:alpha_comp
                    const float w = as * T[p];
                    const float wv = w * u0.z;                               // weight of the visible component
                    sl[p] = fmaf(wv, lg2_approx(fmaxf(wv, 1e-30f)), sl[p]);
                    swv[p] += wv;
                    if (KC) skc[p] = fmaf(wv, kcs[k], skc[p]);
                    T[p] -= w;
                    ua_on[p] = T[p] >= rc.eps_T;
                }
            }
            __syncwarp();
        }
        float h = 0.0f;
        const size_t vg = (size_t)(a.v0 + vb);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            if (!inside[p]) continue;
            // eq:huber: visible components sum wv (k_c - ln wv); prior w0 (k_0 - ln w0)
            const float w0 = fmaxf((1.0f - T[p]) - swv[p], 0.0f);
            float Hs = (KC ? skc[p] : rc.k_c * swv[p]) - kLn2 * sl[p];
            if (w0 > 1e-30f) Hs = fmaf(w0, rc.k_0 - kLn2 * lg2_approx(w0), Hs);
            const size_t pix = (size_t)(j0 + 4 * p) * a.W + i;
            if (a.unc) a.unc[vg * plane + pix] = Hs;
            if (DEPTH) a.depth[vg * plane + pix] = dz[p];
            if (a.rgb) {
                a.rgb[(vg * 3 + 0) * plane + pix] = cr[p];
                a.rgb[(vg * 3 + 1) * plane + pix] = cg[p];
                a.rgb[(vg * 3 + 2) * plane + pix] = cb[p];
            }
            h += Hs;
        }
        // the block's partial sum of the per-pixel entropy (fixed order: deterministic)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
        const uint32_t wp = PAIRS ? __reduce_add_sync(0xffffffffu, npairs) : 0u;
        if (lane == 0) {   // at the block's natural index: summed per view in (tile, block) order
            a.tile_sums[(size_t)bt * BPT + blk] = h;
            if (PAIRS) a.pair_counts[(size_t)bt * BPT + blk] = wp;
        }
    }
}

// Single-view particle visibility.  Each warp owns an 8 x 8 pixel block of
// the tile (each thread two pixels) and walks the tile's depth-sorted list on
// its own, 32 entries at a time, compacting the entries whose footprint box
// touches the block.  Per overlapping entry a pixel contributes its current T
// (fixed point, 2^-18) and a count of one to the Gaussian's sums: the pixel's
// word is (round(T 2^18) << kCntBits) + 1, the warp adds its 64 pixels' words
// with one redux, and the chunk's per-entry sums are flushed to the
// Gaussians' accumulators once per chunk, one atomic pair per entry.  The
// transmittance is kept scaled by 2^18 (exact: a power of two), and alpha is
// 2^(log2(o) - q log2(e)/2).  A warp stops when its pixels saturate.
// round(T) * 2^kCntBits + 1 (one hit carrying its scaled transmittance), for
// 0 <= T < 2^23: adding 2^23 leaves T rounded to the nearest integer (ties to
// even, as __float2uint_rn) in the low bits of the sum, without a conversion
__device__ __forceinline__ uint32_t hit_word(float T)
{
    constexpr uint32_t kMul = 1u << kCntBits;
    return __float_as_uint(T + 8388608.0f) * kMul + (1u - 0x4B000000u * kMul);
}

template <int TILE>
__global__ void __launch_bounds__(TILE *TILE / 2) k_composite_vis(CompositeArgs a)
{
    constexpr int NT = TILE * TILE / 2;
    constexpr int NW = NT / 32;
    __shared__ float4 s_g0[NW][32];
    __shared__ float2 s_g1[NW][32];
    __shared__ uint32_t s_idx[NW][32];
    __shared__ uint32_t s_sum[NW][32];

    const int tiles = a.TW * a.TH;
    const int vb = blockIdx.x / tiles;
    const int t = blockIdx.x - vb * tiles;
    const int tx = t % a.TW, ty = t / a.TW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int wx = (warp % (TILE / 8)) * 8, wy = (warp / (TILE / 8)) * 8;
    const int i = tx * TILE + wx + (lane & 7);
    const int j0 = ty * TILE + wy + (lane >> 3);
    const float bx0 = (float)(tx * TILE + wx) + 0.5f, bx1 = bx0 + 7.0f;
    const float by0 = (float)(ty * TILE + wy) + 0.5f, by1 = by0 + 7.0f;
    const float px = (float)i + 0.5f, py0 = (float)j0 + 0.5f, py1 = py0 + 4.0f;
    const uint2 rg = a.ranges[blockIdx.x];
    const size_t vrow = (size_t)vb * (size_t)a.n;
    const float eps = a.rc.eps_T * kTScale, qcut = a.rc.q_cut;

    float T0 = kTScale, T1 = kTScale;   // transmittance x 2^18
    bool on0 = i < a.W && j0 < a.H, on1 = i < a.W && j0 + 4 < a.H;
    uint32_t wpairs = 0;
    float4 *g0s = s_g0[warp];
    float2 *g1s = s_g1[warp];
    uint32_t *ids = s_idx[warp];
    uint32_t *sums = s_sum[warp];
    constexpr uint32_t kCntMul = 1u << kCntBits;

    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        if (!__any_sync(0xffffffffu, on0 || on1)) break;
        const uint32_t e = base + lane;
        bool mine = false;
        GeoRec gr;
        uint32_t g = 0;
        if (e < rg.y) {
            g = a.vals[e];
            gr = a.geo[vrow + g];
            mine = !box_misses(footprint_box(gr.a.x, gr.a.y, gr.b.w), bx0, bx1, by0, by1) &&
                   !ellipse_misses(gr.a.x, gr.a.y, gr.a.z, gr.a.w, gr.b.x, bx0, bx1, by0, by1, qcut);
        }
        const unsigned mk = __ballot_sync(0xffffffffu, mine);
        if (mine) {
            const int slot = __popc(mk & lt);
            g0s[slot] = gr.a;
            g1s[slot] = make_float2(gr.b.x, gr.b.y);
            ids[slot] = g;
        }
        sums[lane] = 0u;   // entries the warp does not reach (it saturated) add nothing
        // pad the survivors to a multiple of four with entries that overlap no
        // pixel (q = +inf), so the loop below takes four at a time and tests
        // for saturation once per four
        const int nk = __popc(mk);
        const int nk4 = (nk + 3) & ~3;
        if (lane >= nk && lane < nk4) {
            g0s[lane] = make_float4(1e30f, 1e30f, 1.0f, 0.0f);
            g1s[lane] = make_float2(1.0f, -INFINITY);
        }
        __syncwarp();
        for (int k = 0; k < nk4; k += 4) {
            if (!__any_sync(0xffffffffu, on0 || on1)) break;   // warp-uniform
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 g0 = g0s[k + u];
                const float2 g1 = g1s[k + u];
                const float q0 = footprint_q(px, py0, g0.x, g0.y, g0.z, g0.w, g1.x);
                const float q1 = footprint_q(px, py1, g0.x, g0.y, g0.z, g0.w, g1.x);
                const bool h0 = on0 && (q0 <= qcut), h1 = on1 && (q1 <= qcut);
                uint32_t w = 0u;
                if (h0) w = hit_word(T0);
                if (h1) w += hit_word(T1);
                const uint32_t sum = __reduce_add_sync(0xffffffffu, w);
                if (lane == 0) sums[k + u] = sum;   // the same in every lane
                if (h0) {
                    T0 = fmaf(-T0, ex2_approx(fmaf(q0, kNegHalfLog2e, g1.y)), T0);
                    on0 = T0 >= eps;
                }
                if (h1) {
                    T1 = fmaf(-T1, ex2_approx(fmaf(q1, kNegHalfLog2e, g1.y)), T1);
                    on1 = T1 >= eps;
                }
            }
        }
        __syncwarp();
        // lane k adds slot k's sums to its Gaussian's accumulators
        const uint32_t my = sums[lane];
        const uint32_t my_cnt = my & (kCntMul - 1u);
        if (my_cnt) {
            const size_t r = vrow + ids[lane];
            atomicAdd(&a.sumT[r], (unsigned long long)(my >> kCntBits));
            atomicAdd(&a.cnt[r], my_cnt);
            wpairs += my_cnt;
        }
        __syncwarp();
    }
    if (a.pairs) {
        const uint32_t wp = __reduce_add_sync(0xffffffffu, wpairs);
        if (lane == 0 && wp) atomicAdd(a.pairs, (unsigned long long)wp);
    }
}

// instrumentation: sum of the per-warp pair counts into one counter
__global__ void k_sum_counts(const uint32_t *c, size_t count, unsigned long long *out)
{
    __shared__ unsigned long long s[256];
    unsigned long long acc = 0;
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (size_t)gridDim.x * 256) acc += c[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && s[0]) atomicAdd(out, s[0]);
}

__global__ void k_view_reduce(const float *tile_sums, int tiles, float inv_pixels, float *score)
{
    __shared__ float s[256];
    const float *ts = tile_sums + (size_t)blockIdx.x * tiles;
    float acc = 0.0f;
    for (int k = threadIdx.x; k < tiles; k += 256) acc += ts[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) score[blockIdx.x] = s[0] * inv_pixels;
}

__global__ void k_argmax(const float *score, int n, int32_t *best)
{
    __shared__ float sv[1024];
    __shared__ int si[1024];
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int k = threadIdx.x; k < n; k += 1024) {
        float x = score[k];
        if (x > bv || (x == bv && k < bi)) { bv = x; bi = k; }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            float x = sv[threadIdx.x + o];
            int xi = si[threadIdx.x + o];
            if (x > sv[threadIdx.x] || (x == sv[threadIdx.x] && xi < si[threadIdx.x])) {
                sv[threadIdx.x] = x;
                si[threadIdx.x] = xi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *best = si[0] == 0x7fffffff ? -1 : si[0];
}

template <int L>
__global__ void __launch_bounds__(128) k_vf_accumulate(AccumArgs a)
{
    extern __shared__ gavis_camera s_cams[];
    for (int k = threadIdx.x; k < a.nv; k += blockDim.x) s_cams[k] = a.cams[k];
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    constexpr int K = (L + 1) * (L + 1);
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = a.gamma32[(size_t)g * K + k];
    const float mx = a.means[3 * g], my = a.means[3 * g + 1], mz = a.means[3 * g + 2];
    // views in groups of VG: the group's counts, then its sums, are loaded
    // before any is used (independent loads in flight); accumulation stays in
    // view order
    constexpr int VG = 8;
    for (int v0 = 0; v0 < a.nv; v0 += VG) {
        uint32_t c[VG];
        unsigned long long st[VG];
#pragma unroll
        for (int u = 0; u < VG; ++u)
            c[u] = v0 + u < a.nv ? a.cnt[(size_t)(v0 + u) * (size_t)a.n + (size_t)g] : 0u;
#pragma unroll
        for (int u = 0; u < VG; ++u) st[u] = c[u] ? a.sumT[(size_t)(v0 + u) * (size_t)a.n + (size_t)g] : 0ull;
#pragma unroll
        for (int u = 0; u < VG; ++u) {
            if (c[u] == 0u) continue;   // Phi = 0: no pixel of this view reaches g
            const float vis = (float)st[u] * (1.0f / kTScale) / (float)c[u];
            const gavis_camera &cam = s_cams[v0 + u];
            const float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
            const float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
            float Y[K];
            sh_basis<L>(dx * rn, dy * rn, dz * rn, Y);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int l = k >= 25 ? 5 : (k >= 16 ? 4 : (k >= 9 ? 3 : (k >= 4 ? 2 : (k >= 1 ? 1 : 0))));   // k in [l^2, (l+1)^2)
                acc[k] = fmaf(vis * a.a_l[l], Y[k], acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) a.gamma32[(size_t)g * K + k] = acc[k];
}

__global__ void k_vf_store(const float *src, size_t count, void *out, int dtype, int accumulate)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float x = src[i];
    if (dtype == GAVIS_F16) {
        __half *o = reinterpret_cast<__half *>(out);
        o[i] = __float2half_rn(x);
    } else if (dtype == GAVIS_BF16) {
        __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out);
        o[i] = __float2bfloat16_rn(x);
    } else {
        reinterpret_cast<float *>(out)[i] = x;
    }
    (void)accumulate;
}

__global__ void k_vf_load(const void *in, int dtype, size_t count, float *dst)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float x;
    if (dtype == GAVIS_F16) x = __half2float(reinterpret_cast<const __half *>(in)[i]);
    else if (dtype == GAVIS_BF16) x = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(in)[i]);
    else x = reinterpret_cast<const float *>(in)[i];
    dst[i] = x;
}

__global__ void k_vis_export(const unsigned long long *sumT, const uint32_t *cnt, size_t count, float *sumT_f,
                             uint32_t *cnt_out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (sumT_f) sumT_f[i] = (float)((double)sumT[i] / (double)kTScale);
    if (cnt_out) cnt_out[i] = cnt[i];
}

// ------------------------------------------------------------------ density control
// virtual particles: identity rotation, isotropic scale, zero opacity
__global__ void k_virtual_fill(const float *vmeans, int64_t n_virt, float scale, float *means, float *scales,
                               float *rots, float *opac)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_virt) return;
    for (int k = 0; k < 3; ++k) {
        means[3 * j + k] = vmeans[3 * j + k];
        scales[3 * j + k] = scale;
    }
    reinterpret_cast<float4 *>(rots)[j] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    opac[j] = 0.0f;
}

__global__ void k_fill_f32(float *x, size_t count, float value)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) x[i] = value;
}

// count 16-bit elements set to one bit pattern (1.0 in f16 or bf16)
__global__ void k_fill_u16(uint16_t *x, size_t count, uint16_t bits)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) x[i] = bits;
}

// prod[j] *= 1 - v_p[first + j] for every view p of the batch
__global__ void k_vf_product(const unsigned long long *sumT, const uint32_t *cnt, int nv, int64_t n_all, int64_t first,
                             int64_t n_virt, float *prod)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_virt) return;
    float pr = prod[j];
    for (int v = 0; v < nv; ++v) {
        const size_t r = (size_t)v * (size_t)n_all + (size_t)(first + j);
        const uint32_t c = cnt[r];
        if (c) pr *= 1.0f - (float)sumT[r] * (1.0f / kTScale) / (float)c;
    }
    prod[j] = pr;
}

__global__ void k_density_finalize(const float *prod, int64_t n_virt, float eps_v, float *vis, uint8_t *keep,
                                   uint32_t *keep_u32)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_virt) return;
    const float v = 1.0f - prod[j];
    const bool k = v <= eps_v;   // low visibility: under-explored, kept
    if (vis) vis[j] = v;
    keep[j] = (uint8_t)k;
    keep_u32[j] = (uint32_t)k;
}

__global__ void k_compact_kept(const float *vmeans, const uint32_t *keep_u32, const uint32_t *pos, int64_t n_virt,
                               float *kept_means)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_virt || !keep_u32[j]) return;
    const uint32_t q = pos[j];
    for (int k = 0; k < 3; ++k) kept_means[3 * (size_t)q + k] = vmeans[3 * j + k];
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_emit_records(const uint32_t *counts, const uint32_t *pos, const GeoRec *geo, int nv, int64_t n,
                                int zb, uint32_t zmin, uint64_t *keyA, uint32_t *valA, cudaStream_t s,
                                size_t cap_R, uint32_t *overflow)
{
    const size_t total = (size_t)nv * (size_t)n;
    if (total == 0) return cudaSuccess;
    k_emit_records<<<nblk(total, 256), 256, 0, s>>>(counts, pos, geo, nv, n, zb, zmin, keyA, valA, cap_R, overflow);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_entry_offsets(const uint32_t *warp_off, const uint2 *rect_sorted, const uint32_t *voff, int nv,
                                 uint32_t M, uint32_t *eoff, cudaStream_t s)
{
    if (nv <= 0) return cudaSuccess;
    k_entry_offsets<<<1, 256, 0, s>>>(warp_off, rect_sorted, voff, nv, M, eoff); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather_counts(const uint32_t *valA, const uint32_t *counts, size_t nrec, uint32_t *cnt_sorted,
                                 cudaStream_t s, const unsigned long long *d_nrec)
{
    if (nrec == 0) return cudaSuccess;
    k_gather_counts<<<nblk(nrec, 256), 256, 0, s>>>(valA, counts, nrec, cnt_sorted, d_nrec); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather_rects(const uint32_t *valA, const uint2 *rect, size_t nrec, uint32_t *warp_cnt,
                                uint2 *rect_sorted, cudaStream_t s, const unsigned long long *d_nrec)
{
    if (nrec == 0) return cudaSuccess;
    k_gather_rects<<<nblk(nrec, 256), 256, 0, s>>>(valA, rect, nrec, warp_cnt, rect_sorted, d_nrec); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_emit_tiles(const uint32_t *valA, const uint32_t *off_sorted, size_t nrec, const uint2 *rect,
                              int64_t n, int TW, int TH, uint32_t *keyB, uint32_t *valB, cudaStream_t s,
                              const unsigned long long *d_nrec, size_t cap_M, uint32_t *overflow, int tb,
                              const uint2 *rect_sorted, const uint32_t *warp_off)
{
    if (nrec == 0) return cudaSuccess;
    k_emit_tiles<<<nblk(nrec, 256), 256, 0, s>>>(valA, off_sorted, nrec, rect, n, divu32((uint32_t)n), TW, TH, keyB,
                                                 valB, d_nrec, cap_M, overflow, tb, rect_sorted, warp_off);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t *keys, size_t M, uint2 *ranges, cudaStream_t s, const unsigned long long *d_M,
                          int tb, uint32_t TT)
{
    if (M == 0) return cudaSuccess;
    k_ranges<<<nblk((M + 3) / 4, 256), 256, 0, s>>>(keys, M, ranges, d_M, tb, TT); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_order_keys(const uint2 *ranges, size_t nt, uint32_t *keys, uint32_t *vals, cudaStream_t s)
{
    if (nt == 0) return cudaSuccess;
    k_order_keys<<<nblk(nt, 256), 256, 0, s>>>(ranges, nt, keys, vals); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_keys_export(const uint32_t *keyB, const uint32_t *valB, size_t M, const GeoRec *geo, int64_t n,
                               int tiles_per_view, uint64_t *out, cudaStream_t s, int tb)
{
    if (M == 0) return cudaSuccess;
    k_keys_export<<<nblk(M, 256), 256, 0, s>>>(keyB, valB, M, geo, n, tiles_per_view, out, tb); count_launch();
    return cudaGetLastError();
}

// Persistent grid of the uncertainty pass: as many CTAs as fit on the device
// at once (cached per device and kernel instance), fewer for small batches.
constexpr int kMaxDevices = 64;
struct UaGrid {
    std::atomic<int> ctas[kMaxDevices];
};

template <int TILE, bool KC, bool DEPTH, bool PAIRS>
unsigned ua_resident_ctas()
{
    static UaGrid g;   // zero-initialised: computed on first use per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;
    int c = g.ctas[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        int per_sm = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite_ua<TILE, KC, DEPTH, PAIRS>, kUaWarps * 32,
                                                      0);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        c = (per_sm > 0 ? per_sm : 1) * (nsm > 0 ? nsm : 1);
        g.ctas[dev].store(c, std::memory_order_relaxed);
    }
    return (unsigned)c;
}

template <int TILE, bool KC, bool DEPTH, bool PAIRS>
void launch_ua_inst(const CompositeArgs &a, unsigned long long items, cudaStream_t s)
{
    const unsigned long long want = (items + kUaWarps - 1) / kUaWarps;
    const unsigned cap = ua_resident_ctas<TILE, KC, DEPTH, PAIRS>();
    const unsigned blocks = want < cap ? (unsigned)want : cap;
    k_composite_ua<TILE, KC, DEPTH, PAIRS><<<blocks, kUaWarps * 32, 0, s>>>(a);
}

template <int TILE, bool KC, bool DEPTH>
void launch_ua_pairs(const CompositeArgs &a, unsigned long long items, cudaStream_t s)
{
    if (a.pair_counts) launch_ua_inst<TILE, KC, DEPTH, true>(a, items, s);
    else launch_ua_inst<TILE, KC, DEPTH, false>(a, items, s);
}

template <int TILE>
void launch_ua_tile(const CompositeArgs &a, unsigned long long items, cudaStream_t s)
{
    const bool d = a.depth != nullptr;
    if (a.per_entry_kc) {
        if (d) launch_ua_pairs<TILE, true, true>(a, items, s);
        else launch_ua_pairs<TILE, true, false>(a, items, s);
    } else {
        if (d) launch_ua_pairs<TILE, false, true>(a, items, s);
        else launch_ua_pairs<TILE, false, false>(a, items, s);
    }
    count_launch();
}

template <int TILE>
void prepare_ua_tile()
{
    ua_resident_ctas<TILE, true, true, false>();
    ua_resident_ctas<TILE, true, false, false>();
    ua_resident_ctas<TILE, false, true, false>();
    ua_resident_ctas<TILE, false, false, false>();
    ua_resident_ctas<TILE, true, true, true>();
    ua_resident_ctas<TILE, true, false, true>();
    ua_resident_ctas<TILE, false, true, true>();
    ua_resident_ctas<TILE, false, false, true>();
}

cudaError_t launch_composite_ua(const CompositeArgs &a_in, cudaStream_t s)
{
    const unsigned long long items =
        (unsigned long long)a_in.nv * (unsigned long long)(a_in.TW * a_in.TH) *
        (unsigned long long)blocks_per_tile(a_in.tile);
    if (items == 0) return cudaSuccess;
    // (view, tile) indices are 32-bit in the kernel
    if (!a_in.work || (unsigned long long)a_in.nv * (unsigned long long)(a_in.TW * a_in.TH) >= (1ull << 32))
        return cudaErrorInvalidValue;
    CompositeArgs a = a_in;
    a.div_tiles = divu32((uint32_t)(a.TW * a.TH));
    a.div_TW = divu32((uint32_t)a.TW);
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);   // the work counter
    if (e != cudaSuccess) return e;
    switch (a.tile) {
    case 8: launch_ua_tile<8>(a, items, s); break;
    case 16: launch_ua_tile<16>(a, items, s); break;
    case 32: launch_ua_tile<32>(a, items, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

void composite_prepare(int tile)
{
    if (tile == 8) prepare_ua_tile<8>();
    if (tile == 16) prepare_ua_tile<16>();
    if (tile == 32) prepare_ua_tile<32>();
}

cudaError_t launch_composite_vis(const CompositeArgs &a, cudaStream_t s)
{
    const unsigned blocks = (unsigned)(a.nv * a.TW * a.TH);
    if (blocks == 0) return cudaSuccess;
    // one thread per two pixels of the tile, as the kernel is written for
    switch (a.tile) {
    case 8: k_composite_vis<8><<<blocks, 8 * 8 / 2, 0, s>>>(a); count_launch(); break;
    case 16: k_composite_vis<16><<<blocks, 16 * 16 / 2, 0, s>>>(a); count_launch(); break;
    case 32: k_composite_vis<32><<<blocks, 32 * 32 / 2, 0, s>>>(a); count_launch(); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sum_counts(const uint32_t *c, size_t count, unsigned long long *out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    unsigned blocks = nblk(count, 256);
    if (blocks > 1024) blocks = 1024;
    k_sum_counts<<<blocks, 256, 0, s>>>(c, count, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_view_reduce(const float *tile_sums, int nv, int sums_per_view, float inv_pixels, float *score,
                               cudaStream_t s)
{
    if (nv == 0) return cudaSuccess;
    k_view_reduce<<<nv, 256, 0, s>>>(tile_sums, sums_per_view, inv_pixels, score); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_argmax(const float *score, int n, int32_t *best, cudaStream_t s)
{
    k_argmax<<<1, 1024, 0, s>>>(score, n, best); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vf_accumulate(const AccumArgs &a, cudaStream_t s)
{
    if (a.n == 0 || a.nv == 0) return cudaSuccess;
    const unsigned blocks = nblk((size_t)a.n, 128);
    const size_t smem = sizeof(gavis_camera) * (size_t)a.nv;
    switch (a.L) {
#define GAVIS_ACC_CASE(L)                                                                                   \
    case L:                                                                                                 \
        if (smem > 48 * 1024)                                                                               \
            cudaFuncSetAttribute(k_vf_accumulate<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_vf_accumulate<L><<<blocks, 128, smem, s>>>(a); count_launch();                                                    \
        break;
        GAVIS_ACC_CASE(0) GAVIS_ACC_CASE(1) GAVIS_ACC_CASE(2) GAVIS_ACC_CASE(3) GAVIS_ACC_CASE(4) GAVIS_ACC_CASE(5)
#undef GAVIS_ACC_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_vf_store(const float *gamma32, size_t count, void *out, int dtype, int accumulate, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_vf_store<<<nblk(count, 256), 256, 0, s>>>(gamma32, count, out, dtype, accumulate); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vf_load(const void *in, int dtype, size_t count, float *gamma32, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_vf_load<<<nblk(count, 256), 256, 0, s>>>(in, dtype, count, gamma32); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_virtual_fill(const float *vmeans, int64_t n_virt, float scale, float *means, float *scales,
                                float *rots, float *opac, cudaStream_t s)
{
    if (n_virt == 0) return cudaSuccess;
    k_virtual_fill<<<nblk((size_t)n_virt, 256), 256, 0, s>>>(vmeans, n_virt, scale, means, scales, rots, opac); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(float *x, size_t count, float value, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_fill_f32<<<nblk(count, 256), 256, 0, s>>>(x, count, value); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill_u16(uint16_t *x, size_t count, uint16_t bits, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_fill_u16<<<nblk(count, 256), 256, 0, s>>>(x, count, bits); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vf_product(const unsigned long long *sumT, const uint32_t *cnt, int nv, int64_t n_all, int64_t first,
                              int64_t n_virt, float *prod, cudaStream_t s)
{
    if (n_virt == 0 || nv == 0) return cudaSuccess;
    k_vf_product<<<nblk((size_t)n_virt, 256), 256, 0, s>>>(sumT, cnt, nv, n_all, first, n_virt, prod); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_density_finalize(const float *prod, int64_t n_virt, float eps_v, float *vis, uint8_t *keep,
                                    uint32_t *keep_u32, cudaStream_t s)
{
    if (n_virt == 0) return cudaSuccess;
    k_density_finalize<<<nblk((size_t)n_virt, 256), 256, 0, s>>>(prod, n_virt, eps_v, vis, keep, keep_u32); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_compact_kept(const float *vmeans, const uint32_t *keep_u32, const uint32_t *pos, int64_t n_virt,
                                float *kept_means, cudaStream_t s)
{
    if (n_virt == 0) return cudaSuccess;
    k_compact_kept<<<nblk((size_t)n_virt, 256), 256, 0, s>>>(vmeans, keep_u32, pos, n_virt, kept_means); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vis_export(const unsigned long long *sumT, const uint32_t *cnt, size_t count, float *sumT_f,
                              uint32_t *cnt_out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_vis_export<<<nblk(count, 256), 256, 0, s>>>(sumT, cnt, count, sumT_f, cnt_out); count_launch();
    return cudaGetLastError();
}

}  // namespace gavis
