// gavis_internal.cuh -- shared declarations of the CUDA translation units.
//
// Record layouts (HBM, one entry per (view-in-batch, Gaussian), index v*N + g):
//   GeoRec  32 B  a = (u, v, A, 2B)  b = (C, log2(opacity), depth z, ext)
//           image-space centre and conic of the projected Gaussian (log2 of
//           the opacity, -inf for opacity 0); ext packs the footprint
//           half-extents (ex, ey) as two halves rounded up.
//   UaRec   32 B  a = (a1, a0, V, r)  b = (g, b, kc, 0)
//           alpha* = a1 * alpha + a0 (eq:alpha_comp, a1 = V + beta(1-V),
//           a0 = o0(1-beta)(1-V)), the queried visibility V (eq:vis_bound) and
//           the SH colour (eq:rgb_sh); kc = 1/2 log((2 pi e)^3 |Q_c|) of
//           the Gaussian in that view (eq:huber).
//   rect    8 B   (x0 | x1 << 16, y0 | y1 << 16) inclusive tile rectangle.
//   counts  4 B   tiles touched (0 = culled).
// Canonical order of a batch's tile lists: by key ((view * TW*TH + tile) << 32)
// | float_bits(depth), ties by Gaussian index.  Depths are positive, so their
// bit patterns order like the depths; zmin/zmax are the smallest/largest of
// the batch and zb the bits of zmax - zmin (depth keys are stored minus zmin).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "gavis.h"

namespace gavis {

// number of kernels this library has launched (all contexts)
extern std::atomic<long long> g_launches;
inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
// sets the text gavis_last_error returns
void set_error(gavis_ctx *c, const char *msg);

struct __align__(16) GeoRec {
    float4 a;
    float4 b;
};
struct __align__(16) UaRec {
    float4 a;
    float4 b;
};

// q = floor(x / d) for 32-bit x and a divisor d fixed for a launch, by a
// multiply-high and shifts (Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994: the unsigned case with a 33-bit
// multiplier 2^32 + m).  The host derives m, s1, s2 from d (d >= 1).
struct DivU32 {
    uint32_t m, s1, s2;
};
inline DivU32 divu32(uint32_t d)
{
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < (unsigned long long)d) ++l;   // ceil(log2 d)
    DivU32 r;
    r.m = (uint32_t)((((1ull << l) - (unsigned long long)d) << 32) / (unsigned long long)d + 1ull);
    r.s1 = l < 1 ? l : 1u;
    r.s2 = l > 1 ? l - 1u : 0u;
    return r;
}
__device__ __forceinline__ uint32_t div_u32(uint32_t x, DivU32 d)
{
    const uint32_t t = __umulhi(d.m, x);
    return (t + ((x - t) >> d.s1)) >> d.s2;
}

struct RasterConsts {
    float eps_T, q_cut, beta, o0;
    float k_c;   // 1/2 log|Q_c| + 3/2 log(2 pi e)
    float k_0;   // 1/2 log|Q_0| + 3/2 log(2 pi e)
};

// fixed-point scale of the transmittance sums of the visibility pass: 2^18,
// so that a warp's per-entry sum of 64 pixels' round(T 2^18) shifted left by
// kCntBits, plus their hit count in the low kCntBits bits, fits 32 bits
constexpr float kTScale = 262144.0f;   // 2^18
constexpr int kCntBits = 7;
// views one projection or query launch takes: their cameras sit in shared memory
constexpr int kMaxBatchViews = 1024;
// keys per block of the radix sort passes (one histogram row per block)
constexpr int kRadixTile = 4096;

// ---------------------------------------------------------------- project.cu
struct ProjectArgs {
    const float *means, *scales, *rots, *opac;
    const void *sh;
    int sh_degree, sh_dtype;
    const void *sh_var;     // colour coefficient variances or NULL (constant Q_c)
    float k_c;              // 1/2 log((2 pi e)^3 |Q_c|) for the constant Q_c
    const void *gamma;      // VF coefficients (NULL -> V = 0)
    int vf_degree, vf_dtype, n_train;
    float q_cut, beta, o0;
    int tile, TW, TH;
    const gavis_camera *cams;  // device [nv]
    int nv;
    int64_t n;
    GeoRec *geo;
    UaRec *ua;              // NULL for the visibility pass
    uint2 *rect;
    uint32_t *counts;       // optional: tile count of each visible record (and 0 for culled ones unless vis_words is given)
    uint32_t *vis_words;    // [nv][ceil(n/32)] visibility bits (bit g%32 of word g/32), or NULL
    float *zrec;            // camera depth of each visible record (dense copy of GeoRec b.z), or NULL
    uint32_t *zrange;       // [2] min and max depth bits of visible records (atomic)
    unsigned long long *visible;   // count of visible records (atomic)
    unsigned long long *total;     // count of tile entries (atomic)
};
cudaError_t launch_project(const ProjectArgs &a, cudaStream_t s);

struct QueryArgs {
    const float *means;
    const void *gamma;
    int vf_degree, vf_dtype, n_train;
    const gavis_camera *cams;
    int nv;
    int64_t n;
    float *V;
};
cudaError_t launch_query(const QueryArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- sort.cu
// exclusive scan of n uint32 into out (may alias in); writes the total (u64)
// to *d_total (device).  flags = true scans (in[i] != 0) instead of in[i].
// tmp: scan_tmp_bytes(n) bytes.  d_n (optional): the actual count in device
// memory (<= n); out is then written for the first *d_n items only.
size_t scan_tmp_bytes(size_t n);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, void *tmp,
                               unsigned long long *d_total, cudaStream_t s, bool flags = false,
                               const unsigned long long *d_n = nullptr);

// Stage A from the visibility bits (nv views x nw words, nw = ceil(n/32)):
// scan_vis_words writes woff[w] = visible records before word w (tmp:
// scan_tmp_bytes(nv * nw)); emit_vis_words then writes, for every visible
// record r = v n + g at its position p among the visible records,
// keyA[p] = ((v & vmask) << zb) | (depth bits - zmin) and valA[p] = r, and
// voff[v] = visible records before view v (v = 0..nv).  The depth is read
// from zrec[r] when given (4 B per record), else from the GeoRec.
cudaError_t scan_vis_words(const uint32_t *words, size_t nwords, uint32_t *woff, void *tmp, cudaStream_t s);
cudaError_t emit_vis_words(const uint32_t *words, const uint32_t *woff, int nv, int64_t n, const GeoRec *geo,
                           const float *zrec, int zb, uint32_t zmin, uint32_t vmask, uint32_t *keyA, uint32_t *valA,
                           uint32_t *voff, cudaStream_t s);

// stable LSD radix sort of (keys, vals) on bits [0, end_bit); ping-pong
// buffers; *result_in_alt tells which buffer holds the result.  KeyT is
// uint64_t or uint32_t.
size_t radix_tmp_bytes(size_t n);
// d_n (optional): the actual item count in device memory (<= n), for chains
// captured in a CUDA graph; the grids are sized by n.
template <typename KeyT>
cudaError_t radix_sort_pairs(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, size_t n, int end_bit,
                             void *tmp, bool *result_in_alt, cudaStream_t s,
                             const unsigned long long *d_n = nullptr);
// kernel attributes the sort sets on first use; call before stream capture
void radix_prepare();

// Segmented sort: several contiguous segments sorted independently on the
// same bits in one sequence of passes.  Each thread block of a pass takes the
// items [start, end) of one segment (at most 4096) and digit d's count of
// that block lives at hist[h0 + d hs]; the histograms of consecutive
// segments are concatenated (segment-major, then digit-major, then block),
// so one exclusive scan of all of them gives every (segment, digit, block)
// its global output position.
struct RsBlock {
    uint32_t start, end, h0, hs;
};
// Fills tbl (host; NULL to count) with the blocks of the segments
// [seg[s], seg[s+1]), s < nseg; returns the number of blocks.
size_t radix_segment_blocks(const uint64_t *seg, int nseg, RsBlock *tbl);
// blk: device copy of the table (nblk blocks); tmp: radix_tmp_bytes of
// nblk * 4096 items.
// prepared: the kernel attributes were set beforehand (radix_prepare; needed
// while a stream is being captured).
template <typename KeyT>
cudaError_t radix_sort_segments(KeyT *keys, uint32_t *vals, KeyT *keys_alt, uint32_t *vals_alt, const RsBlock *blk,
                                size_t nblk, int end_bit, void *tmp, bool *result_in_alt, cudaStream_t s,
                                bool prepared = false);

// ---------------------------------------------------------------- raster.cu
struct BatchInfo {                // device, read back once per batch
    unsigned long long total;     // number of tile entries
    uint32_t zrange[2];           // min, max depth bits of visible records
    unsigned long long visible;   // (view, Gaussian) records with tiles
};
// bits needed to represent x
__host__ __device__ inline int bits_of(uint64_t x)
{
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}
// bits of the depth part of the record keys of a batch
__host__ __device__ inline int depth_bits(uint32_t zmin, uint32_t zmax)
{
    return bits_of(zmax > zmin ? zmax - zmin : 0u);
}

// Stage-A key parameters of a batch computed on the device from its
// BatchInfo, for chains captured in a CUDA graph (the batched call computes
// the same on the host): zmin, zb = depth_bits, and view groups of
// gsz = 2^gb views, gb = min(bits(nv - 1), 32 - zb), vmask = gsz - 1.
struct KeyParams {
    uint32_t zmin, vmask;
    int32_t zb, gsz;
};
cudaError_t launch_key_params(const BatchInfo *info, int nv, KeyParams *kp, cudaStream_t s);
// emit_vis_words with the key parameters read from kp (device); records at
// positions >= cap_R are dropped and set *overflow; depths from zrec when
// given (dense, 4 B a record), else from the GeoRec.
cudaError_t emit_vis_words_dev(const uint32_t *words, const uint32_t *woff, int nv, int64_t n, const GeoRec *geo,
                               const float *zrec, const KeyParams *kp, uint32_t *keyA, uint32_t *valA, uint32_t *voff,
                               size_t cap_R, uint32_t *overflow, cudaStream_t s);
// The block table of a segmented sort built on the device (nv <= 1024):
// segment s covers [off[min(s g, nv)], off[min((s + 1) g, nv)]) clamped to
// cap, for groups of g views (g = kp->gsz when kp is given, else gsz),
// s < ceil(nv / g).  All nblk_max entries are written: the live blocks as
// radix_segment_blocks lays them out, then empty blocks whose histogram
// columns follow the live ones.  nblk_max >= radix_segment_blocks_max.
cudaError_t launch_segment_blocks(const uint32_t *off, int nv, const KeyParams *kp, int gsz, size_t cap,
                                  RsBlock *blk, size_t nblk_max, cudaStream_t s);
size_t radix_segment_blocks_max(size_t cap, int nv);
// eoff[v] (v = 0..nv) as launch_entry_offsets, from device counts: records
// past min(visible, cap_R) and entries past min(total, cap_M) are cut off.
cudaError_t launch_entry_offsets_dev(const uint32_t *warp_off, const uint2 *rect_sorted, const uint32_t *voff, int nv,
                                     const BatchInfo *info, size_t cap_R, size_t cap_M, uint32_t *eoff,
                                     cudaStream_t s);
// Two-level binning.  Stage A: one key per visible (view, Gaussian) record,
// ((view << zb) | (depth bits - zmin)), value the record index, sorted.
// Stage B: in that order, one entry per tile of the record's rectangle with
// key view * TW*TH + tile and value g, stably sorted by tile: each tile's list
// ends up in (depth, index) order.
// Records at positions >= cap_R are not written and set *overflow (when given).
cudaError_t launch_emit_records(const uint32_t *counts, const uint32_t *pos, const GeoRec *geo, int nv, int64_t n,
                                int zb, uint32_t zmin, uint64_t *keyA, uint32_t *valA, cudaStream_t s,
                                size_t cap_R = ~(size_t)0, uint32_t *overflow = nullptr);
// eoff[v] (v = 0..nv) = stage-B tile entries of the views before v: record
// voff[v]'s first entry, from the per-warp offsets (warp_off, of
// launch_gather_rects) and the rectangles of the warp's earlier records
// (rect_sorted); voff is device [nv + 1].
cudaError_t launch_entry_offsets(const uint32_t *warp_off, const uint2 *rect_sorted, const uint32_t *voff, int nv,
                                 uint32_t M, uint32_t *eoff, cudaStream_t s);
// d_nrec / d_M (optional): actual counts in device memory for graph replays;
// entries past cap_M are not written and set *overflow (when given).
cudaError_t launch_gather_counts(const uint32_t *valA, const uint32_t *counts, size_t nrec, uint32_t *cnt_sorted,
                                 cudaStream_t s, const unsigned long long *d_nrec = nullptr);
// rect_sorted[i] = rect[valA[i]] (one gather of the rectangle, in stage-A
// order) and warp_cnt[w] = the tiles of records [32 w, 32 w + 32), for
// ceil(nrec / 32) warps (0 past the live records); an exclusive scan of
// warp_cnt gives the warps' first tile entries (the warp_off of
// launch_emit_tiles).
cudaError_t launch_gather_rects(const uint32_t *valA, const uint2 *rect, size_t nrec, uint32_t *warp_cnt,
                                uint2 *rect_sorted, cudaStream_t s, const unsigned long long *d_nrec = nullptr);
// tb: tile keys are v * TT + tile (tb < 0) or (v << tb) | tile (2^tb >= TT),
// which lets a group of 2^g views be sorted on its low tb + g bits.
// rect_sorted (optional): the rectangles in stage-A order (read in order
// instead of gathered from rect).  warp_off (optional): the first tile entry
// of each warp's 32 records, used instead of off_sorted.
cudaError_t launch_emit_tiles(const uint32_t *valA, const uint32_t *off_sorted, size_t nrec, const uint2 *rect,
                              int64_t n, int TW, int TH, uint32_t *keyB, uint32_t *valB, cudaStream_t s,
                              const unsigned long long *d_nrec = nullptr, size_t cap_M = ~(size_t)0,
                              uint32_t *overflow = nullptr, int tb = -1, const uint2 *rect_sorted = nullptr,
                              const uint32_t *warp_off = nullptr);
cudaError_t launch_ranges(const uint32_t *keys, size_t M, uint2 *ranges, cudaStream_t s,
                          const unsigned long long *d_M = nullptr, int tb = -1, uint32_t TT = 0);
// canonical keys ((view*tiles + tile) << 32) | depth bits, for verification
cudaError_t launch_keys_export(const uint32_t *keyB, const uint32_t *valB, size_t M, const GeoRec *geo, int64_t n,
                               int tiles_per_view, uint64_t *out, cudaStream_t s, int tb = -1);

// ---------------------------------------------------------------- bin.cu
// Stage B by counting (no sort of the tile entries): the lists of every
// (view, tile) of a batch, records in stage-A order, from the rectangles of
// the stage-A-ordered records.  Each view's records go in chunks of
// kBinChunk to one warp, whose per-tile counters live in shared memory, so
// views of up to kBinMaxTiles tiles take this path; larger ones the sort.
// A warp walks its chunk serially, so a batch needs many chunks to fill the
// GPU: the automatic choice takes this path from kBinMinRecords visible
// records a batch (a batch of a few thousand records a view is faster sorted).
constexpr int kBinChunk = 1024;
constexpr int kBinMaxTiles = 2048;
constexpr int kBinMinRecords = 1 << 20;
inline bool bin_by_counting(int TT) { return TT >= 1 && TT <= kBinMaxTiles; }
struct BinLayout {
    uint32_t *roff;        // [nv + 1] records before each view (clamped to the live records)
    uint32_t *chunk_off;   // [nv + 1] chunks before each view
    uint32_t *table;       // [chunks][TT] per-chunk tile counts, then their prefix over the view's chunks
    uint32_t *tile_tot;    // [nv * TT] list lengths
    uint32_t *tile_start;  // [nv * TT] list starts
    void *scan_tmp;
    size_t bytes;
};
// the most chunks cap_R records of nv views can make
size_t bin_chunks_max(size_t cap_R, int nv);
BinLayout bin_layout(void *base, size_t cap_R, int nv, int TT);
// kernel attributes (shared memory above 48 KB); call before stream capture
void bin_prepare();
// recs: record indices v n + g in stage-A order, rect_sorted their
// rectangles, voff[v] (v = 0..nv) the records before view v.  The live
// records are min(cap_R, *d_nrec) (d_nrec optional).  Writes ranges[v TT +
// t] and vals (the Gaussian index of every entry); entries at positions >=
// cap_M are not written and set *overflow, and the ranges are cut off there.
cudaError_t launch_bin_tiles(const uint32_t *recs, const uint2 *rect_sorted, const uint32_t *voff, int nv, int64_t n,
                             int TW, int TT, size_t cap_R, const unsigned long long *d_nrec, const BinLayout &B,
                             uint2 *ranges, uint32_t *vals, size_t cap_M, uint32_t *overflow, cudaStream_t s);
// canonical keys ((view * TT + tile) << 32) | depth bits of the lists'
// entries, at the entries' positions (those below cap)
cudaError_t launch_keys_from_ranges(const uint2 *ranges, const uint32_t *vals, int nv, int TT, const GeoRec *geo,
                                    int64_t n, size_t cap, uint64_t *out, cudaStream_t s);

struct CompositeArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const GeoRec *geo;
    const UaRec *ua;
    int64_t n;
    int nv, v0;            // views in batch, global index of the first
    int W, H, tile, TW, TH;
    RasterConsts rc;
    float *rgb, *unc;      // may be NULL
    float *depth;          // expected depth (sum of colour weight x camera depth) or NULL
    float *tile_sums;      // [nv * TW*TH * blocks_per_tile(tile)]: entropy sum of each 8 x 8 pixel block
    unsigned long long *work;  // uncertainty pass: its work counter (one word, reset by the launch)
    const uint32_t *order;     // uncertainty pass: (view, tile) indices, longest lists first, or NULL (natural order)
    bool per_entry_kc;     // use the per-Gaussian kc of the UaRec (colour variances given)
    // visibility pass
    unsigned long long *sumT;  // [nv * n] fixed point 2^-18 (kTScale)
    uint32_t *cnt;             // [nv * n]
    // optional instrumentation: (pixel, Gaussian) pairs composited; the
    // uncertainty pass writes one count per 8 x 8 block, like tile_sums (summed by launch_sum_counts),
    // the visibility pass adds per warp into *pairs
    uint32_t *pair_counts;
    unsigned long long *pairs;
    // set by the uncertainty pass's launcher: division by the tiles of a view and by TW
    DivU32 div_tiles, div_TW;
};
// 8 x 8 pixel blocks per tile: the uncertainty pass's work items
__host__ __device__ constexpr int blocks_per_tile(int tile) { return (tile / 8) * (tile / 8); }
cudaError_t launch_composite_ua(const CompositeArgs &a, cudaStream_t s);
// occupancy queries of the uncertainty pass for a tile size, ahead of a stream capture
void composite_prepare(int tile);
// Order of the uncertainty pass's tiles: keys[t] = 255 - min(list length / 16, 255),
// vals[t] = t for the nt (view, tile) ranges; sorted stably on the 8 key bits
// (one radix pass) the values list the longest lists first.
cudaError_t launch_order_keys(const uint2 *ranges, size_t nt, uint32_t *keys, uint32_t *vals, cudaStream_t s);
cudaError_t launch_composite_vis(const CompositeArgs &a, cudaStream_t s);
cudaError_t launch_sum_counts(const uint32_t *c, size_t count, unsigned long long *out, cudaStream_t s);
cudaError_t launch_view_reduce(const float *tile_sums, int nv, int sums_per_view, float inv_pixels,
                               float *score, cudaStream_t s);
cudaError_t launch_argmax(const float *score, int n, int32_t *best, cudaStream_t s);

struct AccumArgs {
    const float *means;
    const gavis_camera *cams;   // device [nv]
    int nv;
    int64_t n;
    const unsigned long long *sumT;
    const uint32_t *cnt;
    float a_l[6];               // a_l for l = 0..L (L <= 5)
    int L;
    float *gamma32;             // [n * K], accumulated in place
};
cudaError_t launch_vf_accumulate(const AccumArgs &a, cudaStream_t s);
cudaError_t launch_vf_store(const float *gamma32, size_t count, void *out, int dtype, int accumulate,
                            cudaStream_t s);
cudaError_t launch_vf_load(const void *in, int dtype, size_t count, float *gamma32, cudaStream_t s);
// density control
cudaError_t launch_virtual_fill(const float *vmeans, int64_t n_virt, float scale, float *means, float *scales,
                                float *rots, float *opac, cudaStream_t s);
cudaError_t launch_fill_f32(float *x, size_t count, float value, cudaStream_t s);
cudaError_t launch_fill_u16(uint16_t *x, size_t count, uint16_t bits, cudaStream_t s);
cudaError_t launch_vf_product(const unsigned long long *sumT, const uint32_t *cnt, int nv, int64_t n_all,
                              int64_t first, int64_t n_virt, float *prod, cudaStream_t s);
cudaError_t launch_density_finalize(const float *prod, int64_t n_virt, float eps_v, float *vis, uint8_t *keep,
                                    uint32_t *keep_u32, cudaStream_t s);
cudaError_t launch_compact_kept(const float *vmeans, const uint32_t *keep_u32, const uint32_t *pos, int64_t n_virt,
                                float *kept_means, cudaStream_t s);
cudaError_t launch_vis_export(const unsigned long long *sumT, const uint32_t *cnt, size_t count, float *sumT_f,
                              uint32_t *cnt_out, cudaStream_t s);

}  // namespace gavis
