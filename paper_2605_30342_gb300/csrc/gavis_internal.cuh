// gavis_internal.cuh -- shared declarations of the CUDA translation units.
//
// Record layouts (HBM, one entry per (view-in-batch, Gaussian), index v*N + g):
//   GeoRec  32 B  a = (u, v, A, 2B)  b = (C, opacity, depth z, ext)
//           image-space centre and conic of the projected Gaussian; ext packs
//           the footprint half-extents (ex, ey) as two halves rounded up.
//   UaRec   32 B  a = (a1, a0, V, r)  b = (g, b, 0, 0)
//           alpha* = a1 * alpha + a0 (eq:alpha_comp, a1 = V + beta(1-V),
//           a0 = o0(1-beta)(1-V)), the queried visibility V (eq:vis_bound) and
//           the SH colour (eq:rgb_sh).
//   rect    8 B   (x0 | x1 << 16, y0 | y1 << 16) inclusive tile rectangle.
//   counts  4 B   tiles touched (0 = culled).
// Keys: ((view * TW*TH + tile) << zb) | (float_bits(depth) - zmin); values: g.
// zmin/zmax are the smallest/largest depth bit patterns of the batch (depths
// are positive, so their bit patterns order like the depths) and zb the bits
// of zmax - zmin: the canonical key ((view * TW*TH + tile) << 32) |
// float_bits(depth) orders exactly like this compacted one, which needs fewer
// radix passes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "gavis.h"

namespace gavis {

// number of kernels this library has launched (all contexts)
extern std::atomic<long long> g_launches;
inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

struct __align__(16) GeoRec {
    float4 a;
    float4 b;
};
struct __align__(16) UaRec {
    float4 a;
    float4 b;
};

struct RasterConsts {
    float eps_T, q_cut, beta, o0;
    float k_c;   // 1/2 log|Q_c| + 3/2 log(2 pi e)
    float k_0;   // 1/2 log|Q_0| + 3/2 log(2 pi e)
};

// fixed-point scale of the transmittance sums of the visibility pass
constexpr float kTScale = 16777216.0f;   // 2^24

// ---------------------------------------------------------------- project.cu
struct ProjectArgs {
    const float *means, *scales, *rots, *opac;
    const void *sh;
    int sh_degree, sh_dtype;
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
    uint32_t *counts;
    uint32_t *zrange;       // [2] min and max depth bits of visible records (atomic)
    unsigned long long *visible;   // count of visible records (atomic), or NULL
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
// to *d_total (device).  tmp: scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(size_t n);
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, void *tmp,
                               unsigned long long *d_total, cudaStream_t s);

// stable LSD radix sort of (keys, vals) on bits [0, end_bit); ping-pong
// buffers; *result_in_alt tells which buffer holds the result.
size_t radix_tmp_bytes(size_t n);
cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                             size_t n, int end_bit, void *tmp, bool *result_in_alt, cudaStream_t s);

// ---------------------------------------------------------------- raster.cu
struct BatchInfo {                // device, read back once per batch
    unsigned long long total;     // number of keys
    uint32_t zrange[2];           // min, max depth bits of visible records
    unsigned long long visible;   // (view, Gaussian) records with tiles
};
// key compaction of a batch: bits of the depth part
inline int depth_bits(uint32_t zmin, uint32_t zmax)
{
    int b = 0;
    const uint32_t d = zmax > zmin ? zmax - zmin : 0u;
    while (b < 32 && (d >> b) != 0u) ++b;
    return b;
}
cudaError_t launch_emit(const uint2 *rect, const GeoRec *geo, const uint32_t *counts, const uint32_t *offsets,
                        int nv, int64_t n, int TW, int TH, int zb, uint32_t zmin, uint64_t *keys, uint32_t *vals,
                        cudaStream_t s);
cudaError_t launch_ranges(const uint64_t *keys, size_t M, int zb, uint2 *ranges, cudaStream_t s);
// canonical keys ((tile << 32) | depth bits) from compacted ones
cudaError_t launch_keys_export(const uint64_t *keys, size_t M, int zb, uint32_t zmin, uint64_t *out,
                               cudaStream_t s);

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
    float *tile_sums;      // [nv * TW*TH]
    // visibility pass
    unsigned long long *sumT;  // [nv * n] fixed point 2^-24
    uint32_t *cnt;             // [nv * n]
    // optional instrumentation: (pixel, Gaussian) pairs composited
    unsigned long long *pairs;
};
cudaError_t launch_composite_ua(const CompositeArgs &a, cudaStream_t s);
cudaError_t launch_composite_vis(const CompositeArgs &a, cudaStream_t s);
cudaError_t launch_view_reduce(const float *tile_sums, int nv, int tiles_per_view, float inv_pixels,
                               float *score, cudaStream_t s);
cudaError_t launch_argmax(const float *score, int n, int32_t *best, cudaStream_t s);

struct AccumArgs {
    const float *means;
    const gavis_camera *cams;   // device [nv]
    int nv;
    int64_t n;
    const unsigned long long *sumT;
    const uint32_t *cnt;
    float a_l[4];
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
cudaError_t launch_vf_product(const unsigned long long *sumT, const uint32_t *cnt, int nv, int64_t n_all,
                              int64_t first, int64_t n_virt, float *prod, cudaStream_t s);
cudaError_t launch_density_finalize(const float *prod, int64_t n_virt, float eps_v, float *vis, uint8_t *keep,
                                    uint32_t *keep_u32, cudaStream_t s);
cudaError_t launch_compact_kept(const float *vmeans, const uint32_t *keep_u32, const uint32_t *pos, int64_t n_virt,
                                float *kept_means, cudaStream_t s);
cudaError_t launch_vis_export(const unsigned long long *sumT, const uint32_t *cnt, size_t count, float *sumT_f,
                              uint32_t *cnt_out, cudaStream_t s);

}  // namespace gavis
