// noalloc.cu -- single-view candidate scoring that allocates no memory.
//
// Some callers cannot call cudaMalloc: an application whose memory manager has
// already reserved the GPU's memory for its own pool (so a raw allocation
// fails or fragments that pool), or a real-time planning loop in which the
// device-wide synchronisation that cudaMalloc/cudaFree may imply is not
// acceptable.  gavis_score_view_noalloc serves them: it runs the same kernels
// as gavis_score_views for one candidate view, but all its scratch memory
// (per-Gaussian records, tile keys and their sort buffers, tile ranges) is a
// file-scope device array of fixed size, so the call performs no allocation
// of any kind (no cudaMalloc, no cudaMallocHost, no library allocator).
//
// The array is part of the module image: every GPU that loads this library
// holds it (kNoAllocScratchBytes) until the process exits.  All calls on one
// device share it and it keeps the last call's contents; calls whose GPU work
// overlaps (different streams, or different host threads) race on it.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gavis_internal.cuh"

namespace gavis {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int64_t kMaxGaussians = 32768;
constexpr int kMaxTiles = 4096;                             // e.g. 1024 x 1024 pixels at tile 16
constexpr size_t kMaxKeys = (size_t)1 << 19;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of g_noalloc_scratch per device, cached once it was obtained
// (a failed lookup is not cached: the next call tries again)
std::mutex g_dev_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

int report(char *err, size_t len, int code, const char *fmt, ...)
{
    if (err && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, len, fmt, ap);
        va_end(ap);
    }
    return code;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// carves consecutive 256-byte aligned regions out of the scratch array
struct Carver {
    unsigned char *base;
    size_t off = 0;
    void *take(size_t bytes)
    {
        void *p = base + off;
        off += up256(bytes ? bytes : 1);
        return p;
    }
};

}  // namespace
}  // namespace gavis

using namespace gavis;

#define NA_CK(call)                                                                                        \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return report(err, err_len, GAVIS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

extern "C" int gavis_score_view_noalloc(const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cam,
                                        const gavis_params *p, float *rgb, float *unc, float *score, char *err,
                                        size_t err_len, void *stream)
{
    if (err && err_len) err[0] = '\0';
    if (!gs || !vf || !cam || !p || !score)
        return report(err, err_len, GAVIS_ERR_ARG, "NULL argument");
    if (gs->n < 0 || gs->n > kMaxGaussians)
        return report(err, err_len, GAVIS_ERR_ARG, "n = %lld Gaussians exceeds the no-allocation maximum of %lld",
                      (long long)gs->n, (long long)kMaxGaussians);
    if (gs->n > 0 && (!gs->means || !gs->scales || !gs->rots || !gs->opac || !gs->sh))
        return report(err, err_len, GAVIS_ERR_ARG, "NULL Gaussian array");
    if (gs->n > 0 && ((uintptr_t)gs->rots & 15u)) return report(err, err_len, GAVIS_ERR_ARG, "rots must be 16-byte aligned");
    if (gs->sh_degree < 0 || gs->sh_degree > 3 || gs->sh_dtype < 0 || gs->sh_dtype > 2)
        return report(err, err_len, GAVIS_ERR_ARG, "bad colour SH degree or dtype");
    if (vf->n != gs->n || vf->degree < 0 || vf->degree > 5 || vf->dtype < 0 || vf->dtype > 2 ||
        vf->n_train_views < 0 || (vf->n > 0 && !vf->coeffs))
        return report(err, err_len, GAVIS_ERR_ARG, "bad visibility field");
    if (!(p->tile == 8 || p->tile == 16 || p->tile == 32) || !(p->eps_T > 0.0f && p->eps_T < 1.0f) ||
        !(p->q_cut > 0.0f) || !(p->sigma_c2 > 0.0f) || !(p->beta >= 0.0f && p->beta <= 1.0f) ||
        !(p->o0 >= 0.0f && p->o0 <= 1.0f))
        return report(err, err_len, GAVIS_ERR_ARG, "bad parameters");
    if (cam->W <= 0 || cam->H <= 0 || cam->W > 16384 || cam->H > 16384 || !(cam->fx > 0.0f) || !(cam->fy > 0.0f) ||
        !(cam->znear > 0.0f))
        return report(err, err_len, GAVIS_ERR_ARG, "bad camera");
    const int TW = (cam->W + p->tile - 1) / p->tile, TH = (cam->H + p->tile - 1) / p->tile, TT = TW * TH;
    if (TT > kMaxTiles)
        return report(err, err_len, GAVIS_ERR_ARG, "%d tiles exceed the no-allocation maximum of %d", TT, kMaxTiles);

    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return report(err, err_len, GAVIS_ERR_ARG, "device index %d too large", dev);
    // first successful call per device, with that device current: the device
    // address of the array (host code cannot use the symbol itself)
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (!g_dev_ptr[dev]) {
            void *q = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
            if (e != cudaSuccess || !q) {
                cudaGetLastError();
                return report(err, err_len, GAVIS_ERR_CUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            }
            g_dev_ptr[dev] = reinterpret_cast<unsigned char *>(q);
        }
        base = g_dev_ptr[dev];
    }

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)cam->W * (size_t)cam->H;
    if (gs->n == 0) {   // empty scene: empty lists everywhere
        if (rgb) NA_CK(cudaMemsetAsync(rgb, 0, 3 * plane * sizeof(float), s));
        if (unc) NA_CK(cudaMemsetAsync(unc, 0, plane * sizeof(float), s));
        NA_CK(cudaMemsetAsync(score, 0, sizeof(float), s));
        return GAVIS_OK;
    }

    const size_t n = (size_t)gs->n;
    Carver c{base};
    gavis_camera *d_cam = reinterpret_cast<gavis_camera *>(c.take(sizeof(gavis_camera)));
    BatchInfo *d_info = reinterpret_cast<BatchInfo *>(c.take(sizeof(BatchInfo)));
    GeoRec *geo = reinterpret_cast<GeoRec *>(c.take(n * sizeof(GeoRec)));
    UaRec *ua = reinterpret_cast<UaRec *>(c.take(n * sizeof(UaRec)));
    uint2 *rect = reinterpret_cast<uint2 *>(c.take(n * sizeof(uint2)));
    uint32_t *counts = reinterpret_cast<uint32_t *>(c.take(n * sizeof(uint32_t)));
    uint32_t *pos = reinterpret_cast<uint32_t *>(c.take(n * sizeof(uint32_t)));
    void *scan_tmp = c.take(scan_tmp_bytes(n));
    uint2 *ranges = reinterpret_cast<uint2 *>(c.take((size_t)TT * sizeof(uint2)));
    const int bpt = blocks_per_tile(p->tile);
    float *tile_sums = reinterpret_cast<float *>(c.take((size_t)TT * (size_t)bpt * sizeof(float)));
    unsigned long long *work = reinterpret_cast<unsigned long long *>(c.take(sizeof(unsigned long long)));
    if (c.off > kNoAllocScratchBytes)
        return report(err, err_len, GAVIS_ERR_BUDGET, "scratch layout exceeds %zu bytes", kNoAllocScratchBytes);

    NA_CK(cudaMemcpyAsync(d_cam, cam, sizeof(gavis_camera), cudaMemcpyHostToDevice, s));
    ProjectArgs pa{};
    pa.means = gs->means; pa.scales = gs->scales; pa.rots = gs->rots; pa.opac = gs->opac;
    pa.sh = gs->sh; pa.sh_degree = gs->sh_degree; pa.sh_dtype = gs->sh_dtype;
    pa.sh_var = gs->sh_var;
    pa.k_c = (float)(1.5 * std::log((double)p->sigma_c2) + 1.5 * (std::log(2.0 * M_PI) + 1.0));
    pa.gamma = vf->coeffs; pa.vf_degree = vf->degree; pa.vf_dtype = vf->dtype; pa.n_train = vf->n_train_views;
    pa.q_cut = p->q_cut; pa.beta = p->beta; pa.o0 = p->o0;
    pa.tile = p->tile; pa.TW = TW; pa.TH = TH;
    pa.cams = d_cam; pa.nv = 1; pa.n = gs->n;
    pa.geo = geo; pa.ua = ua; pa.rect = rect; pa.counts = counts;
    pa.zrange = d_info->zrange;
    pa.visible = &d_info->visible;
    pa.total = &d_info->total;
    // what must start at fixed values: the counters (0) and the depth minimum (all ones)
    NA_CK(cudaMemsetAsync(d_info, 0, sizeof(BatchInfo), s));
    NA_CK(cudaMemsetAsync(&d_info->zrange[0], 0xff, sizeof(uint32_t), s));
    NA_CK(launch_project(pa, s));
    NA_CK(exclusive_scan_u32(counts, pos, n, scan_tmp, nullptr, s, true));
    BatchInfo info;   // pageable host variable: no pinned allocation
    NA_CK(cudaMemcpyAsync(&info, d_info, sizeof(info), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    const unsigned long long M = info.total, nrec = info.visible;
    const uint32_t zmin = info.zrange[0];
    const int zb = nrec ? depth_bits(zmin, info.zrange[1]) : 0;
    if (M > kMaxKeys)
        return report(err, err_len, GAVIS_ERR_BUDGET, "%llu tile entries exceed the no-allocation maximum of %zu", M,
                      kMaxKeys);
    uint64_t *a_k0 = reinterpret_cast<uint64_t *>(c.take(nrec * 8));
    uint64_t *a_k1 = reinterpret_cast<uint64_t *>(c.take(nrec * 8));
    uint32_t *a_v0 = reinterpret_cast<uint32_t *>(c.take(nrec * 4));
    uint32_t *a_v1 = reinterpret_cast<uint32_t *>(c.take(nrec * 4));
    uint32_t *a_cnt = reinterpret_cast<uint32_t *>(c.take(nrec * 4));
    uint32_t *a_off = reinterpret_cast<uint32_t *>(c.take(nrec * 4));
    uint32_t *b_k0 = reinterpret_cast<uint32_t *>(c.take(M * 4));
    uint32_t *b_k1 = reinterpret_cast<uint32_t *>(c.take(M * 4));
    uint32_t *b_v0 = reinterpret_cast<uint32_t *>(c.take(M * 4));
    uint32_t *b_v1 = reinterpret_cast<uint32_t *>(c.take(M * 4));
    const size_t big = nrec > M ? (size_t)nrec : (size_t)M;
    void *rtmp = c.take(radix_tmp_bytes(big) + scan_tmp_bytes(big) + 64);
    if (c.off > kNoAllocScratchBytes)
        return report(err, err_len, GAVIS_ERR_BUDGET, "tile entries do not fit the %zu-byte scratch array",
                      kNoAllocScratchBytes);
    bool alt_a = false, alt_b = false;
    NA_CK(launch_emit_records(counts, pos, geo, 1, gs->n, zb, zmin, a_k0, a_v0, s));
    NA_CK(radix_sort_pairs<uint64_t>(a_k0, a_v0, a_k1, a_v1, (size_t)nrec, zb, rtmp, &alt_a, s));
    const uint32_t *recs = alt_a ? a_v1 : a_v0;
    NA_CK(launch_gather_counts(recs, counts, (size_t)nrec, a_cnt, s));
    NA_CK(exclusive_scan_u32(a_cnt, a_off, (size_t)nrec, rtmp, nullptr, s));
    NA_CK(launch_emit_tiles(recs, a_off, (size_t)nrec, rect, gs->n, TW, TH, b_k0, b_v0, s));
    NA_CK(radix_sort_pairs<uint32_t>(b_k0, b_v0, b_k1, b_v1, (size_t)M, bits_of((uint64_t)TT - 1), rtmp, &alt_b, s));
    const uint32_t *keys = alt_b ? b_k1 : b_k0;
    const uint32_t *vals = alt_b ? b_v1 : b_v0;
    NA_CK(cudaMemsetAsync(ranges, 0, (size_t)TT * sizeof(uint2), s));   // tiles without entries stay empty
    NA_CK(launch_ranges(keys, (size_t)M, ranges, s));

    CompositeArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.ranges = ranges; ca.vals = vals; ca.geo = geo; ca.ua = ua;
    ca.n = gs->n; ca.nv = 1; ca.v0 = 0; ca.W = cam->W; ca.H = cam->H; ca.tile = p->tile; ca.TW = TW; ca.TH = TH;
    ca.rc.eps_T = p->eps_T;
    ca.rc.q_cut = p->q_cut;
    ca.rc.beta = p->beta;
    ca.rc.o0 = p->o0;
    const double l2pie = std::log(2.0 * M_PI) + 1.0;
    ca.rc.k_c = (float)(1.5 * std::log((double)p->sigma_c2) + 1.5 * l2pie);
    ca.rc.k_0 = (float)(0.5 * (double)p->logdet_Q0 + 1.5 * l2pie);
    ca.rgb = rgb; ca.unc = unc; ca.tile_sums = tile_sums; ca.work = work;
    ca.per_entry_kc = gs->sh_var != nullptr;
    NA_CK(launch_composite_ua(ca, s));
    NA_CK(launch_view_reduce(tile_sums, 1, TT * bpt, 1.0f / ((float)cam->W * (float)cam->H), score, s));
    return GAVIS_OK;
}
