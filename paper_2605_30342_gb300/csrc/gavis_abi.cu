// gavis_abi.cu -- host side of the C ABI declared in include/gavis.h.
//
// Every entry point validates its arguments, then runs the kernel chain on the
// caller's stream in batches of views:
//
//   project (+ VF query + colour)  ->  exclusive scan of tile counts  ->
//   [sync: read the key count]  ->  emit keys  ->  radix sort  ->  ranges  ->
//   composite (uncertainty + colour, or particle visibility)  ->  reductions
//
// The batch size is the number of views whose per-(view, Gaussian) records fit
// in the context's workspace budget; if a batch's keys do not fit, the batch is
// halved and re-run.  Nothing here runs the method on the host: the host only
// sizes buffers, copies camera records and launches kernels.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gavis_internal.cuh"
#include "sh_basis.cuh"

using namespace gavis;

std::atomic<long long> gavis::g_launches{0};

namespace {

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

struct gavis_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    std::string err;
    // the workspace comes from this context's own stream-ordered pool, so that
    // growing a buffer never waits for the device (nor for other contexts)
    cudaMemPool_t mem = nullptr;
    Buf rec, vis, keys, small, gamma, cams, aug, tune;
    BatchInfo *h_info = nullptr;             // pinned
    uint32_t *h_voff = nullptr;              // pinned, per-view record offsets of a batch
    size_t h_voff_cap = 0;
    RsBlock *h_blk = nullptr;                // pinned, block table of a segmented sort
    size_t h_blk_cap = 0;
    int32_t *h_best = nullptr;               // pinned
    // instrumentation
    bool prof_on = false;     // stage events
    bool prof_pairs = false;  // and the composited pairs (device counters in the composites)
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[GAVIS_STAGE_COUNT] = {};
    long long prof_launches[GAVIS_STAGE_COUNT] = {};
    unsigned long long *d_pairs = nullptr;   // device [2]
    unsigned long long prof_keys = 0;        // tile entries since gavis_prof_enable
    unsigned long long prof_visible = 0;     // visible (view, Gaussian) records since then
    unsigned long long prof_sorted = 0;      // tile entries whose lists were built by sorting
    // end of the last call's GPU work, for ordering the next call after it
    cudaEvent_t tail = nullptr;
    cudaStream_t tail_stream = nullptr;
    bool tail_set = false;
};

// Calls on one context share its workspace, so their GPU work must not
// overlap: a call on another stream than the previous call's first makes its
// stream wait for that call's end, and every call records its own end.
struct CallOrder {
    gavis_ctx *c;
    cudaStream_t s;
    CallOrder(gavis_ctx *ctx, cudaStream_t st) : c(ctx), s(st)
    {
        if (c->tail && c->tail_set && c->tail_stream != s) cudaStreamWaitEvent(s, c->tail, 0);
    }
    ~CallOrder()
    {
        if (c->tail && cudaEventRecord(c->tail, s) == cudaSuccess) {
            c->tail_stream = s;
            c->tail_set = true;
        }
    }
};

namespace {

int fail(gavis_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(ctx, GAVIS_ERR_CUDA, "%s: %s (%s:%d)", #call,                  \
                                           cudaGetErrorString(e_), __FILE__, __LINE__);                   \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Grow-only device buffer within the context budget, in stream order on s:
// the old buffer is released once the work queued on s before this point
// has run, and the new one is ready for the work queued after it (every call
// on a context runs after the previous one, see CallOrder).  No device-wide
// synchronisation.
int ensure(gavis_ctx *ctx, Buf &b, size_t bytes, cudaStream_t s)
{
    bytes = align256(bytes ? bytes : 256);
    if (b.cap >= bytes) return GAVIS_OK;
    const size_t other = ctx->used - b.cap;
    if (other + bytes > ctx->budget)
        return fail(ctx, GAVIS_ERR_BUDGET, "workspace of %zu bytes exceeds the budget (%zu used of %zu)", bytes,
                    other, ctx->budget);
    if (b.p) {
        CK(cudaFreeAsync(b.p, s));
        b.p = nullptr;
        ctx->used -= b.cap;
        b.cap = 0;
    }
    cudaError_t e = cudaMallocFromPoolAsync(&b.p, bytes, ctx->mem, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(ctx, GAVIS_ERR_OOM, "cudaMallocFromPoolAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.cap = bytes;
    ctx->used += bytes;
    return GAVIS_OK;
}

cudaEvent_t take_event(gavis_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records the device time and launch count of one stage (RAII scope).
struct Stage {
    gavis_ctx *ctx;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    long long l0;
    Stage(gavis_ctx *c, int st, cudaStream_t str) : ctx(c), stage(st), s(str), l0(g_launches.load())
    {
        if (ctx->prof_on) {
            a = take_event(ctx);
            cudaEventRecord(a, s);
        }
    }
    ~Stage()
    {
        if (ctx->prof_on) {
            ctx->prof_launches[stage] += g_launches.load() - l0;
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, s);
            ctx->pending.push_back({stage, a, b});
        }
    }
};

bool is_pow2_tile(int t) { return t == 8 || t == 16 || t == 32; }

int check_params(gavis_ctx *ctx, const gavis_params *p)
{
    if (!p) return fail(ctx, GAVIS_ERR_ARG, "params is NULL");
    if (!is_pow2_tile(p->tile)) return fail(ctx, GAVIS_ERR_ARG, "tile must be 8, 16 or 32 (got %d)", p->tile);
    if (!(p->eps_T > 0.0f && p->eps_T < 1.0f)) return fail(ctx, GAVIS_ERR_ARG, "eps_T must be in (0,1)");
    if (!(p->q_cut > 0.0f)) return fail(ctx, GAVIS_ERR_ARG, "q_cut must be > 0");
    if (!(p->beta >= 0.0f && p->beta <= 1.0f)) return fail(ctx, GAVIS_ERR_ARG, "beta must be in [0,1]");
    if (!(p->o0 >= 0.0f && p->o0 <= 1.0f)) return fail(ctx, GAVIS_ERR_ARG, "o0 must be in [0,1]");
    if (!(p->sigma_c2 > 0.0f)) return fail(ctx, GAVIS_ERR_ARG, "sigma_c2 must be > 0");
    if (!(p->kappa >= 0.0f)) return fail(ctx, GAVIS_ERR_ARG, "kappa must be >= 0");
    if (p->views_per_batch < 0) return fail(ctx, GAVIS_ERR_ARG, "views_per_batch must be >= 0");
    if (p->tile_lists < 0 || p->tile_lists > 2) return fail(ctx, GAVIS_ERR_ARG, "tile_lists must be 0, 1 or 2");
    return GAVIS_OK;
}

int check_gaussians(gavis_ctx *ctx, const gavis_gaussians *gs, bool need_sh)
{
    if (!gs) return fail(ctx, GAVIS_ERR_ARG, "gaussians is NULL");
    if (gs->n < 0 || gs->n >= (int64_t)1 << 31) return fail(ctx, GAVIS_ERR_ARG, "n out of range");
    if (gs->n > 0 && (!gs->means || !gs->scales || !gs->rots || !gs->opac))
        return fail(ctx, GAVIS_ERR_ARG, "NULL Gaussian array");
    if (need_sh) {
        if (gs->sh_degree < 0 || gs->sh_degree > 3) return fail(ctx, GAVIS_ERR_ARG, "sh_degree must be 0..3");
        if (gs->sh_dtype < 0 || gs->sh_dtype > 2) return fail(ctx, GAVIS_ERR_ARG, "bad sh_dtype");
        if (gs->n > 0 && !gs->sh) return fail(ctx, GAVIS_ERR_ARG, "sh is NULL");
    }
    if (gs->n > 0 && ((uintptr_t)gs->rots & 15u)) return fail(ctx, GAVIS_ERR_ARG, "rots must be 16-byte aligned");
    return GAVIS_OK;
}

int check_cams(gavis_ctx *ctx, const gavis_camera *cams, int n)
{
    if (n < 0) return fail(ctx, GAVIS_ERR_ARG, "negative camera count");
    if (n > 0 && !cams) return fail(ctx, GAVIS_ERR_ARG, "cameras is NULL");
    for (int i = 0; i < n; ++i) {
        const gavis_camera &c = cams[i];
        if (c.W <= 0 || c.H <= 0 || c.W > 16384 || c.H > 16384)
            return fail(ctx, GAVIS_ERR_ARG, "camera %d: W, H must be in 1..16384", i);
        if (c.W != cams[0].W || c.H != cams[0].H)
            return fail(ctx, GAVIS_ERR_ARG, "camera %d: every camera in a call must share W x H", i);
        if (!(c.fx > 0.0f && c.fy > 0.0f)) return fail(ctx, GAVIS_ERR_ARG, "camera %d: focal lengths must be > 0", i);
        if (!(c.znear > 0.0f)) return fail(ctx, GAVIS_ERR_ARG, "camera %d: znear must be > 0", i);
    }
    return GAVIS_OK;
}

RasterConsts raster_consts(const gavis_params *p)
{
    RasterConsts rc;
    rc.eps_T = p->eps_T;
    rc.q_cut = p->q_cut;
    rc.beta = p->beta;
    rc.o0 = p->o0;
    const double l2pie = std::log(2.0 * M_PI) + 1.0;
    rc.k_c = (float)(0.5 * 3.0 * std::log((double)p->sigma_c2) + 1.5 * l2pie);
    rc.k_0 = (float)(0.5 * (double)p->logdet_Q0 + 1.5 * l2pie);
    return rc;
}

// i_l(kappa) by closed forms and upward recurrence (kappa >= 1) or the power
// series (kappa < 1).
void bessel_i(int L, double x, double *out)
{
    // power series where the upward recurrence would lose digits (x < L)
    if (x < 1.0 || x < (double)L) {
        for (int l = 0; l <= L; ++l) {
            double df = 1.0;
            for (int k = 3; k <= 2 * l + 1; k += 2) df *= (double)k;
            double term = std::pow(x, l) / df, sum = term;
            for (int k = 1; k < 60; ++k) {
                term *= 0.5 * x * x / ((double)k * (double)(2 * l + 2 * k + 1));
                sum += term;
            }
            out[l] = sum;
        }
        return;
    }
    out[0] = std::sinh(x) / x;
    if (L >= 1) out[1] = (x * std::cosh(x) - std::sinh(x)) / (x * x);
    for (int l = 1; l < L; ++l) out[l + 1] = out[l - 1] - (2.0 * l + 1.0) / x * out[l];
}

struct Geometry {
    int W, H, TW, TH, TT;
};

Geometry geometry_of(const gavis_camera *cams, int tile)
{
    Geometry g;
    g.W = cams[0].W;
    g.H = cams[0].H;
    g.TW = (g.W + tile - 1) / tile;
    g.TH = (g.H + tile - 1) / tile;
    g.TT = g.TW * g.TH;
    return g;
}


// per-batch workspace: records, tile rectangles, flag-scan partials
struct RecLayout {
    GeoRec *geo;
    UaRec *ua;
    uint2 *rect;
    uint32_t *vis_words, *woff;   // [nv][ceil(n/32)] visibility bits and their record offsets
    float *zrec;                  // camera depth per visible record (what stage A's keys are made of)
    void *scan_tmp;
    size_t bytes;
};

RecLayout rec_layout(void *base, size_t nvn, bool ua, size_t nwords)
{
    RecLayout L;
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t b) { char *q = p ? p + off : nullptr; off += align256(b); return q; };
    L.geo = reinterpret_cast<GeoRec *>(take(nvn * sizeof(GeoRec)));
    L.ua = ua ? reinterpret_cast<UaRec *>(take(nvn * sizeof(UaRec))) : nullptr;
    L.rect = reinterpret_cast<uint2 *>(take(nvn * sizeof(uint2)));
    L.vis_words = reinterpret_cast<uint32_t *>(take(nwords * sizeof(uint32_t)));
    L.woff = reinterpret_cast<uint32_t *>(take(nwords * sizeof(uint32_t)));
    L.zrec = reinterpret_cast<float *>(take(nvn * sizeof(float)));
    L.scan_tmp = take(scan_tmp_bytes(nwords) + 64);
    L.bytes = off;
    return L;
}

// per-batch workspace of the two-level binning: stage A over the nrec visible
// records (32-bit keys in 8-byte slots, which hold the records' tile
// rectangles once the keys are sorted; record indices, their tile counts and
// offsets), stage B over the M tile entries (tile ids, Gaussian indices)
struct KeyLayout {
    uint64_t *a_k0, *a_k1;
    uint32_t *a_v0, *a_v1, *a_cnt, *a_off;
    uint32_t *b_k0, *b_k1, *b_v0, *b_v1;   // stage B by counting: b_v0 only
    RsBlock *blk_a, *blk_b;   // block tables of the segmented sorts
    BinLayout bin;            // stage B by counting
    void *tmp;
    size_t bytes;
};

// nseg: the most segments (view groups) either sort splits into; bin_tt > 0:
// stage B by counting over nv views of bin_tt tiles (no stage-B sort space)
KeyLayout key_layout(void *base, size_t nrec, size_t M, size_t nseg, int nv = 0, int bin_tt = 0)
{
    KeyLayout L;
    memset(&L, 0, sizeof(L));
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t b) { char *q = p ? p + off : nullptr; off += align256(b); return q; };
    const bool counting = bin_tt > 0;
    L.a_k0 = reinterpret_cast<uint64_t *>(take(nrec * 8));
    L.a_k1 = reinterpret_cast<uint64_t *>(take(nrec * 8));
    L.a_v0 = reinterpret_cast<uint32_t *>(take(nrec * 4));
    L.a_v1 = reinterpret_cast<uint32_t *>(take(nrec * 4));
    L.a_cnt = reinterpret_cast<uint32_t *>(take(nrec * 4));
    L.a_off = reinterpret_cast<uint32_t *>(take(nrec * 4));
    L.b_v0 = reinterpret_cast<uint32_t *>(take(M * 4));
    if (!counting) {
        L.b_k0 = reinterpret_cast<uint32_t *>(take(M * 4));
        L.b_k1 = reinterpret_cast<uint32_t *>(take(M * 4));
        L.b_v1 = reinterpret_cast<uint32_t *>(take(M * 4));
        L.blk_b = reinterpret_cast<RsBlock *>(take((M / kRadixTile + nseg + 1) * sizeof(RsBlock)));
    }
    L.blk_a = reinterpret_cast<RsBlock *>(take((nrec / kRadixTile + nseg + 1) * sizeof(RsBlock)));
    const size_t sorted = counting ? nrec : (nrec > M ? nrec : M);
    const size_t big = sorted + (nseg + 1) * (size_t)kRadixTile;   // a partial block per segment at most
    L.tmp = take(radix_tmp_bytes(big) + scan_tmp_bytes(big) + 64);
    if (counting) {
        const BinLayout b0 = bin_layout(nullptr, nrec, nv, bin_tt);
        L.bin = bin_layout(take(b0.bytes), nrec, nv, bin_tt);
    }
    L.bytes = off;
    return L;
}

struct SmallLayout {
    uint2 *ranges;
    float *tile_sums;        // one per 8 x 8 pixel block
    uint32_t *pair_counts;   // likewise
    unsigned long long *work;
    uint32_t *ok0, *ok1, *ov0, *ov1;   // tile order of the uncertainty pass (keys, values, double-buffered)
    void *otmp;
    BatchInfo *info;
    int32_t *best;
    uint32_t *voff;   // [nv + 1] visible records before each view, then [nv + 1] tile entries before each view
    uint32_t *eoff;
    size_t bytes;
};

SmallLayout small_layout(void *base, size_t nvt, size_t nv = 0, int tile = 8)
{
    SmallLayout L;
    char *p = reinterpret_cast<char *>(base);
    size_t off = 0;
    auto take = [&](size_t b) { char *q = p ? p + off : nullptr; off += align256(b); return q; };
    L.ranges = reinterpret_cast<uint2 *>(take(nvt * sizeof(uint2)));
    const size_t nblk = nvt * (size_t)blocks_per_tile(tile);
    L.tile_sums = reinterpret_cast<float *>(take(nblk * sizeof(float)));
    L.pair_counts = reinterpret_cast<uint32_t *>(take(nblk * sizeof(uint32_t)));
    L.work = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long)));
    L.ok0 = reinterpret_cast<uint32_t *>(take(nvt * sizeof(uint32_t)));
    L.ok1 = reinterpret_cast<uint32_t *>(take(nvt * sizeof(uint32_t)));
    L.ov0 = reinterpret_cast<uint32_t *>(take(nvt * sizeof(uint32_t)));
    L.ov1 = reinterpret_cast<uint32_t *>(take(nvt * sizeof(uint32_t)));
    L.otmp = take(radix_tmp_bytes(nvt) + 64);
    L.info = reinterpret_cast<BatchInfo *>(take(sizeof(BatchInfo)));
    L.best = reinterpret_cast<int32_t *>(take(sizeof(int32_t)));
    L.voff = reinterpret_cast<uint32_t *>(take((2 * nv + 2) * sizeof(uint32_t)));
    L.eoff = L.voff ? L.voff + nv + 1 : nullptr;
    L.bytes = off;
    return L;
}

enum Mode { MODE_SCORE, MODE_VIS, MODE_BINS };

struct ChainOut {
    // score mode
    float *rgb = nullptr, *unc = nullptr, *depth = nullptr, *score = nullptr;
    // vis mode: per-batch sums land in ctx->vis; callback consumes them
    // bins mode
    uint64_t *keys = nullptr;
    uint32_t *vals = nullptr;
    int64_t cap = 0;
    int64_t M = 0;
    uint32_t *ranges = nullptr;
};

size_t per_view_bytes(int64_t n, int TT, Mode m)
{
    size_t rec = (size_t)n * (sizeof(GeoRec) + (m == MODE_SCORE ? sizeof(UaRec) : 0) + 8 + 4 + 4 + 4);
    size_t vis = m == MODE_VIS ? (size_t)n * 12 : 0;
    size_t keys = (size_t)n * 2 * 24;   // typical: ~2 tiles per Gaussian per view
    return rec + vis + keys + (size_t)TT * 12;
}

int auto_batch(gavis_ctx *ctx, int64_t n, int TT, int n_views, Mode m, int requested)
{
    // record indices v * n + g of a batch are 32-bit
    const long long idx_cap = n > 0 ? (long long)(0xffffffffull / (unsigned long long)n) : n_views;
    long long nv;
    if (requested > 0) {
        nv = requested < n_views ? requested : n_views;
    } else {
        const size_t per = per_view_bytes(n, TT, m);
        // buffers are reused across batches, so the whole budget is available
        nv = (long long)((ctx->budget * 7 / 10) / (per ? per : 1));
        if (nv > 256) nv = 256;
        if (nv > n_views) nv = n_views;
    }
    if (nv > kMaxBatchViews) nv = kMaxBatchViews;
    if (nv > idx_cap) nv = idx_cap;
    if (nv < 1) nv = 1;
    return (int)nv;
}

// One batch of views [v0, v0+nv) through project -> ... -> composite.
// Returns GAVIS_ERR_BUDGET (without side effects on outputs) when the keys of
// this batch do not fit, so the caller can halve the batch.
int run_batch(gavis_ctx *ctx, Mode mode, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *d_cams,
              int nv, int v0, const gavis_params *p, const Geometry &G, ChainOut &out, cudaStream_t s,
              const gavis_camera *h_cams_all)
{
    const int64_t n = gs->n;
    const size_t nvn = (size_t)nv * (size_t)n;
    const size_t nvt = (size_t)nv * (size_t)G.TT;
    int rc;

    const size_t nwords = (size_t)nv * (size_t)((n + 31) / 32);
    RecLayout RL = rec_layout(nullptr, nvn, mode == MODE_SCORE, nwords);
    if ((rc = ensure(ctx, ctx->rec, RL.bytes, s)) != GAVIS_OK) return rc;
    RL = rec_layout(ctx->rec.p, nvn, mode == MODE_SCORE, nwords);
    SmallLayout SL = small_layout(nullptr, nvt, (size_t)nv, p->tile);
    if ((rc = ensure(ctx, ctx->small, SL.bytes, s)) != GAVIS_OK) return rc;
    SL = small_layout(ctx->small.p, nvt, (size_t)nv, p->tile);
    if (ctx->h_voff_cap < 2 * (size_t)nv + 2) {
        if (ctx->h_voff) cudaFreeHost(ctx->h_voff);
        ctx->h_voff = nullptr;
        ctx->h_voff_cap = 0;
        // sized once for the largest batch (a batch has at most kMaxBatchViews views)
        const size_t cap = 2 * (size_t)(nv > kMaxBatchViews ? nv : kMaxBatchViews) + 2;
        CK(cudaMallocHost(&ctx->h_voff, cap * sizeof(uint32_t)));
        ctx->h_voff_cap = cap;
    }
    uint32_t *h_eoff = ctx->h_voff + nv + 1;

    ProjectArgs pa{};
    pa.means = gs->means; pa.scales = gs->scales; pa.rots = gs->rots; pa.opac = gs->opac;
    pa.sh = gs->sh; pa.sh_degree = gs->sh_degree; pa.sh_dtype = gs->sh_dtype;
    pa.sh_var = mode == MODE_SCORE ? gs->sh_var : nullptr;
    pa.k_c = (float)(1.5 * std::log((double)p->sigma_c2) + 1.5 * (std::log(2.0 * M_PI) + 1.0));
    pa.gamma = (mode == MODE_SCORE && vf) ? vf->coeffs : nullptr;
    pa.vf_degree = (mode == MODE_SCORE && vf) ? vf->degree : 0;
    pa.vf_dtype = (mode == MODE_SCORE && vf) ? vf->dtype : 0;
    pa.n_train = (mode == MODE_SCORE && vf) ? vf->n_train_views : 0;
    pa.q_cut = p->q_cut; pa.beta = p->beta; pa.o0 = p->o0;
    pa.tile = p->tile; pa.TW = G.TW; pa.TH = G.TH;
    pa.cams = d_cams + v0; pa.nv = nv; pa.n = n;
    pa.geo = RL.geo; pa.ua = RL.ua; pa.rect = RL.rect; pa.counts = nullptr;   // the rectangles give the counts
    pa.vis_words = RL.vis_words;
    pa.zrec = RL.zrec;
    pa.zrange = SL.info->zrange;
    pa.visible = &SL.info->visible;
    pa.total = &SL.info->total;
    {
        Stage st(ctx, GAVIS_STAGE_PROJECT, s);
        CK(cudaMemsetAsync(SL.info, 0, sizeof(BatchInfo), s));
        CK(cudaMemsetAsync(&SL.info->zrange[0], 0xff, sizeof(uint32_t), s));   // zmin = all ones
        CK(launch_project(pa, s));
    }
    {
        // record offsets of the visibility words, in (view, index) order
        Stage st(ctx, GAVIS_STAGE_SCAN, s);
        CK(scan_vis_words(RL.vis_words, nwords, RL.woff, RL.scan_tmp, s));
    }
    CK(cudaMemcpyAsync(ctx->h_info, SL.info, sizeof(BatchInfo), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const unsigned long long M = ctx->h_info->total, nrec = ctx->h_info->visible;
    const uint32_t zmin = ctx->h_info->zrange[0];
    const int zb = nrec ? depth_bits(zmin, ctx->h_info->zrange[1]) : 0;
    if (M >= (1ull << 32) - 1) return fail(ctx, GAVIS_ERR_BUDGET, "more than 2^32 tile entries in one batch");
    if (ctx->prof_on) {
        ctx->prof_keys += M;
        ctx->prof_visible += nrec;
    }

    const int vb = bits_of((uint64_t)nv - 1);
    const int gb = vb + zb <= 32 ? vb : 32 - zb;
    const int gsz_a = 1 << gb, nseg_a = (nv + gsz_a - 1) / gsz_a;
    const int tbits = bits_of((uint64_t)G.TT - 1);
    int tb = -1, gbb = 0;
    if (tbits + vb > 16 && tbits <= 16 && ((nv - 1) >> (16 - tbits)) < 64) {
        tb = tbits;
        gbb = 16 - tbits;
    }
    const int nseg_b = tb < 0 ? 1 : (nv + (1 << gbb) - 1) >> gbb;
    const size_t nseg = (size_t)(nseg_a > nseg_b ? nseg_a : nseg_b);
    // stage B by counting where a view's tile counters fit shared memory and
    // (automatic choice) the batch is large enough to keep the GPU busy
    const bool counting = bin_by_counting(G.TT) && p->tile_lists != 2 &&
                          (p->tile_lists == 1 || nrec >= (unsigned long long)kBinMinRecords);
    if (ctx->prof_on && !counting) ctx->prof_sorted += M;
    const int bin_tt = counting ? G.TT : 0;
    KeyLayout KL = key_layout(nullptr, (size_t)nrec, (size_t)M, nseg, nv, bin_tt);
    if ((rc = ensure(ctx, ctx->keys, KL.bytes, s)) != GAVIS_OK) return rc;
    KL = key_layout(ctx->keys.p, (size_t)nrec, (size_t)M, nseg, nv, bin_tt);
    // block table of a segmented sort over the segments [seg[s], seg[s+1]),
    // staged through pinned memory (the previous table's copy has finished:
    // a stream synchronisation lies between any two uses)
    auto upload_blocks = [&](const std::vector<uint64_t> &seg, RsBlock *dst, size_t &nblk) -> int {
        nblk = radix_segment_blocks(seg.data(), (int)seg.size() - 1, nullptr);
        if (nblk > ctx->h_blk_cap) {
            if (ctx->h_blk) cudaFreeHost(ctx->h_blk);
            ctx->h_blk = nullptr;
            ctx->h_blk_cap = 0;
            // geometric growth: the rare regrowth (a pinned free waits for the
            // device) stays out of the steady state
            size_t cap = ctx->h_blk_cap ? 2 * ctx->h_blk_cap : ((size_t)1 << 16);
            while (cap < nblk) cap *= 2;
            CK(cudaMallocHost(&ctx->h_blk, cap * sizeof(RsBlock)));
            ctx->h_blk_cap = cap;
        }
        radix_segment_blocks(seg.data(), (int)seg.size() - 1, ctx->h_blk);
        if (nblk) CK(cudaMemcpyAsync(dst, ctx->h_blk, nblk * sizeof(RsBlock), cudaMemcpyHostToDevice, s));
        return GAVIS_OK;
    };
    bool alt_a = false, alt_b = false;
    // stage A: records sorted by (view, depth), ties in index order.  Keys
    // are 32 bits, ((view & (2^gb - 1)) << zb) | (depth bits - zmin) with
    // gb + zb <= 32 (depth bits of positive floats span zb <= 31 bits); the
    // groups of 2^gb views are sorted one after another, each over its
    // contiguous range of records (records are emitted in view order).  The
    // keys are written from the visibility bits the projection leaves.
    uint32_t *k0 = reinterpret_cast<uint32_t *>(KL.a_k0), *k1 = reinterpret_cast<uint32_t *>(KL.a_k1);
    {
        Stage st(ctx, GAVIS_STAGE_EMIT, s);
        CK(emit_vis_words(RL.vis_words, RL.woff, nv, n, RL.geo, RL.zrec, zb, zmin, (uint32_t)(gsz_a - 1), k0, KL.a_v0,
                          SL.voff, s));
    }
    if (gsz_a < nv) {   // group boundaries: a second read-back
        CK(cudaMemcpyAsync(ctx->h_voff, SL.voff, ((size_t)nv + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        ctx->h_voff[0] = 0u;
        ctx->h_voff[nv] = (uint32_t)nrec;
    }
    {
        Stage st(ctx, GAVIS_STAGE_SORT, s);
        std::vector<uint64_t> seg((size_t)nseg_a + 1);
        for (int g = 0; g <= nseg_a; ++g) seg[(size_t)g] = ctx->h_voff[g * gsz_a < nv ? g * gsz_a : nv];
        size_t nblk = 0;
        if ((rc = upload_blocks(seg, KL.blk_a, nblk)) != GAVIS_OK) return rc;
        CK(radix_sort_segments<uint32_t>(k0, KL.a_v0, k1, KL.a_v1, KL.blk_a, nblk, gb + zb, KL.tmp, &alt_a, s));
    }
    const uint32_t *recs = alt_a ? KL.a_v1 : KL.a_v0;
    const uint32_t *keys = nullptr, *vals = KL.b_v0;
    if (counting) {
        // stage B by counting: the lists and their ranges straight from the
        // records' rectangles in stage-A order
        Stage st(ctx, GAVIS_STAGE_EMIT, s);
        uint2 *rect_sorted = reinterpret_cast<uint2 *>(KL.a_k0);   // the stage-A keys are spent
        CK(launch_gather_rects(recs, RL.rect, (size_t)nrec, KL.a_cnt, rect_sorted, s));
        CK(launch_bin_tiles(recs, rect_sorted, SL.voff, nv, n, G.TW, G.TT, (size_t)nrec, nullptr, KL.bin, SL.ranges,
                            KL.b_v0, ~(size_t)0, nullptr, s));
    } else {
        // stage B: tile entries in stage-A order, i.e. view by view.  When the
        // tile index fits in tb <= 16 bits the keys are (view << tb) | tile and
        // each group of 2^(16 - tb) views is sorted on 16 bits (two passes) over
        // its contiguous entries; otherwise keys are view * TT + tile, one sort.
        {
            Stage st(ctx, GAVIS_STAGE_EMIT, s);
            // the stage-A keys are spent: their buffer holds the rectangles in stage-A order
            // the stage-B offsets per warp of 32 records (each warp scans its own records)
            uint2 *rect_sorted = reinterpret_cast<uint2 *>(KL.a_k0);
            uint32_t *warp_cnt = KL.a_cnt, *warp_off = KL.a_off;
            const size_t nwarps = ((size_t)nrec + 31) / 32;
            CK(launch_gather_rects(recs, RL.rect, (size_t)nrec, warp_cnt, rect_sorted, s));
            CK(exclusive_scan_u32(warp_cnt, warp_off, nwarps, KL.tmp, nullptr, s));
            CK(launch_emit_tiles(recs, nullptr, (size_t)nrec, RL.rect, n, G.TW, G.TH, KL.b_k0, KL.b_v0, s, nullptr,
                                 ~(size_t)0, nullptr, tb, rect_sorted, warp_off));
            if (tb >= 0) {   // tile entries before each view: a second read-back
                CK(launch_entry_offsets(warp_off, rect_sorted, SL.voff, nv, (uint32_t)M, SL.eoff, s));
                CK(cudaMemcpyAsync(h_eoff, SL.eoff, ((size_t)nv + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
            }
        }
        {
            Stage st(ctx, GAVIS_STAGE_SORT, s);
            if (tb < 0) {
                CK(radix_sort_pairs<uint32_t>(KL.b_k0, KL.b_v0, KL.b_k1, KL.b_v1, (size_t)M, bits_of((uint64_t)nvt - 1),
                                              KL.tmp, &alt_b, s));
            } else {
                const int gsz = 1 << gbb;
                std::vector<uint64_t> seg((size_t)nseg_b + 1);
                for (int g = 0; g <= nseg_b; ++g) {
                    seg[(size_t)g] = h_eoff[g * gsz < nv ? g * gsz : nv];
                    if (seg[(size_t)g] > M || (g > 0 && seg[(size_t)g] < seg[(size_t)g - 1]))
                        return fail(ctx, GAVIS_ERR_CUDA, "internal: inconsistent per-view entry offsets");
                }
                size_t nblk = 0;
                if ((rc = upload_blocks(seg, KL.blk_b, nblk)) != GAVIS_OK) return rc;
                CK(radix_sort_segments<uint32_t>(KL.b_k0, KL.b_v0, KL.b_k1, KL.b_v1, KL.blk_b, nblk, 16, KL.tmp, &alt_b,
                                                 s));
            }
        }
        keys = alt_b ? KL.b_k1 : KL.b_k0;
        vals = alt_b ? KL.b_v1 : KL.b_v0;
        {
            Stage st(ctx, GAVIS_STAGE_RANGES, s);
            CK(cudaMemsetAsync(SL.ranges, 0, nvt * sizeof(uint2), s));
            CK(launch_ranges(keys, (size_t)M, SL.ranges, s, nullptr, tb, (uint32_t)G.TT));
        }
    }
    // The uncertainty pass takes tiles longest list first, so that its
    // persistent warps do not end on a few long lists; at tile 32 the natural
    // order (neighbouring tiles, shared records in L2) measured faster.
    const uint32_t *order = nullptr;
    if (mode == MODE_SCORE && p->tile <= 16) {
        Stage st(ctx, GAVIS_STAGE_RANGES, s);
        CK(launch_order_keys(SL.ranges, nvt, SL.ok0, SL.ov0, s));
        bool alt_o = false;
        CK(radix_sort_pairs<uint32_t>(SL.ok0, SL.ov0, SL.ok1, SL.ov1, nvt, 8, SL.otmp, &alt_o, s));
        order = alt_o ? SL.ov1 : SL.ov0;
    }

    if (mode == MODE_BINS) {
        const int64_t off = out.M;
        if (off < out.cap && out.keys) {
            const int64_t m = (int64_t)M < out.cap - off ? (int64_t)M : out.cap - off;
            // canonical keys; one batch, so the view index is the call's
            if (counting)
                CK(launch_keys_from_ranges(SL.ranges, vals, nv, G.TT, RL.geo, n, (size_t)m, out.keys + off, s));
            else
                CK(launch_keys_export(keys, vals, (size_t)m, RL.geo, n, G.TT, out.keys + off, s, tb));
            CK(cudaMemcpyAsync(out.vals + off, vals, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
        }
        if (out.ranges)
            CK(cudaMemcpyAsync(out.ranges + 2 * (size_t)v0 * G.TT, SL.ranges, nvt * sizeof(uint2),
                               cudaMemcpyDeviceToDevice, s));
        out.M += (int64_t)M;
        return GAVIS_OK;
    }

    CompositeArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.ranges = SL.ranges; ca.vals = vals; ca.geo = RL.geo; ca.ua = RL.ua;
    ca.n = n; ca.nv = nv; ca.v0 = v0; ca.W = G.W; ca.H = G.H; ca.tile = p->tile; ca.TW = G.TW; ca.TH = G.TH;
    ca.rc = raster_consts(p);
    ca.tile_sums = SL.tile_sums;
    ca.work = SL.work;
    ca.order = order;
    if (mode == MODE_SCORE) {
        ca.rgb = out.rgb; ca.unc = out.unc; ca.depth = out.depth;
        ca.per_entry_kc = gs->sh_var != nullptr;
        ca.pair_counts = ctx->prof_pairs ? SL.pair_counts : nullptr;
        {
            Stage st(ctx, GAVIS_STAGE_COMPOSITE_UA, s);
            CK(launch_composite_ua(ca, s));
        }
        const int bpt = blocks_per_tile(p->tile);
        if (ca.pair_counts) CK(launch_sum_counts(SL.pair_counts, nvt * (size_t)bpt, ctx->d_pairs, s));
        Stage st(ctx, GAVIS_STAGE_REDUCE, s);
        CK(launch_view_reduce(SL.tile_sums, nv, G.TT * bpt, 1.0f / ((float)G.W * (float)G.H), out.score + v0, s));
    } else {
        if ((rc = ensure(ctx, ctx->vis, nvn * 12, s)) != GAVIS_OK) return rc;
        ca.sumT = reinterpret_cast<unsigned long long *>(ctx->vis.p);
        ca.cnt = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(ctx->vis.p) + nvn * 8);
        ca.pairs = ctx->prof_pairs ? ctx->d_pairs + 1 : nullptr;
        Stage st(ctx, GAVIS_STAGE_COMPOSITE_VIS, s);
        CK(cudaMemsetAsync(ctx->vis.p, 0, nvn * 12, s));
        CK(launch_composite_vis(ca, s));
    }
    (void)h_cams_all;
    return GAVIS_OK;
}

int upload_cams(gavis_ctx *ctx, const gavis_camera *cams, int n, cudaStream_t s)
{
    int rc = ensure(ctx, ctx->cams, sizeof(gavis_camera) * (size_t)(n > 0 ? n : 1), s);
    if (rc != GAVIS_OK) return rc;
    if (n > 0)
        CK(cudaMemcpyAsync(ctx->cams.p, cams, sizeof(gavis_camera) * (size_t)n, cudaMemcpyHostToDevice, s));
    return GAVIS_OK;
}

// Runs the chain over all views in batches, halving a batch whose keys do
// not fit.  `after` is called once per completed batch (VF accumulation).
template <class After>
int run_views(gavis_ctx *ctx, Mode mode, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cams,
              int n_views, const gavis_params *p, ChainOut &out, cudaStream_t s, After after)
{
    if (n_views == 0 || gs->n == 0) return GAVIS_OK;
    const Geometry G = geometry_of(cams, p->tile);
    int rc = upload_cams(ctx, cams, n_views, s);
    if (rc != GAVIS_OK) return rc;
    const gavis_camera *d_cams = reinterpret_cast<const gavis_camera *>(ctx->cams.p);
    int nv = auto_batch(ctx, gs->n, G.TT, n_views, mode, p->views_per_batch);
    int v0 = 0;
    while (v0 < n_views) {
        int cur = nv < n_views - v0 ? nv : n_views - v0;
        rc = run_batch(ctx, mode, gs, vf, d_cams, cur, v0, p, G, out, s, cams);
        if (rc == GAVIS_ERR_BUDGET && cur > 1 && mode != MODE_BINS) {
            nv = cur / 2;
            continue;
        }
        if (rc != GAVIS_OK) return rc;
        rc = after(v0, cur);
        if (rc != GAVIS_OK) return rc;
        v0 += cur;
    }
    return GAVIS_OK;
}

int check_vf(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf)
{
    if (!vf) return fail(ctx, GAVIS_ERR_ARG, "vf is NULL");
    if (vf->n != gs->n) return fail(ctx, GAVIS_ERR_ARG, "vf->n (%lld) != gaussians n (%lld)", (long long)vf->n,
                                    (long long)gs->n);
    if (vf->degree < 0 || vf->degree > kMaxVfDegree) return fail(ctx, GAVIS_ERR_ARG, "vf degree must be 0..5");
    if (vf->dtype < 0 || vf->dtype > 2) return fail(ctx, GAVIS_ERR_ARG, "bad vf dtype");
    if (vf->n_train_views < 0) return fail(ctx, GAVIS_ERR_ARG, "negative n_train_views");
    if (vf->n > 0 && !vf->coeffs) return fail(ctx, GAVIS_ERR_ARG, "vf coeffs is NULL");
    return GAVIS_OK;
}

}  // namespace

namespace gavis {
void set_error(gavis_ctx *c, const char *msg)
{
    if (c) c->err = msg;
}
}  // namespace gavis

extern "C" {

int gavis_ctx_create(gavis_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return GAVIS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GAVIS_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return GAVIS_ERR_CUDA;
    gavis_ctx *ctx = new gavis_ctx();
    ctx->device = device;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete ctx;
        return GAVIS_ERR_CUDA;
    }
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : fr / 10 * 6;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->mem, &props) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GAVIS_ERR_CUDA;
    }
    // keep released blocks in the pool (up to the budget) for the next growth
    uint64_t keep = (uint64_t)ctx->budget;
    cudaMemPoolSetAttribute(ctx->mem, cudaMemPoolAttrReleaseThreshold, &keep);
    if (cudaMallocHost(&ctx->h_info, sizeof(BatchInfo)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_best, sizeof(int32_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->tail, cudaEventDisableTiming) != cudaSuccess) {
        if (ctx->h_info) cudaFreeHost(ctx->h_info);
        if (ctx->h_best) cudaFreeHost(ctx->h_best);
        cudaMemPoolDestroy(ctx->mem);
        delete ctx;
        return GAVIS_ERR_CUDA;
    }
    *out = ctx;
    return GAVIS_OK;
}

void gavis_ctx_destroy(gavis_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (Buf *b : {&ctx->rec, &ctx->vis, &ctx->keys, &ctx->small, &ctx->gamma, &ctx->cams, &ctx->aug, &ctx->tune})
        if (b->p) cudaFree(b->p);
    if (ctx->mem) cudaMemPoolDestroy(ctx->mem);
    if (ctx->h_info) cudaFreeHost(ctx->h_info);
    if (ctx->h_voff) cudaFreeHost(ctx->h_voff);
    if (ctx->h_blk) cudaFreeHost(ctx->h_blk);
    if (ctx->h_best) cudaFreeHost(ctx->h_best);
    if (ctx->d_pairs) cudaFree(ctx->d_pairs);
    for (auto &r : ctx->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    if (ctx->tail) cudaEventDestroy(ctx->tail);
    delete ctx;
}

int gavis_prof_enable(gavis_ctx *ctx, int on)
{
    if (!ctx) return GAVIS_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!ctx->d_pairs) CK(cudaMalloc(&ctx->d_pairs, 2 * sizeof(unsigned long long)));
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(ctx->d_pairs, 0, 2 * sizeof(unsigned long long)));
    for (auto &r : ctx->pending) {
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < GAVIS_STAGE_COUNT; ++k) {
        ctx->prof_ms[k] = 0.0;
        ctx->prof_launches[k] = 0;
    }
    ctx->prof_keys = 0;
    ctx->prof_visible = 0;
    ctx->prof_sorted = 0;
    ctx->prof_on = on != 0;
    ctx->prof_pairs = on >= 2;
    return GAVIS_OK;
}

int gavis_prof_read(gavis_ctx *ctx, double *ms, int64_t *launches, int64_t *total_launches, uint64_t *pairs)
{
    if (!ctx) return GAVIS_ERR_ARG;
    cudaSetDevice(ctx->device);
    CK(cudaDeviceSynchronize());
    for (auto &r : ctx->pending) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        ctx->prof_ms[r.stage] += (double)t;
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < GAVIS_STAGE_COUNT; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_launches[k];
    }
    if (total_launches) *total_launches = g_launches.load();
    if (pairs) {
        unsigned long long h[2] = {0, 0};
        if (ctx->d_pairs) CK(cudaMemcpy(h, ctx->d_pairs, sizeof(h), cudaMemcpyDeviceToHost));
        pairs[0] = h[0];
        pairs[1] = h[1];
        pairs[2] = ctx->prof_keys;
        pairs[3] = ctx->prof_visible;
        pairs[4] = ctx->prof_sorted;
    }
    return GAVIS_OK;
}

const char *gavis_last_error(const gavis_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int gavis_params_default(gavis_params *p)
{
    if (!p) return GAVIS_ERR_ARG;
    p->kappa = 1.0f;
    p->vf_degree = 2;
    p->eps_T = 1e-4f;
    p->q_cut = 9.0f;
    p->beta = 0.5f;
    p->o0 = 0.15f;
    p->sigma_c2 = 0.01f;
    p->logdet_Q0 = 0.0f;
    p->tile = 16;
    p->views_per_batch = 0;
    p->tile_lists = 0;
    return GAVIS_OK;
}

int gavis_vmf_coeffs(int L, double kappa, double *a)
{
    if (!a || L < 0 || L > kMaxVfDegree || !(kappa >= 0.0)) return GAVIS_ERR_ARG;
    double i[kMaxVfDegree + 1] = {};
    if (kappa == 0.0) {
        i[0] = 1.0;
    } else {
        bessel_i(L, kappa, i);
    }
    const double zeta = std::exp(-kappa);
    for (int l = 0; l <= L; ++l) a[l] = 4.0 * M_PI * zeta * i[l];
    return GAVIS_OK;
}

int gavis_vf_build(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_camera *train, int n_train,
                   const gavis_params *p, gavis_vf *out, int accumulate, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, false)) || (rc = check_cams(ctx, train, n_train)))
        return rc;
    if (!out) return fail(ctx, GAVIS_ERR_ARG, "out is NULL");
    if (out->n != gs->n) return fail(ctx, GAVIS_ERR_ARG, "out->n != gaussians n");
    if (out->degree < 0 || out->degree > kMaxVfDegree) return fail(ctx, GAVIS_ERR_ARG, "out degree must be 0..5");
    if (out->dtype < 0 || out->dtype > 2) return fail(ctx, GAVIS_ERR_ARG, "bad out dtype");
    if (out->n > 0 && !out->coeffs) return fail(ctx, GAVIS_ERR_ARG, "out coeffs is NULL");
    if (accumulate && out->n_train_views < 0) return fail(ctx, GAVIS_ERR_ARG, "negative n_train_views");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    const int L = out->degree;
    const size_t K = (size_t)(L + 1) * (L + 1);
    const size_t count = (size_t)gs->n * K;
    if ((rc = ensure(ctx, ctx->gamma, count * sizeof(float), s)) != GAVIS_OK) return rc;
    float *g32 = reinterpret_cast<float *>(ctx->gamma.p);
    if (accumulate) CK(launch_vf_load(out->coeffs, out->dtype, count, g32, s));
    else CK(cudaMemsetAsync(g32, 0, count * sizeof(float), s));
    double ad[kMaxVfDegree + 1] = {};
    gavis_vmf_coeffs(L, (double)p->kappa, ad);
    ChainOut co;
    auto after = [&](int v0, int nv) -> int {
        AccumArgs aa;
        aa.means = gs->means;
        aa.cams = reinterpret_cast<const gavis_camera *>(ctx->cams.p) + v0;
        aa.nv = nv;
        aa.n = gs->n;
        const size_t nvn = (size_t)nv * (size_t)gs->n;
        aa.sumT = reinterpret_cast<const unsigned long long *>(ctx->vis.p);
        aa.cnt = reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(ctx->vis.p) + nvn * 8);
        for (int l = 0; l <= kMaxVfDegree; ++l) aa.a_l[l] = (float)ad[l];
        aa.L = L;
        aa.gamma32 = g32;
        Stage st(ctx, GAVIS_STAGE_VF_ACCUM, s);
        CK(launch_vf_accumulate(aa, s));
        return GAVIS_OK;
    };
    rc = run_views(ctx, MODE_VIS, gs, nullptr, train, n_train, p, co, s, after);
    if (rc != GAVIS_OK) return rc;
    CK(launch_vf_store(g32, count, out->coeffs, out->dtype, accumulate, s));
    out->n_train_views = accumulate ? out->n_train_views + n_train : n_train;
    out->kappa = p->kappa;
    return GAVIS_OK;
}

int gavis_score_views(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cand,
                      int n_cand, const gavis_params *p, float *rgb, float *unc, float *score, int32_t *best_dev,
                      int32_t *best_host, void *stream)
{
    gavis_views_out o;
    o.rgb = rgb;
    o.unc = unc;
    o.depth = nullptr;
    o.score = score;
    o.best_dev = best_dev;
    o.best_host = best_host;
    return gavis_render_views(ctx, gs, vf, cand, n_cand, p, &o, stream);
}

int gavis_render_views(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cand,
                       int n_cand, const gavis_params *p, const gavis_views_out *out, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    if (!out) return fail(ctx, GAVIS_ERR_ARG, "out is NULL");
    float *rgb = out->rgb, *unc = out->unc, *depth = out->depth, *score = out->score;
    int32_t *best_dev = out->best_dev, *best_host = out->best_host;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, true)) || (rc = check_vf(ctx, gs, vf)) ||
        (rc = check_cams(ctx, cand, n_cand)))
        return rc;
    if (n_cand > 0 && !score) return fail(ctx, GAVIS_ERR_ARG, "score is NULL");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    ChainOut co;
    co.rgb = rgb;
    co.unc = unc;
    co.depth = depth;
    co.score = score;
    if (gs->n == 0 && n_cand > 0) {
        // empty scene: every pixel has an empty list, H = 0, rgb = 0, depth = 0
        const size_t plane = (size_t)cand[0].W * cand[0].H;
        if (rgb) CK(cudaMemsetAsync(rgb, 0, (size_t)n_cand * 3 * plane * sizeof(float), s));
        if (unc) CK(cudaMemsetAsync(unc, 0, (size_t)n_cand * plane * sizeof(float), s));
        if (depth) CK(cudaMemsetAsync(depth, 0, (size_t)n_cand * plane * sizeof(float), s));
        CK(cudaMemsetAsync(score, 0, (size_t)n_cand * sizeof(float), s));
    } else {
        rc = run_views(ctx, MODE_SCORE, gs, vf, cand, n_cand, p, co, s, [](int, int) { return GAVIS_OK; });
        if (rc != GAVIS_OK) return rc;
    }
    if (best_dev || best_host) {
        SmallLayout SL = small_layout(nullptr, 1);
        if ((rc = ensure(ctx, ctx->small, SL.bytes, s)) != GAVIS_OK) return rc;
        SL = small_layout(ctx->small.p, 1);
        int32_t *dbest = best_dev ? best_dev : SL.best;
        Stage st(ctx, GAVIS_STAGE_REDUCE, s);
        if (n_cand > 0) CK(launch_argmax(score, n_cand, dbest, s));
        else CK(cudaMemsetAsync(dbest, 0xff, sizeof(int32_t), s));
        if (best_host) {
            CK(cudaMemcpyAsync(ctx->h_best, dbest, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            *best_host = *ctx->h_best;
        }
    }
    return GAVIS_OK;
}

int gavis_vf_query(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cams,
                   int n_cams, const gavis_params *p, float *V, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, false)) || (rc = check_vf(ctx, gs, vf)) ||
        (rc = check_cams(ctx, cams, n_cams)))
        return rc;
    if (n_cams > 0 && gs->n > 0 && !V) return fail(ctx, GAVIS_ERR_ARG, "V is NULL");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    if ((rc = upload_cams(ctx, cams, n_cams, s)) != GAVIS_OK) return rc;
    QueryArgs qa;
    qa.means = gs->means;
    qa.gamma = vf->coeffs;
    qa.vf_degree = vf->degree;
    qa.vf_dtype = vf->dtype;
    qa.n_train = vf->n_train_views;
    qa.n = gs->n;
    for (int v0 = 0; v0 < n_cams; v0 += kMaxBatchViews) {   // cameras of a launch sit in shared memory
        qa.cams = reinterpret_cast<const gavis_camera *>(ctx->cams.p) + v0;
        qa.nv = n_cams - v0 < kMaxBatchViews ? n_cams - v0 : kMaxBatchViews;
        qa.V = V + (size_t)v0 * (size_t)gs->n;
        CK(launch_query(qa, s));
    }
    return GAVIS_OK;
}

int gavis_debug_bins(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_camera *cams, int n_cams,
                     const gavis_params *p, uint64_t *keys, uint32_t *vals, int64_t cap, int64_t *M_out,
                     uint32_t *ranges, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, false)) || (rc = check_cams(ctx, cams, n_cams)))
        return rc;
    if (!M_out) return fail(ctx, GAVIS_ERR_ARG, "M_out is NULL");
    if (n_cams > kMaxBatchViews) return fail(ctx, GAVIS_ERR_ARG, "gavis_debug_bins takes at most %d cameras", kMaxBatchViews);
    if (cap > 0 && (!keys || !vals)) return fail(ctx, GAVIS_ERR_ARG, "keys/vals NULL with cap > 0");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    gavis_params q = *p;
    q.views_per_batch = n_cams;   // one batch: keys carry the view index within the call
    ChainOut co;
    co.keys = keys;
    co.vals = vals;
    co.cap = cap;
    co.ranges = ranges;
    if (ranges && n_cams > 0 && gs->n == 0) {
        const Geometry G = geometry_of(cams, p->tile);
        CK(cudaMemsetAsync(ranges, 0, (size_t)n_cams * G.TT * 8, s));
    }
    rc = run_views(ctx, MODE_BINS, gs, nullptr, cams, n_cams, &q, co, s, [](int, int) { return GAVIS_OK; });
    if (rc != GAVIS_OK) return rc;
    CK(cudaStreamSynchronize(s));
    *M_out = co.M;
    return GAVIS_OK;
}

int gavis_vf_density_control(gavis_ctx *ctx, const gavis_gaussians *gs, const float *virt_means, int64_t n_virt,
                             const gavis_camera *train, int n_train, const gavis_params *p, float rho, float eta,
                             float eps_v, float *vis_out, uint8_t *keep, float *kept_means, int64_t *n_keep,
                             float *scale_out, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, false)) || (rc = check_cams(ctx, train, n_train)))
        return rc;
    if (n_virt < 0 || gs->n + n_virt >= ((int64_t)1 << 31)) return fail(ctx, GAVIS_ERR_ARG, "n_virt out of range");
    if (n_virt > 0 && (!virt_means || !keep)) return fail(ctx, GAVIS_ERR_ARG, "virt_means/keep is NULL");
    if (!(rho > 0.0f) || !(eta > -1.0f)) return fail(ctx, GAVIS_ERR_ARG, "rho must be > 0 and eta > -1");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    const double sd = std::cbrt(3.0 * (1.0 + (double)eta) / (4.0 * M_PI * (double)rho));
    if (scale_out) *scale_out = (float)sd;
    if (n_virt == 0) {
        if (n_keep) *n_keep = 0;
        return GAVIS_OK;
    }
    // the union of the scene and the virtual particles, plus the per-particle
    // product, keep flags and their scan
    const int64_t na = gs->n + n_virt;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align256(b); return o; };
    const size_t o_m = take((size_t)na * 12), o_s = take((size_t)na * 12), o_r = take((size_t)na * 16),
                 o_o = take((size_t)na * 4), o_p = take((size_t)n_virt * 4), o_k = take((size_t)n_virt * 4),
                 o_q = take((size_t)n_virt * 4), o_t = take(scan_tmp_bytes((size_t)n_virt) + 64),
                 o_n = take(sizeof(unsigned long long));
    if ((rc = ensure(ctx, ctx->aug, off, s)) != GAVIS_OK) return rc;
    char *base = reinterpret_cast<char *>(ctx->aug.p);
    float *am = reinterpret_cast<float *>(base + o_m), *as = reinterpret_cast<float *>(base + o_s);
    float *ar = reinterpret_cast<float *>(base + o_r), *ao = reinterpret_cast<float *>(base + o_o);
    float *prod = reinterpret_cast<float *>(base + o_p);
    uint32_t *keep32 = reinterpret_cast<uint32_t *>(base + o_k), *pos = reinterpret_cast<uint32_t *>(base + o_q);
    void *stmp = base + o_t;
    unsigned long long *d_nk = reinterpret_cast<unsigned long long *>(base + o_n);
    const size_t n = (size_t)gs->n;
    if (n) {
        CK(cudaMemcpyAsync(am, gs->means, n * 12, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(as, gs->scales, n * 12, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ar, gs->rots, n * 16, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ao, gs->opac, n * 4, cudaMemcpyDeviceToDevice, s));
    }
    CK(launch_virtual_fill(virt_means, n_virt, (float)sd, am + 3 * n, as + 3 * n, ar + 4 * n, ao + n, s));
    CK(launch_fill_f32(prod, (size_t)n_virt, 1.0f, s));
    gavis_gaussians all = *gs;
    all.n = na;
    all.means = am; all.scales = as; all.rots = ar; all.opac = ao;
    ChainOut co;
    auto after = [&](int, int nv) -> int {
        const size_t nvn = (size_t)nv * (size_t)na;
        const unsigned long long *sT = reinterpret_cast<const unsigned long long *>(ctx->vis.p);
        const uint32_t *c = reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(ctx->vis.p) + nvn * 8);
        CK(launch_vf_product(sT, c, nv, na, gs->n, n_virt, prod, s));
        return GAVIS_OK;
    };
    rc = run_views(ctx, MODE_VIS, &all, nullptr, train, n_train, p, co, s, after);
    if (rc != GAVIS_OK) return rc;
    CK(launch_density_finalize(prod, n_virt, eps_v, vis_out, keep, keep32, s));
    CK(exclusive_scan_u32(keep32, pos, (size_t)n_virt, stmp, d_nk, s));
    if (kept_means) CK(launch_compact_kept(virt_means, keep32, pos, n_virt, kept_means, s));
    if (n_keep) {
        CK(cudaMemcpyAsync(ctx->h_info, d_nk, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *n_keep = (int64_t)ctx->h_info->total;
    }
    return GAVIS_OK;
}

int gavis_augment(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const float *kept_means,
                  int64_t n_kept, float scale, float *means, float *scales, float *rots, float *opac, void *sh,
                  void *sh_var, void *coeffs, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_gaussians(ctx, gs, true)) || (rc = check_vf(ctx, gs, vf))) return rc;
    if (n_kept < 0 || gs->n + n_kept >= ((int64_t)1 << 31)) return fail(ctx, GAVIS_ERR_ARG, "n_kept out of range");
    if (n_kept > 0 && !kept_means) return fail(ctx, GAVIS_ERR_ARG, "kept_means is NULL");
    if (!(scale > 0.0f)) return fail(ctx, GAVIS_ERR_ARG, "scale must be > 0");
    if (!means || !scales || !rots || !opac || !sh || !coeffs)
        return fail(ctx, GAVIS_ERR_ARG, "NULL output array");
    if ((gs->sh_var != nullptr) != (sh_var != nullptr))
        return fail(ctx, GAVIS_ERR_ARG, "sh_var output must be given exactly when the scene has colour variances");
    if ((uintptr_t)rots & 15u) return fail(ctx, GAVIS_ERR_ARG, "rots must be 16-byte aligned");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    const size_t n = (size_t)gs->n, k = (size_t)n_kept;
    const size_t esh = gs->sh_dtype == GAVIS_F32 ? 4 : 2, evf = vf->dtype == GAVIS_F32 ? 4 : 2;
    const size_t Kc = (size_t)(gs->sh_degree + 1) * (gs->sh_degree + 1) * 3;
    const size_t Kv = (size_t)(vf->degree + 1) * (vf->degree + 1);
    // the trained Gaussians, unchanged, then the kept virtual particles
    if (n) {
        CK(cudaMemcpyAsync(means, gs->means, n * 12, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(scales, gs->scales, n * 12, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(rots, gs->rots, n * 16, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(opac, gs->opac, n * 4, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(sh, gs->sh, n * Kc * esh, cudaMemcpyDeviceToDevice, s));
        if (sh_var) CK(cudaMemcpyAsync(sh_var, gs->sh_var, n * Kc * esh, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(coeffs, vf->coeffs, n * Kv * evf, cudaMemcpyDeviceToDevice, s));
    }
    if (k) {
        // identity rotation, isotropic scale, zero opacity; zero colour and
        // zero field (V = 0: only the prior component of eq:alpha_comp)
        CK(launch_virtual_fill(kept_means, n_kept, scale, means + 3 * n, scales + 3 * n, rots + 4 * n, opac + n, s));
        CK(cudaMemsetAsync(static_cast<char *>(sh) + n * Kc * esh, 0, k * Kc * esh, s));
        CK(cudaMemsetAsync(static_cast<char *>(coeffs) + n * Kv * evf, 0, k * Kv * evf, s));
        if (sh_var) {   // any positive variance will do: a Gaussian with V = 0 has no visible component
            char *dst = static_cast<char *>(sh_var) + n * Kc * esh;
            if (gs->sh_dtype == GAVIS_F32)
                CK(launch_fill_f32(reinterpret_cast<float *>(dst), k * Kc, 1.0f, s));
            else
                CK(launch_fill_u16(reinterpret_cast<uint16_t *>(dst), k * Kc,
                                   gs->sh_dtype == GAVIS_F16 ? (uint16_t)0x3c00u : (uint16_t)0x3f80u, s));
        }
    }
    return GAVIS_OK;
}

// ---------------------------------------------------------------- autotuner
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;   // workload key -> tile edge

std::string tune_key(int mode, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *c, int n)
{
    char buf[160];
    // the Gaussian count is bucketed by powers of two
    snprintf(buf, sizeof(buf), "m%d_w%d_h%d_n%d_sh%d_vf%d_v%d", mode, c->W, c->H, bits_of((uint64_t)gs->n),
             gs->sh_degree, vf ? vf->degree : -1, bits_of((uint64_t)n));
    return buf;
}

void tune_cache_load(const char *path)
{
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[160];
    int tile;
    while (fscanf(f, "%159s %d", key, &tile) == 2) g_tune_cache[key] = tile;
    fclose(f);
}

void tune_cache_store(const char *path, const std::string &key, int tile)
{
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), tile);
    fclose(f);
}

}  // namespace

int gavis_autotune(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cams, int n_cams,
                   int mode, gavis_params *p, double *best_ms, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, mode == 0)) || (rc = check_cams(ctx, cams, n_cams)))
        return rc;
    if (mode != 0 && mode != 1) return fail(ctx, GAVIS_ERR_ARG, "mode must be 0 (scoring) or 1 (field construction)");
    if (mode == 0 && (rc = check_vf(ctx, gs, vf))) return rc;
    if (n_cams < 1 || gs->n == 0) return GAVIS_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    const std::string key = tune_key(mode, gs, vf, cams, n_cams);
    const char *path = std::getenv("GAVIS_AUTOTUNE_CACHE");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        static bool loaded = false;
        if (path && !loaded) {
            tune_cache_load(path);
            loaded = true;
        }
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->tile = it->second;
            if (best_ms) *best_ms = -1.0;
            return GAVIS_OK;
        }
    }
    // scratch outputs of the trial runs: scoring trials write the uncertainty
    // and the colour (the full output of the UQ rasterizer, whose colour path
    // is part of the composite's cost)
    const size_t plane = (size_t)cams[0].W * cams[0].H;
    const int L = mode == 0 ? vf->degree : p->vf_degree;
    const size_t K = (size_t)(L + 1) * (L + 1);
    const size_t bytes = mode == 0 ? align256((size_t)n_cams * 4) + align256((size_t)n_cams * plane * 4) +
                                         (size_t)n_cams * plane * 12
                                   : (size_t)gs->n * K * 4;
    if ((rc = ensure(ctx, ctx->tune, bytes, s)) != GAVIS_OK) return rc;
    float *score = reinterpret_cast<float *>(ctx->tune.p);
    float *unc = reinterpret_cast<float *>(reinterpret_cast<char *>(ctx->tune.p) + align256((size_t)n_cams * 4));
    float *rgb = reinterpret_cast<float *>(reinterpret_cast<char *>(unc) + align256((size_t)n_cams * plane * 4));
    gavis_vf tv;
    tv.n = gs->n; tv.coeffs = ctx->tune.p; tv.degree = L; tv.dtype = GAVIS_F32; tv.n_train_views = 0; tv.kappa = 0;
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    const int tiles[3] = {8, 16, 32};
    double best = 1e300;
    int best_tile = p->tile;
    for (int t : tiles) {
        gavis_params q = *p;
        q.tile = t;
        double ms_sum = 0.0;
        for (int rep = 0; rep < 3; ++rep) {   // the first run warms up the workspace
            CK(cudaEventRecord(e0, s));
            rc = mode == 0 ? gavis_score_views(ctx, gs, vf, cams, n_cams, &q, rgb, unc, score, nullptr, nullptr, stream)
                           : gavis_vf_build(ctx, gs, cams, n_cams, &q, &tv, 0, stream);
            if (rc != GAVIS_OK) return rc;
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) ms_sum += ms;
        }
        const double ms = ms_sum / 2.0;
        if (ms < best) {
            best = ms;
            best_tile = t;
        }
    }
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    p->tile = best_tile;
    if (best_ms) *best_ms = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_tile;
    if (path) tune_cache_store(path, key, best_tile);
    return GAVIS_OK;
}

int gavis_debug_visibility(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_camera *cams, int n_cams,
                           const gavis_params *p, float *sumT, uint32_t *cnt, void *stream)
{
    if (!ctx) return GAVIS_ERR_ARG;
    int rc;
    if ((rc = check_params(ctx, p)) || (rc = check_gaussians(ctx, gs, false)) || (rc = check_cams(ctx, cams, n_cams)))
        return rc;
    if (n_cams > 0 && gs->n > 0 && (!sumT || !cnt)) return fail(ctx, GAVIS_ERR_ARG, "sumT/cnt is NULL");
    cudaSetDevice(ctx->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CallOrder order(ctx, s);
    ChainOut co;
    auto after = [&](int v0, int nv) -> int {
        const size_t nvn = (size_t)nv * (size_t)gs->n;
        const unsigned long long *sT = reinterpret_cast<const unsigned long long *>(ctx->vis.p);
        const uint32_t *c = reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(ctx->vis.p) + nvn * 8);
        CK(launch_vis_export(sT, c, nvn, sumT + (size_t)v0 * gs->n, cnt + (size_t)v0 * gs->n, s));
        return GAVIS_OK;
    };
    return run_views(ctx, MODE_VIS, gs, nullptr, cams, n_cams, p, co, s, after);
}

}  // extern "C"
