// plan.cu -- candidate-view scoring captured once as a CUDA graph and
// replayed (no counterpart in the paper: it removes the per-call host work of
// the paper's per-planning-step scoring).
//
// A plan fixes the scene, the field, the number of candidate views, their
// resolution, the parameters and the output buffers.  The views go through
// the chain in batches of p->views_per_batch (0: all at once), captured one
// after another over the same buffers, which are sized statically for one
// batch: projected records for every (view, Gaussian), sort space for
// `record_capacity` visible records and `entry_capacity` tile entries.  The
// kernels after the projection read the actual numbers of visible records
// and tile entries from device memory (grids are sized by the capacities),
// so nothing in the chain waits for the host; if a replay needs more than a
// capacity, the excess is dropped, a device flag is set, and
// gavis_plan_overflowed reports it (the caller then rebuilds the plan with
// larger capacities).
// The sorts are sized on the device as the batched call sizes them on the
// host: after the projection a kernel derives the depth bits and the view
// groups of the stage-A keys from the batch's depth range, the record and
// tile-entry offsets of every view give the segments of the two segmented
// sorts, and kernels build their block tables (as many blocks as the
// capacities can need; the unused ones are empty).  So a replay runs the
// same passes over the same keys as gavis_score_views, and its outputs are
// the same bits.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "gavis_internal.cuh"

using namespace gavis;

namespace {

struct PlanInfo {              // device
    BatchInfo b;
    uint32_t entries_over;     // a launch needed more tile entries than the capacity
    uint32_t records_over;     // ... more visible records than the capacity
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct gavis_plan {
    int device = 0;
    int n_cams = 0, n_batches = 1, W = 0, H = 0;
    size_t record_cap = 0, entry_cap = 0;
    void *buf = nullptr;                // one device allocation for everything
    gavis_camera *h_cams = nullptr;     // pinned staging of the poses
    gavis_camera *d_cams = nullptr;
    PlanInfo *d_info = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    long long kernels = 0;              // kernels per replay
    bool launched = false;
};

namespace {

void plan_free(gavis_plan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->done) cudaEventDestroy(pl->done);
    if (pl->h_cams) cudaFreeHost(pl->h_cams);
    if (pl->buf) cudaFree(pl->buf);
    delete pl;
}

#define PK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            char m_[320];                                                                              \
            snprintf(m_, sizeof(m_), "%s: %s", #call, cudaGetErrorString(e_));                         \
            set_error(ctx, m_);                                                                        \
            if (capturing) {                                                                           \
                cudaGraph_t g_ = nullptr;                                                              \
                cudaStreamEndCapture(cs, &g_);                                                         \
                if (g_) cudaGraphDestroy(g_);                                                          \
            }                                                                                          \
            if (cs) cudaStreamDestroy(cs);                                                             \
            plan_free(pl);                                                                             \
            cudaGetLastError();                                                                        \
            return GAVIS_ERR_CUDA;                                                                     \
        }                                                                                              \
    } while (0)

}  // namespace

extern "C" {

int gavis_plan_create(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, int n_cams, int W, int H,
                      const gavis_params *p, int64_t record_capacity, int64_t entry_capacity, float *rgb,
                      float *unc, float *score, int32_t *best_dev, gavis_plan **out)
{
    if (!out) return GAVIS_ERR_ARG;
    *out = nullptr;
    if (!gs || !vf || !p || !score || n_cams < 1 || n_cams > 16384 || W < 1 || H < 1 || W > 16384 || H > 16384 ||
        entry_capacity < 1 || record_capacity < 0 || gs->n < 1 || gs->n >= ((int64_t)1 << 31) || !gs->sh ||
        vf->n != gs->n || !(p->tile == 8 || p->tile == 16 || p->tile == 32) || p->views_per_batch < 0 ||
        p->tile_lists < 0 || p->tile_lists > 2 ||
        ((uintptr_t)gs->rots & 15u)) {
        set_error(ctx, "gavis_plan_create: invalid argument (sizes, tile must be 8/16/32, rots 16-byte aligned)");
        return GAVIS_ERR_ARG;
    }
    const int64_t n = gs->n;
    const int TW = (W + p->tile - 1) / p->tile, TH = (H + p->tile - 1) / p->tile, TT = TW * TH;
    // views per batch: every batch reuses the same buffers, one after another
    int B = p->views_per_batch > 0 && p->views_per_batch < n_cams ? p->views_per_batch : n_cams;
    if (B > kMaxBatchViews) B = kMaxBatchViews;   // one projection launch per batch
    const int nb = (n_cams + B - 1) / B;
    const size_t nvn = (size_t)B * (size_t)n, nvt = (size_t)B * (size_t)TT;
    const size_t M = (size_t)entry_capacity;
    const size_t R = record_capacity == 0 || (size_t)record_capacity > nvn ? nvn : (size_t)record_capacity;
    if (nvn >= ((size_t)1 << 32) || M >= ((size_t)1 << 32)) {
        set_error(ctx, "gavis_plan_create: views per batch x n and entry_capacity must each be below 2^32");
        return GAVIS_ERR_ARG;
    }

    gavis_plan *pl = new gavis_plan();
    cudaStream_t cs = nullptr;
    bool capturing = false;
    PK(cudaGetDevice(&pl->device));
    pl->n_cams = n_cams;
    pl->n_batches = nb;
    pl->W = W;
    pl->H = H;
    pl->record_cap = R;
    pl->entry_cap = M;

    // static layout
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += up256(b ? b : 1); return o; };
    const size_t o_cams = take((size_t)n_cams * sizeof(gavis_camera)), o_info = take(nb * sizeof(PlanInfo));
    const size_t o_geo = take(nvn * sizeof(GeoRec)), o_ua = take(nvn * sizeof(UaRec)), o_rect = take(nvn * 8);
    const size_t nwords = (size_t)B * (size_t)((n + 31) / 32);
    const size_t o_words = take(nwords * 4), o_woff = take(nwords * 4);
    const size_t o_zrec = take(nvn * 4);   // dense depth copy of the visible records (stage-A keys)
    const size_t o_scan = take(scan_tmp_bytes(nwords) + 64);
    const size_t o_ak0 = take(R * 4), o_ak1 = take(R * 4), o_av0 = take(R * 4), o_av1 = take(R * 4);
    const size_t o_acnt = take(R * 4), o_aoff = take(R * 4), o_rs = take(R * 8);
    // stage B by counting (views of up to kBinMaxTiles tiles): one value
    // array and the count tables; else keys and values of a sort
    const bool counting = bin_by_counting(TT) && p->tile_lists != 2 &&
                          (p->tile_lists == 1 || R >= (size_t)kBinMinRecords);
    const size_t o_bv0 = take(M * 4);
    const size_t o_bk0 = counting ? 0 : take(M * 4), o_bk1 = counting ? 0 : take(M * 4);
    const size_t o_bv1 = counting ? 0 : take(M * 4);
    const size_t o_bin = counting ? take(bin_layout(nullptr, R, B, TT).bytes) : 0;
    // segmented sorts: block tables for the largest batch, key parameters,
    // per-view record and entry offsets
    const size_t nblk_a = radix_segment_blocks_max(R, B), nblk_b = counting ? 0 : radix_segment_blocks_max(M, B);
    const size_t o_blka = take(nblk_a * sizeof(RsBlock)), o_blkb = take(nblk_b * sizeof(RsBlock));
    const size_t o_kp = take(sizeof(KeyParams));
    const size_t o_voff = take(((size_t)B + 1) * 4), o_eoff = take(((size_t)B + 1) * 4);
    size_t big = counting || R > M ? R : M;   // the largest sort
    if (nvt > big) big = nvt;   // the tile-order sort shares the temporary space
    const size_t seg_items = (nblk_a > nblk_b ? nblk_a : nblk_b) * (size_t)kRadixTile;
    const size_t o_tmp = take(radix_tmp_bytes(big > seg_items ? big : seg_items) + scan_tmp_bytes(big) + 64);
    const int bpt = blocks_per_tile(p->tile);
    const size_t o_rng = take(nvt * sizeof(uint2)), o_ts = take(nvt * (size_t)bpt * sizeof(float));
    const size_t o_work = take(sizeof(unsigned long long));
    // tile order of the uncertainty pass (keys, values, double-buffered) and
    // the device copy of the largest batch's tile count (sort size bound)
    const bool ordered = p->tile <= 16;
    const size_t o_ok0 = take(nvt * 4), o_ok1 = take(nvt * 4), o_ov0 = take(nvt * 4), o_ov1 = take(nvt * 4);
    const size_t o_nt = take(sizeof(unsigned long long));
    PK(cudaMalloc(&pl->buf, off));
    PK(cudaMallocHost(&pl->h_cams, (size_t)n_cams * sizeof(gavis_camera)));
    std::memset(pl->h_cams, 0, (size_t)n_cams * sizeof(gavis_camera));
    for (int k = 0; k < n_cams; ++k) {   // placeholder poses until the first launch
        pl->h_cams[k].W = W;
        pl->h_cams[k].H = H;
    }
    PK(cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming));
    char *b = reinterpret_cast<char *>(pl->buf);
    pl->d_cams = reinterpret_cast<gavis_camera *>(b + o_cams);
    pl->d_info = reinterpret_cast<PlanInfo *>(b + o_info);
    GeoRec *geo = reinterpret_cast<GeoRec *>(b + o_geo);
    UaRec *ua = reinterpret_cast<UaRec *>(b + o_ua);
    uint2 *rect = reinterpret_cast<uint2 *>(b + o_rect);
    uint32_t *vis_words = reinterpret_cast<uint32_t *>(b + o_words), *woff = reinterpret_cast<uint32_t *>(b + o_woff);
    float *zrec = reinterpret_cast<float *>(b + o_zrec);
    uint32_t *ak0 = reinterpret_cast<uint32_t *>(b + o_ak0), *ak1 = reinterpret_cast<uint32_t *>(b + o_ak1);
    RsBlock *blk_a = reinterpret_cast<RsBlock *>(b + o_blka), *blk_b = reinterpret_cast<RsBlock *>(b + o_blkb);
    KeyParams *kp = reinterpret_cast<KeyParams *>(b + o_kp);
    uint32_t *voff = reinterpret_cast<uint32_t *>(b + o_voff), *eoff = reinterpret_cast<uint32_t *>(b + o_eoff);
    uint32_t *av0 = reinterpret_cast<uint32_t *>(b + o_av0), *av1 = reinterpret_cast<uint32_t *>(b + o_av1);
    uint32_t *acnt = reinterpret_cast<uint32_t *>(b + o_acnt), *aoff = reinterpret_cast<uint32_t *>(b + o_aoff);
    uint2 *rect_sorted = reinterpret_cast<uint2 *>(b + o_rs);
    uint32_t *bk0 = counting ? nullptr : reinterpret_cast<uint32_t *>(b + o_bk0);
    uint32_t *bk1 = counting ? nullptr : reinterpret_cast<uint32_t *>(b + o_bk1);
    uint32_t *bv0 = reinterpret_cast<uint32_t *>(b + o_bv0);
    uint32_t *bv1 = counting ? nullptr : reinterpret_cast<uint32_t *>(b + o_bv1);
    const BinLayout bins = counting ? bin_layout(b + o_bin, R, B, TT) : BinLayout{};
    void *tmp = b + o_tmp, *scan_tmp = b + o_scan;
    uint2 *ranges = reinterpret_cast<uint2 *>(b + o_rng);
    float *tile_sums = reinterpret_cast<float *>(b + o_ts);
    unsigned long long *work = reinterpret_cast<unsigned long long *>(b + o_work);
    uint32_t *ok0 = reinterpret_cast<uint32_t *>(b + o_ok0), *ok1 = reinterpret_cast<uint32_t *>(b + o_ok1);
    uint32_t *ov0 = reinterpret_cast<uint32_t *>(b + o_ov0), *ov1 = reinterpret_cast<uint32_t *>(b + o_ov1);
    unsigned long long *d_nt = reinterpret_cast<unsigned long long *>(b + o_nt);
    {
        const unsigned long long nt64 = (unsigned long long)nvt;
        PK(cudaMemcpy(d_nt, &nt64, sizeof(nt64), cudaMemcpyHostToDevice));
    }

    ProjectArgs pa{};
    pa.means = gs->means; pa.scales = gs->scales; pa.rots = gs->rots; pa.opac = gs->opac;
    pa.sh = gs->sh; pa.sh_degree = gs->sh_degree; pa.sh_dtype = gs->sh_dtype;
    pa.sh_var = gs->sh_var;
    pa.k_c = (float)(1.5 * std::log((double)p->sigma_c2) + 1.5 * (std::log(2.0 * M_PI) + 1.0));
    pa.gamma = vf->coeffs; pa.vf_degree = vf->degree; pa.vf_dtype = vf->dtype; pa.n_train = vf->n_train_views;
    pa.q_cut = p->q_cut; pa.beta = p->beta; pa.o0 = p->o0;
    pa.tile = p->tile; pa.TW = TW; pa.TH = TH;
    pa.n = n;
    pa.geo = geo; pa.ua = ua; pa.rect = rect; pa.counts = nullptr;   // the rectangles give the counts
    pa.vis_words = vis_words;
    pa.zrec = zrec;
    CompositeArgs ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.ranges = ranges; ca.geo = geo; ca.ua = ua;
    ca.n = n; ca.W = W; ca.H = H; ca.tile = p->tile; ca.TW = TW; ca.TH = TH;
    ca.rc.eps_T = p->eps_T; ca.rc.q_cut = p->q_cut; ca.rc.beta = p->beta; ca.rc.o0 = p->o0;
    const double l2pie = std::log(2.0 * M_PI) + 1.0;
    ca.rc.k_c = pa.k_c;
    ca.rc.k_0 = (float)(0.5 * (double)p->logdet_Q0 + 1.5 * l2pie);
    ca.rgb = rgb; ca.unc = unc; ca.tile_sums = tile_sums; ca.work = work;
    ca.per_entry_kc = gs->sh_var != nullptr;

    // the chain of every batch, captured on a private stream
    radix_prepare();
    bin_prepare();
    composite_prepare(p->tile);
    PK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const long long k0 = g_launches.load();
    PK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    capturing = true;
    PK(cudaMemcpyAsync(pl->d_cams, pl->h_cams, (size_t)n_cams * sizeof(gavis_camera), cudaMemcpyHostToDevice, cs));
    PK(cudaMemsetAsync(pl->d_info, 0, nb * sizeof(PlanInfo), cs));
    for (int bi = 0; bi < nb; ++bi) {
        const int v0 = bi * B, nv = n_cams - v0 < B ? n_cams - v0 : B;
        const size_t nvt_b = (size_t)nv * (size_t)TT;
        PlanInfo *info = pl->d_info + bi;
        pa.cams = pl->d_cams + v0; pa.nv = nv;
        pa.zrange = info->b.zrange;
        pa.visible = &info->b.visible;
        pa.total = &info->b.total;
        ca.nv = nv; ca.v0 = v0;
        PK(cudaMemsetAsync(&info->b.zrange[0], 0xff, sizeof(uint32_t), cs));
        PK(launch_project(pa, cs));
        const size_t nwords_b = (size_t)nv * (size_t)((n + 31) / 32);
        PK(scan_vis_words(vis_words, nwords_b, woff, scan_tmp, cs));
        // stage A: 32-bit (view in group, depth) keys, groups of views sorted
        // as segments (one sequence of four 8-bit passes)
        PK(launch_key_params(&info->b, nv, kp, cs));
        PK(emit_vis_words_dev(vis_words, woff, nv, n, geo, zrec, kp, ak0, av0, voff, R, &info->records_over, cs));
        PK(launch_segment_blocks(voff, nv, kp, 0, R, blk_a, nblk_a, cs));
        bool alt_a = false, alt_b = false;
        PK(radix_sort_segments<uint32_t>(ak0, av0, ak1, av1, blk_a, nblk_a, 32, tmp, &alt_a, cs, true));
        const uint32_t *recs = alt_a ? av1 : av0;
        if (counting) {   // stage B by counting, as the batched call
            PK(launch_gather_rects(recs, rect, R, acnt, rect_sorted, cs, &info->b.visible));
            PK(launch_bin_tiles(recs, rect_sorted, voff, nv, n, TW, TT, R, &info->b.visible, bins, ranges, bv0, M,
                                &info->entries_over, cs));
            ca.vals = bv0;
        } else {
            // stage-B offsets per warp of 32 records (acnt, aoff hold the warps' counts and offsets)
            PK(launch_gather_rects(recs, rect, R, acnt, rect_sorted, cs, &info->b.visible));
            PK(exclusive_scan_u32(acnt, aoff, (R + 31) / 32, tmp, nullptr, cs));
            // stage B: tile keys (view << tb) | tile sorted on 16 bits per group
            // of 2^(16 - tb) views when the tile index fits tb <= 16 bits and the
            // batch's views do not (as the batched call), else view * TT + tile
            const int vb = bits_of((uint64_t)nv - 1), tbits = bits_of((uint64_t)TT - 1);
            const int tb = tbits + vb > 16 && tbits <= 16 && ((nv - 1) >> (16 - tbits)) < 64 ? tbits : -1;
            PK(launch_emit_tiles(recs, nullptr, R, rect, n, TW, TH, bk0, bv0, cs, &info->b.visible, M,
                                 &info->entries_over, tb, rect_sorted, aoff));
            if (tb >= 0) {
                PK(launch_entry_offsets_dev(aoff, rect_sorted, voff, nv, &info->b, R, M, eoff, cs));
                PK(launch_segment_blocks(eoff, nv, nullptr, 1 << (16 - tb), M, blk_b, nblk_b, cs));
                PK(radix_sort_segments<uint32_t>(bk0, bv0, bk1, bv1, blk_b, nblk_b, 16, tmp, &alt_b, cs, true));
            } else {
                PK(radix_sort_pairs<uint32_t>(bk0, bv0, bk1, bv1, M, bits_of((uint64_t)nvt_b - 1), tmp, &alt_b, cs,
                                              &info->b.total));
            }
            const uint32_t *keys = alt_b ? bk1 : bk0;
            ca.vals = alt_b ? bv1 : bv0;
            PK(cudaMemsetAsync(ranges, 0, nvt_b * sizeof(uint2), cs));
            PK(launch_ranges(keys, M, ranges, cs, &info->b.total, tb, (uint32_t)TT));
        }
        ca.order = nullptr;
        if (ordered) {   // the batched call's longest-list-first tile order
            PK(launch_order_keys(ranges, nvt_b, ok0, ov0, cs));
            bool alt_o = false;
            PK(radix_sort_pairs<uint32_t>(ok0, ov0, ok1, ov1, nvt_b, 8, tmp, &alt_o, cs, d_nt));
            ca.order = alt_o ? ov1 : ov0;
        }
        PK(launch_composite_ua(ca, cs));
        PK(launch_view_reduce(tile_sums, nv, TT * bpt, 1.0f / ((float)W * (float)H), score + v0, cs));
    }
    if (best_dev) PK(launch_argmax(score, n_cams, best_dev, cs));
    PK(cudaStreamEndCapture(cs, &pl->graph));
    capturing = false;
    pl->kernels = g_launches.load() - k0;
    g_launches.fetch_sub(pl->kernels);   // captured, not run: counted per replay
    PK(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
    cudaStreamDestroy(cs);
    *out = pl;
    return GAVIS_OK;
}

int gavis_plan_launch(gavis_plan *pl, const gavis_camera *cams, void *stream)
{
    if (!pl || !cams) return GAVIS_ERR_ARG;
    for (int k = 0; k < pl->n_cams; ++k)
        if (cams[k].W != pl->W || cams[k].H != pl->H || !(cams[k].fx > 0.0f) || !(cams[k].fy > 0.0f) ||
            !(cams[k].znear > 0.0f))
            return GAVIS_ERR_ARG;
    // the previous replay must have read the staged poses before they change
    if (pl->launched && cudaEventSynchronize(pl->done) != cudaSuccess) return GAVIS_ERR_CUDA;
    std::memcpy(pl->h_cams, cams, (size_t)pl->n_cams * sizeof(gavis_camera));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaGraphLaunch(pl->exec, s) != cudaSuccess || cudaEventRecord(pl->done, s) != cudaSuccess) {
        cudaGetLastError();
        return GAVIS_ERR_CUDA;
    }
    pl->launched = true;
    count_launch(pl->kernels);
    return GAVIS_OK;
}

int gavis_plan_overflowed(gavis_plan *pl, int *overflowed, int64_t *records_needed, int64_t *entries_needed)
{
    if (!pl) return GAVIS_ERR_ARG;
    if (pl->launched && cudaEventSynchronize(pl->done) != cudaSuccess) return GAVIS_ERR_CUDA;
    bool over = false;
    unsigned long long rec = 0, ent = 0;
    for (int bi = 0; bi < pl->n_batches; ++bi) {   // the largest batch decides
        PlanInfo h;
        if (cudaMemcpy(&h, pl->d_info + bi, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return GAVIS_ERR_CUDA;
        over = over || h.entries_over != 0u || h.records_over != 0u || h.b.total > pl->entry_cap ||
               h.b.visible > pl->record_cap;
        rec = h.b.visible > rec ? h.b.visible : rec;
        ent = h.b.total > ent ? h.b.total : ent;
    }
    if (overflowed) *overflowed = pl->launched ? (int)over : 0;
    if (records_needed) *records_needed = pl->launched ? (int64_t)rec : 0;
    if (entries_needed) *entries_needed = pl->launched ? (int64_t)ent : 0;
    return GAVIS_OK;
}

int64_t gavis_plan_kernels(const gavis_plan *pl) { return pl ? (int64_t)pl->kernels : 0; }

void gavis_plan_destroy(gavis_plan *pl)
{
    if (!pl) return;
    if (pl->launched) cudaEventSynchronize(pl->done);
    plan_free(pl);
}

}  // extern "C"
