// server.cu -- serving loop for candidate-view scoring with continuous
// batching (no counterpart in the paper; it serves the paper's per-planning-
// step scoring to many concurrent clients).
//
// Scenes (Gaussians + visibility field) stay resident in caller-owned device
// memory.  Requests (a scene, a set of candidate cameras of one resolution,
// parameters, output buffers) are queued on arrival and *admitted* while the
// sum of the admitted requests' workspace estimates fits the HBM budget.
// Worker threads, each with its own context (workspace) and CUDA stream, take
// the oldest admitted request that still has unscored views, fill a batch
// with pending views of every admitted request that shares its scene,
// resolution and parameters (in arrival order, up to the batch size), and run
// the scoring chain on it.  A request that arrives while others are on the
// GPU joins the next batch that has room, and requests on different scenes
// overlap on the device through the workers' streams.  Each view is scored by
// the same kernels whatever batch it lands in, so a request's results are the
// same alone and in a mix.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gavis_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id;
    int scene;
    std::vector<gavis_camera> cams;
    gavis_params p;
    float *score, *unc;
    int next = 0;          // next view not yet taken by a batch
    int done = 0;          // views scored
    bool admitted = false;
    bool finished = false;
    int status = GAVIS_OK;
    int32_t best = -1;
    size_t reserve = 0;    // bytes reserved against the budget while admitted
    Clock::time_point t_submit, t_done;
};

struct Scene {
    gavis_gaussians gs;
    gavis_vf vf;
};

bool same_group(const Request &a, const Request &b)
{
    return a.scene == b.scene && a.cams[0].W == b.cams[0].W && a.cams[0].H == b.cams[0].H &&
           std::memcmp(&a.p, &b.p, sizeof(gavis_params)) == 0;
}

}  // namespace

struct gavis_server {
    int device = 0;
    size_t budget = 0, reserved = 0, peak_reserved = 0;
    int max_batch = 64;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    bool paused = false;   // workers take no new batch while set
    std::vector<Scene> scenes;
    std::deque<std::shared_ptr<Request>> waiting;            // not yet admitted, arrival order
    std::vector<std::shared_ptr<Request>> active;            // admitted, arrival order
    std::map<int64_t, std::shared_ptr<Request>> all;         // until collected by wait
    int64_t next_id = 1;
    std::vector<std::thread> workers;
    std::string err;
    // statistics
    int64_t views_scored = 0, batches = 0, max_requests_in_batch = 0;
};

namespace {

int sfail(gavis_server *s, int code, const char *msg)
{
    if (s) s->err = msg;
    return code;
}

// Workspace estimate of one admitted request on one scene: the views of it
// that can be in flight at once (at most one batch), each with the projected
// records of every Gaussian, stage-A keys for every Gaussian (an upper
// bound), stage-B tile entries for a quarter of the Gaussians visible at four
// tiles each (the measured scale of the room workloads at tile 16; the true
// count depends on the poses), and the staging of its uncertainty map.  An
// estimate: what the workers allocate is bounded by their contexts' budgets
// (budget / workers each), and a batch whose keys do not fit one context is
// halved.
size_t estimate_bytes(const Scene &sc, const Request &r, int max_batch)
{
    const size_t n = (size_t)sc.gs.n;
    const size_t v = r.cams.size() < (size_t)max_batch ? r.cams.size() : (size_t)max_batch;
    const size_t plane = (size_t)r.cams[0].W * r.cams[0].H;
    return v * (n * (sizeof(gavis::GeoRec) + sizeof(gavis::UaRec) + 16) + n * 2 * 24 + n / 4 * 4 * 16 + plane * 4 +
                64);
}

// admit waiting requests in arrival order while they fit the budget (a
// request larger than the whole budget is admitted alone)
void admit_locked(gavis_server *s)
{
    while (!s->waiting.empty()) {
        auto &r = s->waiting.front();
        if (s->reserved + r->reserve > s->budget && !(s->active.empty() && s->reserved == 0)) break;
        r->admitted = true;
        s->reserved += r->reserve;
        if (s->reserved > s->peak_reserved) s->peak_reserved = s->reserved;
        s->active.push_back(r);
        s->waiting.pop_front();
    }
}

struct Slot {   // one view of a batch
    std::shared_ptr<Request> req;
    int view;
};

void worker_main(gavis_server *s, size_t ws_budget)
{
    // a worker whose set-up failed stays up and fails every batch it takes
    // with that status (no batch runs on a missing stream or buffer)
    int rc0 = GAVIS_OK;
    if (cudaSetDevice(s->device) != cudaSuccess) rc0 = GAVIS_ERR_CUDA;
    cudaStream_t stream = nullptr;
    if (rc0 == GAVIS_OK && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        stream = nullptr;
        rc0 = GAVIS_ERR_CUDA;
    }
    gavis_ctx *ctx = nullptr;
    if (rc0 == GAVIS_OK) rc0 = gavis_ctx_create(&ctx, s->device, ws_budget);
    float *score_stage = nullptr, *unc_stage = nullptr;
    size_t unc_cap = 0;
    int32_t *d_best = nullptr;
    if (rc0 == GAVIS_OK && cudaMalloc(&score_stage, sizeof(float) * (size_t)s->max_batch) != cudaSuccess) {
        score_stage = nullptr;
        rc0 = GAVIS_ERR_OOM;
    }
    if (rc0 == GAVIS_OK && cudaMalloc(&d_best, sizeof(int32_t)) != cudaSuccess) {
        d_best = nullptr;
        rc0 = GAVIS_ERR_OOM;
    }
    if (rc0 != GAVIS_OK) cudaGetLastError();
    std::vector<gavis_camera> cams;
    std::vector<Slot> slots;
    for (;;) {
        slots.clear();
        Scene sc;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->stop) return true;
                if (s->paused) return false;
                for (auto &r : s->active)
                    if (r->next < (int)r->cams.size()) return true;
                return false;
            });
            if (s->stop) break;
            // the oldest admitted request with pending views leads the batch
            std::shared_ptr<Request> lead;
            for (auto &r : s->active)
                if (r->next < (int)r->cams.size()) {
                    lead = r;
                    break;
                }
            int nreq = 0;
            for (auto &r : s->active) {
                if ((int)slots.size() >= s->max_batch) break;
                if (r->next >= (int)r->cams.size() || !same_group(*lead, *r)) continue;
                ++nreq;
                while (r->next < (int)r->cams.size() && (int)slots.size() < s->max_batch) slots.push_back({r, r->next++});
            }
            s->batches += 1;
            if (nreq > s->max_requests_in_batch) s->max_requests_in_batch = nreq;
            sc = s->scenes[lead->scene];
        }
        // run the batch outside the lock
        const Request &lead = *slots[0].req;
        const int nb = (int)slots.size();
        const size_t plane = (size_t)lead.cams[0].W * lead.cams[0].H;
        bool want_unc = false;
        cams.resize(nb);
        for (int k = 0; k < nb; ++k) {
            cams[k] = slots[k].req->cams[slots[k].view];
            want_unc = want_unc || slots[k].req->unc;
        }
        int rc = rc0;
        if (rc == GAVIS_OK && want_unc && unc_cap < (size_t)nb * plane) {
            // stream-ordered on the worker's stream: other workers' streams never wait for it
            if (unc_stage) cudaFreeAsync(unc_stage, stream);
            unc_stage = nullptr;
            unc_cap = 0;
            const size_t want = (size_t)s->max_batch * plane;
            if (cudaMallocAsync(reinterpret_cast<void **>(&unc_stage), want * sizeof(float), stream) == cudaSuccess) {
                unc_cap = want;
            } else {
                unc_stage = nullptr;
                cudaGetLastError();
                rc = GAVIS_ERR_OOM;
            }
        }
        if (rc == GAVIS_OK) {
            gavis_params p = lead.p;
            p.views_per_batch = nb;
            rc = gavis_score_views(ctx, &sc.gs, &sc.vf, cams.data(), nb, &p, nullptr, want_unc ? unc_stage : nullptr,
                                   score_stage, nullptr, nullptr, stream);
        }
        if (rc == GAVIS_OK) {
            for (int k = 0; k < nb && rc == GAVIS_OK; ++k) {
                Request &r = *slots[k].req;
                if (cudaMemcpyAsync(r.score + slots[k].view, score_stage + k, sizeof(float), cudaMemcpyDeviceToDevice,
                                    stream) != cudaSuccess)
                    rc = GAVIS_ERR_CUDA;
                if (r.unc && cudaMemcpyAsync(r.unc + (size_t)slots[k].view * plane, unc_stage + (size_t)k * plane,
                                             plane * sizeof(float), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
                    rc = GAVIS_ERR_CUDA;
            }
        }
        if (stream && cudaStreamSynchronize(stream) != cudaSuccess && rc == GAVIS_OK) rc = GAVIS_ERR_CUDA;
        // completion: argmax of every request whose last view is in
        std::vector<std::shared_ptr<Request>> completed;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->views_scored += nb;
            for (int k = 0; k < nb; ++k) {
                Request &r = *slots[k].req;
                r.done += 1;
                if (rc != GAVIS_OK) r.status = rc;
                if (r.done == (int)r.cams.size()) completed.push_back(slots[k].req);
            }
        }
        for (auto &r : completed) {
            int32_t best = -1;
            if (r->status == GAVIS_OK) {
                if (gavis::launch_argmax(r->score, (int)r->cams.size(), d_best, stream) != cudaSuccess ||
                    cudaMemcpyAsync(&best, d_best, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                    cudaStreamSynchronize(stream) != cudaSuccess)
                    r->status = GAVIS_ERR_CUDA;
            }
            std::lock_guard<std::mutex> lk(s->mu);
            r->best = best;
            r->finished = true;
            r->t_done = Clock::now();
            s->reserved -= r->reserve;
            for (size_t k = 0; k < s->active.size(); ++k)
                if (s->active[k].get() == r.get()) {
                    s->active.erase(s->active.begin() + (long)k);
                    break;
                }
            admit_locked(s);
        }
        if (!completed.empty()) {
            s->cv_done.notify_all();
            s->cv_work.notify_all();
        }
    }
    if (ctx) gavis_ctx_destroy(ctx);
    if (score_stage) cudaFree(score_stage);
    if (unc_stage) cudaFreeAsync(unc_stage, stream);
    if (stream) cudaStreamSynchronize(stream);
    if (d_best) cudaFree(d_best);
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

int gavis_server_create(gavis_server **out, int device, size_t hbm_budget_bytes, int n_workers, int max_views_per_batch)
{
    if (!out || n_workers < 1 || n_workers > 16 || max_views_per_batch < 1 || max_views_per_batch > 1024)
        return GAVIS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GAVIS_ERR_CUDA;
    }
    cudaSetDevice(device);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return GAVIS_ERR_CUDA;
    gavis_server *s = new gavis_server();
    s->device = device;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : fr / 10 * 6;
    s->max_batch = max_views_per_batch;
    for (int k = 0; k < n_workers; ++k) s->workers.emplace_back(worker_main, s, s->budget / (size_t)n_workers);
    *out = s;
    return GAVIS_OK;
}

void gavis_server_destroy(gavis_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
}

const char *gavis_server_last_error(const gavis_server *s) { return s ? s->err.c_str() : "no server"; }

int gavis_server_pause(gavis_server *s, int paused)
{
    if (!s) return GAVIS_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_all();
    return GAVIS_OK;
}

int gavis_server_add_scene(gavis_server *s, const gavis_gaussians *gs, const gavis_vf *vf, int *scene_id)
{
    if (!s || !gs || !vf || !scene_id) return sfail(s, GAVIS_ERR_ARG, "NULL argument");
    if (vf->n != gs->n || gs->n < 0 || (gs->n > 0 && (!gs->sh || !vf->coeffs)))
        return sfail(s, GAVIS_ERR_ARG, "scene and visibility field disagree");
    std::lock_guard<std::mutex> lk(s->mu);
    s->scenes.push_back({*gs, *vf});
    *scene_id = (int)s->scenes.size() - 1;
    return GAVIS_OK;
}

int gavis_server_submit(gavis_server *s, int scene_id, const gavis_camera *cams, int n_cams, const gavis_params *p,
                        float *score, float *unc, int64_t *request_id)
{
    if (!s || !cams || !p || !score || !request_id || n_cams < 1) return sfail(s, GAVIS_ERR_ARG, "bad argument");
    for (int k = 1; k < n_cams; ++k)
        if (cams[k].W != cams[0].W || cams[k].H != cams[0].H)
            return sfail(s, GAVIS_ERR_ARG, "all cameras of a request share W x H");
    auto r = std::make_shared<Request>();
    r->scene = scene_id;
    r->cams.assign(cams, cams + n_cams);
    r->p = *p;
    r->p.views_per_batch = 0;
    r->score = score;
    r->unc = unc;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (scene_id < 0 || scene_id >= (int)s->scenes.size()) return sfail(s, GAVIS_ERR_ARG, "unknown scene");
        r->reserve = estimate_bytes(s->scenes[scene_id], *r, s->max_batch);
        r->id = s->next_id++;
        s->all[r->id] = r;
        s->waiting.push_back(r);
        admit_locked(s);
        *request_id = r->id;
    }
    s->cv_work.notify_all();
    return GAVIS_OK;
}

int gavis_server_wait(gavis_server *s, int64_t request_id, int timeout_ms, int32_t *best, double *latency_ms)
{
    if (!s) return GAVIS_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end()) return sfail(s, GAVIS_ERR_ARG, "unknown request");
    std::shared_ptr<Request> r = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return r->finished; });
    if (!ok) return sfail(s, GAVIS_ERR_TIMEOUT, "request not finished within the timeout");
    if (best) *best = r->best;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->all.erase(it);
    return r->status;
}

int gavis_server_stats(gavis_server *s, int64_t *views_scored, int64_t *batches, int64_t *max_requests_in_batch,
                       size_t *peak_reserved_bytes, size_t *budget_bytes)
{
    if (!s) return GAVIS_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (views_scored) *views_scored = s->views_scored;
    if (batches) *batches = s->batches;
    if (max_requests_in_batch) *max_requests_in_batch = s->max_requests_in_batch;
    if (peak_reserved_bytes) *peak_reserved_bytes = s->peak_reserved;
    if (budget_bytes) *budget_bytes = s->budget;
    return GAVIS_OK;
}

}  // extern "C"
