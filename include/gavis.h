/*
 * gavis.h -- C ABI of the GB300 (sm_103a) GAVIS hot path.
 *
 * GAVIS (arxiv 2605.30342) scores candidate camera views of a 3D Gaussian
 * Splatting scene by the entropy of an uncertainty-aware rendering in which
 * every Gaussian carries an anisotropic visibility field, stored as spherical
 * harmonic (SH) coefficients gamma.  This library implements the two
 * data-parallel halves of that method:
 *
 *   gavis_vf_build     visibility-field construction (Alg. "Anisotropic
 *                      Visibility Field Construction", eq:vis_gamma), using
 *                      Alg. "Single-view Particle Visibility" per training view;
 *   gavis_score_views  visibility-field query (Alg. "Query Anisotropic
 *                      Visibility Field", eq:vis_bound) fused into an
 *                      uncertainty-aware tile rasterizer (Alg. "3DGS Uncertainty
 *                      Quantification with Visibility Field", eq:alpha_comp,
 *                      eq:huber), the per-view score (eq:id without the
 *                      correlation correction) and the next-best-view argmax
 *                      (eq:i_gain).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Arguments documented as "device" are CUDA device pointers on the
 *   context's device; "host" are ordinary host pointers.  The caller owns every
 *   buffer it passes in; the library never frees or retains them after the
 *   call returns.  The context owns a grow-only device workspace bounded by the
 *   budget given at creation.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued asynchronously on it; outputs are valid once the
 *   stream has reached the end of the call's work.  A call may synchronise the
 *   stream internally (to size the sort buffers); this is documented per call.
 *   Calls on one context share its workspace; their GPU work runs in call
 *   order even on different streams (a call's stream first waits for the
 *   previous call's work when that ran on another stream).
 * Threads.  A context is used by one host thread at a time.
 * Errors.  Every function returns GAVIS_OK (0) or a negative status; the text
 *   of the last error is kept in the context (gavis_last_error).  Nothing
 *   aborts the process.  On error no output is guaranteed to be written.
 * Layout.  Gaussians are structure-of-arrays, index g in [0, n):
 *   means[3n] (x,y,z), scales[3n] (activated, > 0), rots[4n] (quaternion
 *   w,x,y,z; normalised inside), opac[n] (in [0,1]), sh[n][(Lc+1)^2][3]
 *   colour coefficients (coefficient-major, then channel), vf coeffs
 *   [n][(L+1)^2].  SH index j = l*l + l + m, real basis as defined in the
 *   paper's derivation of the vMF coefficients.
 * Cameras.  Pinhole, world->camera rotation R (row-major) and translation t,
 *   camera looks along +z with x right and y down; the centre of pixel (i,j)
 *   is at (i + 0.5, j + 0.5).  Every camera in one call has the same W x H.
 */
#ifndef GAVIS_H
#define GAVIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GAVIS_OK            0
#define GAVIS_ERR_ARG      -1   /* invalid argument (null pointer, bad size, mismatched W x H ...) */
#define GAVIS_ERR_CUDA     -2   /* a CUDA runtime call or kernel launch failed */
#define GAVIS_ERR_OOM      -3   /* device allocation failed */
#define GAVIS_ERR_BUDGET   -4   /* the workspace needed exceeds the context budget */
#define GAVIS_ERR_TIMEOUT  -5   /* a bounded device wait gave up */

typedef enum { GAVIS_F32 = 0, GAVIS_F16 = 1, GAVIS_BF16 = 2 } gavis_dtype;

/* 96 bytes; tan_half_fov* = W/(2 fx), H/(2 fy) computed once on the host. */
typedef struct {
    int32_t W, H;
    float fx, fy, cx, cy;
    float tan_half_fovx, tan_half_fovy;
    float R[9];
    float t[3];
    float campos[3];
    float znear;                 /* Gaussians with camera depth <= znear are culled (0.2) */
} gavis_camera;

typedef struct {
    int64_t n;                   /* number of Gaussians, 0 <= n < 2^31 */
    const float *means;          /* device [3n] */
    const float *scales;         /* device [3n] */
    const float *rots;           /* device [4n] */
    const float *opac;           /* device [n] */
    const void *sh;              /* device [n][(sh_degree+1)^2][3], dtype sh_dtype; may be NULL for VF build */
    int32_t sh_degree;           /* 0..3 */
    int32_t sh_dtype;            /* gavis_dtype */
    const void *sh_var;          /* device [n][(sh_degree+1)^2][3] variances of the colour coefficients
                                    (dtype sh_dtype, > 0), or NULL.  When given, the colour covariance of a
                                    Gaussian seen along d is diagonal with Q_k = sum_j Y_j(d)^2 var_jk
                                    (Sec. "Integration with FisherRF"); when NULL, Q_c = sigma_c2 I_3. */
} gavis_gaussians;

typedef struct {
    int64_t n;                   /* must equal the Gaussians' n */
    void *coeffs;                /* device [n][(degree+1)^2] of dtype (gamma of eq:vis_gamma) */
    int32_t degree;              /* L, 0..5 */
    int32_t dtype;               /* gavis_dtype of coeffs */
    int32_t n_train_views;       /* |P| of eq:vis_bound; 0 means "never seen": V = 0 everywhere */
    float kappa;                 /* concentration used to build it */
} gavis_vf;

typedef struct {
    float kappa;                 /* vMF concentration, paper default 1 */
    int32_t vf_degree;           /* SH degree L of the field, paper default 2 */
    float eps_T;                 /* transmittance cutoff, paper default 1e-4 */
    float q_cut;                 /* footprint: a Gaussian covers a pixel iff d^T Sigma^-1 d <= q_cut (9) */
    float beta;                  /* opacity reliability, paper default 0.5 */
    float o0;                    /* prior opacity, paper default 0.15 */
    float sigma_c2;              /* constant colour variance, Q_c = sigma_c2 I_3 (0.01) */
    float logdet_Q0;             /* log |Q_0| of the prior colour covariance, Q_0 = I_3 -> 0 */
    int32_t tile;                /* tile edge in pixels: 8, 16 or 32 (16) */
    int32_t views_per_batch;     /* views per kernel chain: 0 = as many as the budget allows (at most 256), 1 = plain; at most 1024 are used */
    int32_t tile_lists;          /* how each (view, tile) list of depth-ordered Gaussians is built: 0 = automatic (by
                                    counting when the views have at most 2048 tiles and a batch at least 2^20 visible
                                    (view, Gaussian) records, else by sorting the tile entries), 1 = by counting
                                    whenever the views have at most 2048 tiles, 2 = by sorting; the lists, and so
                                    every output, are the same bits either way */
} gavis_params;

typedef struct gavis_ctx gavis_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * workspace; 0 means 60% of the device memory free at creation.  *out is set
 * to NULL on failure.  Returns GAVIS_ERR_CUDA if the device cannot be used. */
int gavis_ctx_create(gavis_ctx **out, int device, size_t hbm_budget_bytes);

/* Free the context and its workspace (synchronises the device first). */
void gavis_ctx_destroy(gavis_ctx *ctx);

/* Text of the last error on this context ("" if none); valid until the next call. */
const char *gavis_last_error(const gavis_ctx *ctx);

/* Fill *p with the paper's defaults (Alg. UQ inputs and the construction
 * hyperparameters): kappa 1, L 2, eps_T 1e-4, q_cut 9, beta 0.5, o0 0.15,
 * sigma_c2 0.01, logdet_Q0 0, tile 16, views_per_batch 0, tile_lists 0. */
int gavis_params_default(gavis_params *p);

/* a_l = 4 pi e^{-kappa} i_l(kappa), l = 0..L (the per-degree factor of
 * eq:vis_gamma; i_l the modified spherical Bessel function of the first kind).
 * a: host [L+1].  L in 0..5, kappa >= 0. */
int gavis_vmf_coeffs(int L, double kappa, double *a);

/* Visibility-field construction (Alg. "Anisotropic Visibility Field
 * Construction").  For every training view p: the per-Gaussian visibility
 * v_p[g] = (sum of transmittance over the pixels that reach g) / (their count),
 * 0 if no pixel reaches g (Alg. "Single-view Particle Visibility"); then
 * gamma_lm[g] += v_p[g] a_l Y_lm(normalize(x_g - x_p)).
 *   train: host [n_train] cameras (same W x H); n_train >= 0.
 *   out: caller-filled n, coeffs (device, n x (L+1)^2 of out->dtype), degree,
 *        dtype; the call sets n_train_views = n_train and kappa = p->kappa.
 *   accumulate: 0 overwrites coeffs; 1 adds the new views' contributions to
 *        the coefficients already there and adds n_train to n_train_views
 *        (eq:vis_gamma is a sum over views).
 * Accumulates in float32, stores in out->dtype.  Synchronises `stream` once per
 * batch of views (to size the sort). */
int gavis_vf_build(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_camera *train, int n_train,
                   const gavis_params *p, gavis_vf *out, int accumulate, void *stream);

/* Candidate-view scoring.  For every candidate view c: V[g] by the AM-GM bound
 * of eq:vis_bound from gamma (|P| = vf->n_train_views), colour from the SH
 * coefficients, then per pixel front-to-back compositing of the plain colour
 * (eq:orig_vr) and of the uncertainty (Alg. UQ: eq:alpha_comp weights, the
 * Huber entropy bound eq:huber with Q_c = sigma_c2 I_3 and the prior Q_0).
 *   cand: host [n_cand] cameras, same W x H.
 *   rgb:  device [n_cand][3][H][W] float32 (planar) or NULL.
 *   unc:  device [n_cand][H][W] float32 per-pixel entropy bound, or NULL.
 *   score: device [n_cand] float32, mean over pixels of unc (eq:id, f_corr = 0).
 *   best_dev: device int32 argmax of score (lowest index on ties) or NULL.
 *   best_host: host int32 or NULL; if given the call synchronises `stream`.
 * Synchronises `stream` once per batch of views (to size the sort). */
int gavis_score_views(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf,
                      const gavis_camera *cand, int n_cand, const gavis_params *p,
                      float *rgb, float *unc, float *score, int32_t *best_dev, int32_t *best_host,
                      void *stream);

/* Outputs of gavis_render_views.  Any pointer may be NULL except score. */
typedef struct {
    float *rgb;           /* device [n_cand][3][H][W], as for gavis_score_views */
    float *unc;           /* device [n_cand][H][W] */
    float *depth;         /* device [n_cand][H][W]: the expected depth d of eq:id, the sum over the
                             colour weights alpha_i T_c,i of eq:orig_vr of the Gaussians' camera depths
                             (background 0; divide by the accumulated opacity 1 - T_c for the
                             normalised depth) */
    float *score;         /* device [n_cand] */
    int32_t *best_dev;    /* device [1] */
    int32_t *best_host;   /* host [1]; if given the call synchronises `stream` */
} gavis_views_out;

/* gavis_score_views with the optional per-pixel expected depth (the input of
 * the correction term f_corr of eq:id, which this library takes as 0).
 * Same arguments, errors and synchronisation as gavis_score_views. */
int gavis_render_views(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cand,
                       int n_cand, const gavis_params *p, const gavis_views_out *out, void *stream);

/* Visibility-field density control (Alg. "Visibility Field Density Control").
 * Virtual particles at the caller-drawn centres virt_means (device [3 n_virt],
 * uniform in the scene volume; their number is floor(rho * volume)) get an
 * identity rotation, the isotropic scale s with (4/3) pi s^3 rho = 1 + eta and
 * zero opacity.  Alg. "Single-view Particle Visibility" runs on the union of
 * the scene and the virtual particles for every training view (virtual
 * particles are transparent), and each virtual particle's multi-view
 * visibility is 1 - prod_p (1 - v_p).  Particles with visibility <= eps_v lie
 * in under-explored space and are kept; the others (free space) are pruned.
 * Kept particles enter uncertainty scoring with gamma = 0, i.e. V = 0.
 *   vis_out: device [n_virt] float32 or NULL; keep: device [n_virt] uint8 (0/1);
 *   kept_means: device [3 n_virt] or NULL, receives the kept centres in input
 *   order; n_keep: host or NULL (synchronises `stream`); scale_out: host or NULL.
 * Paper defaults: rho 100, eta 0.5, eps_v 0.95. */
int gavis_vf_density_control(gavis_ctx *ctx, const gavis_gaussians *gs, const float *virt_means, int64_t n_virt,
                             const gavis_camera *train, int n_train, const gavis_params *p, float rho, float eta,
                             float eps_v, float *vis_out, uint8_t *keep, float *kept_means, int64_t *n_keep,
                             float *scale_out, void *stream);

/* The scene that Alg. "Visibility Field Density Control" hands to the
 * uncertainty step: the n trained Gaussians followed by the n_kept virtual
 * particles kept by gavis_vf_density_control, each with the identity
 * rotation, the isotropic `scale` (its scale_out), opacity 0, colour 0 and a
 * zero visibility field, so that V = 0 and only the prior term of
 * eq:alpha_comp remains for it.
 *   gs, vf: the scene and its field (device, as for gavis_score_views).
 *   kept_means: device [3 n_kept] float32.
 *   means, scales (device [3(n + n_kept)]), rots (device [4(n + n_kept)],
 *   16-byte aligned), opac (device [n + n_kept]): float32 outputs;
 *   sh: device [(n + n_kept)][(Lc+1)^2][3] of gs->sh_dtype;
 *   sh_var: same shape and dtype, required exactly when gs->sh_var is given
 *   (the virtual particles get variance 1), else NULL;
 *   coeffs: device [(n + n_kept)][(L+1)^2] of vf->dtype.
 * Outputs are caller-allocated and must not overlap the inputs.  Only
 * device-to-device copies and one fill kernel on `stream`; no
 * synchronisation.  Errors: GAVIS_ERR_ARG for NULL or inconsistent
 * arguments, GAVIS_ERR_CUDA if a copy or launch fails. */
int gavis_augment(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const float *kept_means,
                  int64_t n_kept, float scale, float *means, float *scales, float *rots, float *opac, void *sh,
                  void *sh_var, void *coeffs, void *stream);

/* Autotuner (no counterpart in the paper): times the chain on the sample
 * cameras with tile edges 8, 16 and 32 (one warm-up and two timed runs each,
 * CUDA events on `stream`) and writes the fastest into p->tile.  mode 0 tunes
 * gavis_score_views with colour, uncertainty and scores written (vf
 * required), mode 1 gavis_vf_build (vf ignored).
 * Choices are cached per workload shape (mode, W x H, power-of-two buckets of
 * the Gaussian and camera counts, SH degrees) in the process, and appended to
 * the file named by the environment variable GAVIS_AUTOTUNE_CACHE when set
 * (read back on first use); a cached choice returns at once with *best_ms =
 * -1.  best_ms: host or NULL.  Synchronises `stream`. */
int gavis_autotune(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cams, int n_cams,
                   int mode, gavis_params *p, double *best_ms, void *stream);

/* Visibility-field query alone (Alg. "Query Anisotropic Visibility Field").
 * V: device [n_cams][n] float32.  Culling is not applied: every Gaussian gets
 * a value. */
int gavis_vf_query(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf,
                   const gavis_camera *cams, int n_cams, const gavis_params *p, float *V, void *stream);

/* Tile bins of views, for verification.  Keys are
 * ((view * TW*TH + tile) << 32) | float_bits(camera depth), values Gaussian
 * indices, sorted by key with ties in ascending index.  keys/vals: device
 * [cap]; *M_out (host) receives the number of keys (only min(M, cap) are
 * written); ranges: device [n_cams*TW*TH][2] uint32 [start, end) or NULL.
 * n_cams <= 1024 (GAVIS_ERR_ARG beyond).  Synchronises `stream`. */
int gavis_debug_bins(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_camera *cams, int n_cams,
                     const gavis_params *p, uint64_t *keys, uint32_t *vals, int64_t cap,
                     int64_t *M_out, uint32_t *ranges, void *stream);

/* Per-view particle visibility sums (Alg. "Single-view Particle
 * Visibility"), for verification.  sumT: device [n_cams][n] float32 (sum of
 * transmittance over the pixels that reach g); cnt: device [n_cams][n] uint32
 * (number of those pixels). */
int gavis_debug_visibility(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_camera *cams,
                           int n_cams, const gavis_params *p, float *sumT, uint32_t *cnt, void *stream);

/* Allocation-free scoring of ONE candidate view (no counterpart in the paper:
 * an interface addition for callers that cannot allocate device memory).
 * Who needs it: applications whose memory manager has already reserved the
 * GPU's memory for its own pool, so that a raw cudaMalloc would fail or
 * fragment that pool, and real-time loops that cannot accept the device-wide
 * synchronisation cudaMalloc/cudaFree may imply.  The call computes exactly
 * what gavis_score_views computes for a single camera (same kernels), but all
 * scratch memory lives in a fixed 16 MiB array inside the library's device
 * image; it allocates nothing (no cudaMalloc, no pinned host memory, no
 * library allocator) and needs no context.
 *   gs, vf: as for gavis_score_views.  cam: host, one camera.
 *   rgb: device [3][H][W] or NULL; unc: device [H][W] or NULL; score: device [1].
 *   err: optional host buffer of err_len bytes for the error text.
 * Limits: n <= 32768 Gaussians, at most 4096 tiles (e.g. 1024 x 1024 pixels at
 *   tile 16), at most 2^19 tile keys; beyond them the call returns
 *   GAVIS_ERR_ARG (sizes) or GAVIS_ERR_BUDGET (keys) with a message and
 *   launches nothing further.
 * Set-up: the first successful call on each device looks up the array's
 *   device address (with that device current) and keeps it; a failed lookup
 *   is retried by the next call.  Make that first call before any stream
 *   capture.  The kept address belongs to the device's current context: after
 *   cudaDeviceReset it is stale, so do not call this entry point again in
 *   that process.  The array is held by every GPU that loads this library
 *   until the process exits.
 * Sharing: every call on a device uses the same array, which keeps the last
 *   call's contents; calls whose GPU work overlaps (other streams or threads)
 *   race on it and must be serialised by the caller.
 * Synchronises `stream` once (to read the number of tile keys). */
int gavis_score_view_noalloc(const gavis_gaussians *gs, const gavis_vf *vf, const gavis_camera *cam,
                             const gavis_params *p, float *rgb, float *unc, float *score, char *err,
                             size_t err_len, void *stream);

/* ---------------------------------------------------------------------- */
/* Scoring plans (no counterpart in the paper): the candidate-scoring chain  */
/* of gavis_score_views (projection with VF QUERY, Eq. for alpha*, the        */
/* Huber entropy bound, the per-view mean and the argmax of Eq. for i*)      */
/* captured once as a CUDA graph and replayed for new candidate poses.       */
/* ---------------------------------------------------------------------- */
typedef struct gavis_plan gavis_plan;

/* Build a plan for n_cams (1..16384) candidate views of W x H pixels over
 * one scene and field.  The views go through the chain in batches of
 * p->views_per_batch (0: all in one batch; at most 1024), replayed one after another over
 * the same buffers.  The plan allocates all its device memory here, for one
 * batch: one projected record per (view, Gaussian), sort space for
 * record_capacity visible (view, Gaussian) records (0 = views x n, always
 * enough) and for entry_capacity tile entries.  Good values are 1.25 x the
 * largest batch's visible-record and tile-key counts (gavis_prof_read gives
 * totals; gavis_plan_overflowed gives the largest batch's after a launch);
 * grids are sized by the capacities, so oversizing them costs time.  gs, vf, p: as for gavis_score_views; gs and vf stay owned by the
 * caller and must stay alive at the same addresses while the plan is used.
 * The plan captures the sizes, dtypes and |P| (vf->n_train_views); the
 * values behind the pointers are read at every launch, so they may be
 * rewritten between launches (e.g. Gaussians refined in place).  rgb (device [n_cams][3][H][W] or NULL), unc (device
 * [n_cams][H][W] or NULL), score (device [n_cams]) and best_dev (device [1]
 * int32 or NULL) are written by every launch.  *out receives the plan.
 * Errors: GAVIS_ERR_ARG for invalid sizes or parameters (tile must be 8, 16
 * or 32: no autotuning), GAVIS_ERR_CUDA if allocation or capture fails; the
 * message is in gavis_last_error(ctx). */
int gavis_plan_create(gavis_ctx *ctx, const gavis_gaussians *gs, const gavis_vf *vf, int n_cams, int W, int H,
                      const gavis_params *p, int64_t record_capacity, int64_t entry_capacity, float *rgb,
                      float *unc, float *score, int32_t *best_dev, gavis_plan **out);

/* Score the poses cams (host [n_cams], each W x H as at creation) by
 * replaying the graph on `stream`.  The poses are copied into the plan's
 * pinned staging buffer first, after waiting for the previous launch of this
 * plan to finish; the call does not otherwise wait for the GPU.  Results
 * equal gavis_score_views' for the same inputs bit for bit, unless the launch
 * needed more visible records or tile entries than the capacities: then the
 * excess is dropped (the results are incomplete) and gavis_plan_overflowed
 * reports it.  One plan is used from one thread at a
 * time. */
int gavis_plan_launch(gavis_plan *plan, const gavis_camera *cams, void *stream);

/* After the last launch finishes (the call waits for it): *overflowed = 1 if
 * a batch needed more visible records or tile entries than the capacities;
 * *records_needed and *entries_needed = the largest numbers a batch needed.
 * Any pointer may be NULL. */
int gavis_plan_overflowed(gavis_plan *plan, int *overflowed, int64_t *records_needed, int64_t *entries_needed);

/* Kernels one launch runs (for launch accounting). */
int64_t gavis_plan_kernels(const gavis_plan *plan);

/* Waits for the last launch and frees the plan.  NULL is ignored. */
void gavis_plan_destroy(gavis_plan *plan);

/* ---------------------------------------------------------------------- */
/* Serving (no counterpart in the paper): continuous batching of scoring     */
/* requests over resident scenes.                                             */
/* ---------------------------------------------------------------------- */
typedef struct gavis_server gavis_server;

/* Start a server on `device` with n_workers worker threads (1..16), each with
 * its own CUDA stream and workspace (hbm_budget_bytes / n_workers; 0 = 60% of
 * free memory in total), batching at most max_views_per_batch views (1..1024).
 * Requests are admitted in arrival order while the sum of the admitted
 * requests' workspace estimates fits hbm_budget_bytes. */
int gavis_server_create(gavis_server **out, int device, size_t hbm_budget_bytes, int n_workers,
                        int max_views_per_batch);

/* Stop the workers (after the batches in flight) and free the server. */
void gavis_server_destroy(gavis_server *s);

const char *gavis_server_last_error(const gavis_server *s);

/* Register a resident scene; gs and vf point to caller-owned device memory
 * that must stay valid until the server is destroyed.  *scene_id receives
 * its index. */
int gavis_server_add_scene(gavis_server *s, const gavis_gaussians *gs, const gavis_vf *vf, int *scene_id);

/* Queue a scoring request: the host cameras are copied (one W x H per
 * request); score (device [n_cams]) and unc (device [n_cams][H][W] or NULL)
 * must stay valid until gavis_server_wait returns for it.  The views of a
 * request may be scored across several batches and share batches with other
 * requests on the same scene, resolution and parameters; every view gets the
 * result gavis_score_views gives it. */
int gavis_server_submit(gavis_server *s, int scene_id, const gavis_camera *cams, int n_cams, const gavis_params *p,
                        float *score, float *unc, int64_t *request_id);

/* Wait up to timeout_ms for a request; on completion returns its status and
 * sets *best (argmax of its scores, lowest index on ties) and *latency_ms
 * (submit to completion), and forgets the request.  Returns GAVIS_ERR_TIMEOUT
 * (request kept) if it is not finished in time. */
int gavis_server_wait(gavis_server *s, int64_t request_id, int timeout_ms, int32_t *best, double *latency_ms);

/* Pause (paused = 1) or resume (0) the workers: while paused they finish the
 * batch in flight and start no new one; submissions and admission go on, and
 * gavis_server_wait keeps its timeout (for draining a device, and for
 * testing the timeout path). */
int gavis_server_pause(gavis_server *s, int paused);

/* Counters: views scored, batches run, the most requests one batch served,
 * the peak of the admitted workspace estimates and the budget. */
int gavis_server_stats(gavis_server *s, int64_t *views_scored, int64_t *batches, int64_t *max_requests_in_batch,
                       size_t *peak_reserved_bytes, size_t *budget_bytes);

/* ---------------------------------------------------------------------- */
/* Instrumentation (no counterpart in the paper): per-stage device time from  */
/* CUDA events recorded on the call's stream, kernel launch counts, and the   */
/* number of (pixel, Gaussian) pairs composited.                             */
/* ---------------------------------------------------------------------- */
enum {
    GAVIS_STAGE_PROJECT = 0,      /* projection, culling, colour, VF query */
    GAVIS_STAGE_SCAN = 1,         /* exclusive scan of tile counts */
    GAVIS_STAGE_EMIT = 2,         /* key emission */
    GAVIS_STAGE_SORT = 3,         /* radix sort */
    GAVIS_STAGE_RANGES = 4,       /* tile ranges */
    GAVIS_STAGE_COMPOSITE_UA = 5, /* uncertainty + colour compositing */
    GAVIS_STAGE_COMPOSITE_VIS = 6,/* particle-visibility compositing */
    GAVIS_STAGE_REDUCE = 7,       /* per-view score and argmax */
    GAVIS_STAGE_VF_ACCUM = 8,     /* SH accumulation of the field */
    GAVIS_STAGE_COUNT = 9
};

/* on = 1 starts recording stage events on later calls (two events per stage
 * and batch); on = 2 also counts the composited pixel-Gaussian pairs on the
 * device (counters in the composite kernels: slower); 0 stops.  Every call
 * resets the accumulators. */
int gavis_prof_enable(gavis_ctx *ctx, int on);

/* Synchronises the device, then returns per stage the summed device time
 * (ms[GAVIS_STAGE_COUNT], host) and kernel launches (launches[...], host) since
 * gavis_prof_enable, the total number of kernels this library launched in the
 * process (*total_launches, host) and the work counted (pairs[0] pairs
 * composited by the uncertainty pass, pairs[1] by the visibility pass,
 * pairs[2] tile entries (one per record and tile of its rectangle),
 * pairs[3] visible (view, Gaussian) records, pairs[4] the tile entries whose
 * lists were built by sorting (the others were counted: gavis_params
 * tile_lists); host [5]).  Any output pointer may be NULL. */
int gavis_prof_read(gavis_ctx *ctx, double *ms, int64_t *launches, int64_t *total_launches, uint64_t *pairs);

#ifdef __cplusplus
}
#endif
#endif /* GAVIS_H */
