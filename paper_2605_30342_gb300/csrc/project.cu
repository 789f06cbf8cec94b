// project.cu -- per (view, Gaussian) projection, culling, colour and
// visibility-field query.
//
// One thread per Gaussian; the thread loads the Gaussian's parameters once
// (centre, scale, rotation, opacity, colour SH, visibility-field SH) and loops
// over every view of the batch, whose cameras sit in shared memory.  The
// Gaussian record is therefore read from HBM once per batch rather than once
// per view.  Views go in groups of 32.  In the geometry-only launches (field
// construction) the warp deals its (view, Gaussian) projections out to its
// lanes, 32 per round, so that no lane idles while another has views left;
// in the launches with appearance records each lane projects (and then
// colours) its own Gaussian's views in rounds over the lanes with a view
// left, because its 64 colour and field coefficients stay in its registers
// (dealing there spilled and measured no faster).
//
// Image-space geometry is evaluated with explicit round-to-nearest intrinsics
// (no contraction) in a fixed operation order, so that depth keys, conics and
// tile rectangles are reproducible bit for bit by any IEEE-754 float32
// implementation of the same sequence: 3DGS EWA projection (Sigma2D = J W
// Sigma3D W^T J^T + 0.3 I, Jacobian with the 1.3 tan(fov/2) clamp), conic =
// Sigma2D^-1, a footprint of q = d^T conic d <= q_cut, and the tile rectangle
// of the footprint's bounding box inflated by 2^-10 (relative and absolute).
//
// The visibility field is queried here (Alg. "Query Anisotropic Visibility
// Field"): V~ = sum_j gamma_j Y_j(d), d = normalize(x_g - x_cam), clamped to
// [0, |P|], then V = 1 - (1 - V~/|P|)^|P| (eq:vis_bound), evaluated as
// -expm1(|P| log1p(-V~/|P|)).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gavis_internal.cuh"
#include "sh_basis.cuh"

namespace gavis {
namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ float ld_coef(const void *p, size_t i, int dtype)
{
    if (dtype == GAVIS_F16) return __half2float(reinterpret_cast<const __half *>(p)[i]);
    if (dtype == GAVIS_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
    return reinterpret_cast<const float *>(p)[i];
}

struct Sigma3 {
    float s00, s01, s02, s11, s12, s22;
};

// Sigma3D = (R S)(R S)^T from a quaternion (w,x,y,z) and scales.
__device__ __forceinline__ Sigma3 sigma3d(const float *sc, float qw, float qx, float qy, float qz)
{
    float qn = __fsqrt_rn(fa(fa(fa(fm(qw, qw), fm(qx, qx)), fm(qy, qy)), fm(qz, qz)));
    qw = fd(qw, qn); qx = fd(qx, qn); qy = fd(qy, qn); qz = fd(qz, qn);
    float xx = fm(qx, qx), yy = fm(qy, qy), zz = fm(qz, qz);
    float xy = fm(qx, qy), xz = fm(qx, qz), yz = fm(qy, qz);
    float wx = fm(qw, qx), wy = fm(qw, qy), wz = fm(qw, qz);
    float G[9];
    G[0] = fs(1.0f, fm(2.0f, fa(yy, zz))); G[1] = fm(2.0f, fs(xy, wz));        G[2] = fm(2.0f, fa(xz, wy));
    G[3] = fm(2.0f, fa(xy, wz));        G[4] = fs(1.0f, fm(2.0f, fa(xx, zz))); G[5] = fm(2.0f, fs(yz, wx));
    G[6] = fm(2.0f, fs(xz, wy));        G[7] = fm(2.0f, fa(yz, wx));        G[8] = fs(1.0f, fm(2.0f, fa(xx, yy)));
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = fm(G[3 * i + j], sc[j]);
    Sigma3 S;
    S.s00 = fa(fa(fm(M[0], M[0]), fm(M[1], M[1])), fm(M[2], M[2]));
    S.s01 = fa(fa(fm(M[0], M[3]), fm(M[1], M[4])), fm(M[2], M[5]));
    S.s02 = fa(fa(fm(M[0], M[6]), fm(M[1], M[7])), fm(M[2], M[8]));
    S.s11 = fa(fa(fm(M[3], M[3]), fm(M[4], M[4])), fm(M[5], M[5]));
    S.s12 = fa(fa(fm(M[3], M[6]), fm(M[4], M[7])), fm(M[5], M[8]));
    S.s22 = fa(fa(fm(M[6], M[6]), fm(M[7], M[7])), fm(M[8], M[8]));
    return S;
}

// camera depth of a point, in the projection's operation order
__device__ __forceinline__ float cam_depth(const gavis_camera &cam, float x, float y, float z)
{
    const float *R = cam.R, *t = cam.t;
    return fa(fa(fa(fm(R[6], x), fm(R[7], y)), fm(R[8], z)), t[2]);
}

struct Proj {
    float z, u, v, A, B, C, ex, ey;
    int x0, x1, y0, y1;
    int status;   // 0 culled, 1 has tiles, 2 valid but off-screen
};

__device__ __forceinline__ Proj project_one(const gavis_camera &cam, float x, float y, float z, const Sigma3 &S,
                                            float q_cut, float rb, int TW, int TH)
{
    Proj o;
    o.status = 0;
    o.x0 = o.x1 = o.y0 = o.y1 = 0;
    o.u = o.v = o.A = o.B = o.C = o.ex = o.ey = 0.0f;
    const float *R = cam.R, *t = cam.t;
    float tx = fa(fa(fa(fm(R[0], x), fm(R[1], y)), fm(R[2], z)), t[0]);
    float ty = fa(fa(fa(fm(R[3], x), fm(R[4], y)), fm(R[5], z)), t[1]);
    float tz = cam_depth(cam, x, y, z);
    o.z = tz;
    if (!(tz > cam.znear)) return o;
    float limx = fm(1.3f, cam.tan_half_fovx), limy = fm(1.3f, cam.tan_half_fovy);
    float txz = fd(tx, tz), tyz = fd(ty, tz);
    float ctx = fm(fminf(limx, fmaxf(-limx, txz)), tz);
    float cty = fm(fminf(limy, fmaxf(-limy, tyz)), tz);
    float tz2 = fm(tz, tz);
    float J00 = fd(cam.fx, tz), J02 = -fd(fm(cam.fx, ctx), tz2);
    float J11 = fd(cam.fy, tz), J12 = -fd(fm(cam.fy, cty), tz2);
    float T00 = fa(fm(J00, R[0]), fm(J02, R[6])), T01 = fa(fm(J00, R[1]), fm(J02, R[7]));
    float T02 = fa(fm(J00, R[2]), fm(J02, R[8]));
    float T10 = fa(fm(J11, R[3]), fm(J12, R[6])), T11 = fa(fm(J11, R[4]), fm(J12, R[7]));
    float T12 = fa(fm(J11, R[5]), fm(J12, R[8]));
    float U00 = fa(fa(fm(T00, S.s00), fm(T01, S.s01)), fm(T02, S.s02));
    float U01 = fa(fa(fm(T00, S.s01), fm(T01, S.s11)), fm(T02, S.s12));
    float U02 = fa(fa(fm(T00, S.s02), fm(T01, S.s12)), fm(T02, S.s22));
    float U10 = fa(fa(fm(T10, S.s00), fm(T11, S.s01)), fm(T12, S.s02));
    float U11 = fa(fa(fm(T10, S.s01), fm(T11, S.s11)), fm(T12, S.s12));
    float U12 = fa(fa(fm(T10, S.s02), fm(T11, S.s12)), fm(T12, S.s22));
    float a = fa(fa(fa(fm(U00, T00), fm(U01, T01)), fm(U02, T02)), 0.3f);
    float b = fa(fa(fm(U00, T10), fm(U01, T11)), fm(U02, T12));
    float c = fa(fa(fa(fm(U10, T10), fm(U11, T11)), fm(U12, T12)), 0.3f);
    float det = fs(fm(a, c), fm(b, b));
    if (!(det > 0.0f)) return o;
    o.A = fd(c, det);
    o.B = fd(-b, det);
    o.C = fd(a, det);
    o.u = fa(fm(cam.fx, txz), cam.cx);
    o.v = fa(fm(cam.fy, tyz), cam.cy);
    float ex = fa(fm(__fsqrt_rn(fm(q_cut, a)), 1.0009765625f), 0.0009765625f);
    float ey = fa(fm(__fsqrt_rn(fm(q_cut, c)), 1.0009765625f), 0.0009765625f);
    o.ex = ex;
    o.ey = ey;
    float x0 = floorf(fm(fs(fs(o.u, ex), 0.5f), rb)), x1 = floorf(fm(fs(fa(o.u, ex), 0.5f), rb));
    float y0 = floorf(fm(fs(fs(o.v, ey), 0.5f), rb)), y1 = floorf(fm(fs(fa(o.v, ey), 0.5f), rb));
    x0 = fmaxf(x0, 0.0f); y0 = fmaxf(y0, 0.0f);
    x1 = fminf(x1, (float)(TW - 1)); y1 = fminf(y1, (float)(TH - 1));
    if (!(x0 <= x1) || !(y0 <= y1)) { o.status = 2; return o; }
    o.x0 = (int)x0; o.x1 = (int)x1; o.y0 = (int)y0; o.y1 = (int)y1;
    o.status = 1;
    return o;
}

constexpr bool kDealWithAppearance = false;   // see the file header

// A cheap screen test ahead of project_one, conservative by construction:
// it returns false only where project_one returns no tiles.  The centre's
// camera coordinates are computed with project_one's operations (same bits);
// the pixel centre uses an approximate reciprocal, and the footprint
// half-width is bounded from above: the first row of J W is J00 R0 + J02 R2
// with J00 = fx/tz and |J02| <= fx limx / tz (|ctx| <= limx tz), so the
// screen-space variance a <= smax2 (fx/tz)^2 (|R0|^2 + 2 limx |R0.R2| +
// limx^2 |R2|^2) + 0.3 (smax2: the covariance's largest eigenvalue, the
// largest squared scale; any R, orthonormal or not).  kx, ky = those
// factors' square roots times fx, fy with 2% margin, rg = sqrt(q_cut smax2)
// with 1% margin, c0 = sqrt(0.31 q_cut) + 1 pixel; the approximate centre
// adds 1e-5 (|u| + |cx|) of slack.
struct ScreenBound {
    float kx, ky;   // fx, fy times the bound on |J W| rows per unit 1/tz (see may_have_tiles), 2% margin
    float c0;       // sqrt(0.31 q_cut) + 1
    float Wt, Ht;   // extent of the tile grid in pixels
    float pad;
};
static_assert(sizeof(gavis_camera) % 8 == 0, "the bound factors follow the cameras 8-byte aligned");

__device__ __forceinline__ ScreenBound screen_bound(const gavis_camera &c, float q_cut, int TW, int TH, int tile)
{
    const float lx = 1.3f * c.tan_half_fovx, ly = 1.3f * c.tan_half_fovy;
    const float *R = c.R;
    const float n0 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2], n1 = R[3] * R[3] + R[4] * R[4] + R[5] * R[5];
    const float n2 = R[6] * R[6] + R[7] * R[7] + R[8] * R[8];
    const float d02 = fabsf(R[0] * R[6] + R[1] * R[7] + R[2] * R[8]), d12 = fabsf(R[3] * R[6] + R[4] * R[7] + R[5] * R[8]);
    ScreenBound b;
    b.kx = c.fx * sqrtf(n0 + 2.0f * lx * d02 + lx * lx * n2) * 1.02f;
    b.ky = c.fy * sqrtf(n1 + 2.0f * ly * d12 + ly * ly * n2) * 1.02f;
    b.c0 = sqrtf(0.31f * q_cut) + 1.0f;
    b.Wt = (float)(TW * tile);
    b.Ht = (float)(TH * tile);
    b.pad = 0.0f;
    return b;
}

__device__ __forceinline__ bool may_have_tiles(const gavis_camera &cam, const ScreenBound &sb, float x, float y,
                                               float z, float rg)
{
    const float tz = cam_depth(cam, x, y, z);
    if (!(tz > cam.znear)) return false;
    const float *R = cam.R, *t = cam.t;
    const float tx = fa(fa(fa(fm(R[0], x), fm(R[1], y)), fm(R[2], z)), t[0]);
    const float ty = fa(fa(fa(fm(R[3], x), fm(R[4], y)), fm(R[5], z)), t[1]);
    const float iz = __fdividef(1.0f, tz);
    const float u = fmaf(cam.fx, tx * iz, cam.cx), v = fmaf(cam.fy, ty * iz, cam.cy);
    const float ex = fmaf(rg * sb.kx, iz, sb.c0) + (fabsf(u) + fabsf(cam.cx)) * 1e-5f;
    const float ey = fmaf(rg * sb.ky, iz, sb.c0) + (fabsf(v) + fabsf(cam.cy)) * 1e-5f;
    return u + ex > 0.5f && u - ex - 0.5f < sb.Wt && v + ey > 0.5f && v - ey - 0.5f < sb.Ht;
}

// VAR: per-Gaussian colour covariance from coefficient variances
// Geometry-only launches fit six CTAs per SM (80 registers); the appearance
// launches keep 64 coefficient registers per lane and fit four.
template <int LC, int LV, bool UA, bool VAR>
__global__ void __launch_bounds__(128, UA ? 4 : 6) k_project(ProjectArgs a)
{
    extern __shared__ gavis_camera s_cams[];   // nv cameras, then their screen-bound factors
    ScreenBound *s_sb = reinterpret_cast<ScreenBound *>(s_cams + a.nv);
    __shared__ uint32_t s_vis[4][32];   // per warp: visibility bits of each lane's Gaussian in the group's views
    for (int i = threadIdx.x; i < a.nv; i += blockDim.x) {
        s_cams[i] = a.cams[i];
        s_sb[i] = screen_bound(a.cams[i], a.q_cut, a.TW, a.TH, a.tile);
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    s_vis[wib][lane] = 0u;
    __syncthreads();
    // every lane of a warp stays to the end (the warp redistributes its
    // projections over its lanes); a lane past the last Gaussian has none in front
    const int64_t g_raw = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = g_raw < a.n;
    const int64_t g = live ? g_raw : a.n - 1;   // loads stay in bounds; nothing is written for it
    const int64_t gw0 = g_raw - lane;           // the warp's first Gaussian
    const float mx = a.means[3 * g], my = a.means[3 * g + 1], mz = a.means[3 * g + 2];
    const float sc[3] = {a.scales[3 * g], a.scales[3 * g + 1], a.scales[3 * g + 2]};
    const float4 q = reinterpret_cast<const float4 *>(a.rots)[g];
    const float op = a.opac[g];
    // the records carry log2(opacity): the composites take alpha = 2^(log2(o) - q log2(e)/2)
    const float lop = op > 0.0f ? log2f(op) : -INFINITY;
    const Sigma3 S = sigma3d(sc, q.x, q.y, q.z, q.w);
    const float rb = 1.0f / (float)a.tile;
    const float smax2 = fmaxf(fmaxf(sc[0] * sc[0], sc[1] * sc[1]), sc[2] * sc[2]);
    const float rg = sqrtf(a.q_cut * smax2) * 1.01f;

    constexpr int KC = (LC + 1) * (LC + 1);
    constexpr int KV = (LV + 1) * (LV + 1);
    constexpr int KM = KC > KV ? KC : KV;
    constexpr int LM = LC > LV ? LC : LV;
    float th[UA ? KC * 3 : 1];
    float gm[UA ? KV : 1];
    if (UA) {
#pragma unroll
        for (int j = 0; j < KC * 3; ++j) th[j] = ld_coef(a.sh, (size_t)g * KC * 3 + j, a.sh_dtype);
#pragma unroll
        for (int j = 0; j < KV; ++j) gm[j] = a.gamma ? ld_coef(a.gamma, (size_t)g * KV + j, a.vf_dtype) : 0.0f;
    }
    const float P = (float)a.n_train;
    uint32_t zlo = 0xffffffffu, zhi = 0u, nvis = 0u, ntiles = 0u;
    constexpr unsigned am0 = 0xffffffffu;   // every lane of the warp runs every view iteration
    // deal the projections out over the warp's lanes (geometry-only launches;
    // the appearance launches keep 64 coefficient registers per lane live)
    constexpr bool kDeal = !UA || kDealWithAppearance;

    // Views in groups of VG.  The camera depth of each view of the group
    // first.  Then the projections: the warp's (view, Gaussian) pairs with
    // the Gaussian possibly on screen (may_have_tiles) are dealt out to its lanes view
    // by view, 32 per round (a lane takes the owner's centre and covariance
    // by shuffle), so every lane works in every round however unevenly the
    // warp's Gaussians face the cameras, and consecutive lanes write
    // consecutive Gaussians of a view.  Then (with appearance records) the
    // appearance of the views where the Gaussian has tiles, in rounds in
    // which every lane with a pending view takes its next one (the appearance
    // needs the Gaussian's colour and field coefficients, which stay in its
    // own lane's registers).
    constexpr int VG = 32;
    const size_t nw = (size_t)((a.n + 31) >> 5);
    for (int v0 = 0; v0 < a.nv; v0 += VG) {
        const int nu = a.nv - v0 < VG ? a.nv - v0 : VG;
        // views of the group where the Gaussian may have tiles (in front of the
        // near plane and not surely off-screen; the rest are culled)
        uint32_t front = 0u;
        if (live)
            for (int u = 0; u < nu; ++u)
                if (may_have_tiles(s_cams[v0 + u], s_sb[v0 + u], mx, my, mz, rg)) front |= 1u << u;
        if (!a.vis_words && live) {
            for (int u = 0; u < nu; ++u)
                if (a.counts && !((front >> u) & 1u)) a.counts[(size_t)(v0 + u) * (size_t)a.n + (size_t)g] = 0u;
        }
        uint32_t vis = 0u;    // bit u: the lane's Gaussian has tiles in view v0 + u
        uint32_t pend = 0u;   // the same, appearance pending
        if (kDeal) {
            // lane u (< nu) holds the lanes whose Gaussian is in front of view v0 + u
            uint32_t own = 0u;
            for (int u = 0; u < nu; ++u) {
                const unsigned b = __ballot_sync(am0, (front >> u) & 1u);
                if (lane == u) own = b;
            }
            const uint32_t cv = (uint32_t)__popc(own);
            uint32_t iv = cv;   // pairs up to and including view u (scan over the lanes)
    #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(am0, iv, o);
                if (lane >= o) iv += y;
            }
            const uint32_t total = __shfl_sync(am0, iv, 31);
            const uint32_t ev = iv - cv;   // pairs before view u
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t j = base + (uint32_t)lane;
                int u = 0;   // the last view whose pairs start at or before j
    #pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const uint32_t e = __shfl_sync(am0, ev, u + st);
                    if (e <= j) u += st;
                }
                uint32_t ow = __shfl_sync(am0, own, u);
                uint32_t m = j - __shfl_sync(am0, ev, u);   // rank of the pair among view u's
                int o = 0;   // its owner lane: the m-th set bit of ow (halving by the set bits' counts)
    #pragma unroll
                for (int h = 16; h > 0; h >>= 1) {
                    const uint32_t c = (uint32_t)__popc(ow & ((1u << h) - 1u));
                    if (m >= c) {
                        m -= c;
                        o += h;
                        ow >>= h;
                    }
                }
                o &= 31;
                const float gx = __shfl_sync(am0, mx, o), gy = __shfl_sync(am0, my, o), gz = __shfl_sync(am0, mz, o);
                Sigma3 So;
                So.s00 = __shfl_sync(am0, S.s00, o); So.s01 = __shfl_sync(am0, S.s01, o);
                So.s02 = __shfl_sync(am0, S.s02, o); So.s11 = __shfl_sync(am0, S.s11, o);
                So.s12 = __shfl_sync(am0, S.s12, o); So.s22 = __shfl_sync(am0, S.s22, o);
                const float glop = __shfl_sync(am0, lop, o);
                if (j < total) {
                    const int v = v0 + u;
                    const Proj p = project_one(s_cams[v], gx, gy, gz, So, a.q_cut, rb, a.TW, a.TH);
                    const size_t r = (size_t)v * (size_t)a.n + (size_t)(gw0 + o);
                    if (p.status != 1) {
                        if (!a.vis_words && a.counts) a.counts[r] = 0u;
                    } else {
                        atomicOr(&s_vis[wib][o], 1u << u);
                        const uint32_t nt = (uint32_t)((p.x1 - p.x0 + 1) * (p.y1 - p.y0 + 1));
                        if (a.counts) a.counts[r] = nt;
                        ntiles += nt;
                        a.rect[r] = make_uint2((uint32_t)p.x0 | ((uint32_t)p.x1 << 16), (uint32_t)p.y0 | ((uint32_t)p.y1 << 16));
                        zlo = min(zlo, __float_as_uint(p.z));
                        zhi = max(zhi, __float_as_uint(p.z));
                        ++nvis;
                        GeoRec gr;
                        gr.a = make_float4(p.u, p.v, p.A, fa(p.B, p.B));
                        // footprint half-extents, rounded up to half precision (conservative)
                        const uint32_t ext = (uint32_t)__half_as_ushort(__float2half_ru(p.ex)) |
                                             ((uint32_t)__half_as_ushort(__float2half_ru(p.ey)) << 16);
                        gr.b = make_float4(p.C, glop, p.z, __uint_as_float(ext));
                        a.geo[r] = gr;
                        if (a.zrec) a.zrec[r] = p.z;
                    }
                }
            }
            __syncwarp();
            vis = s_vis[wib][lane];
            __syncwarp();
            s_vis[wib][lane] = 0u;   // for the next group
            __syncwarp();
        } else {
            // per-lane rounds: every lane with a pending view takes its next one
            while (__any_sync(am0, front != 0u)) {
                if (front) {
                    const int u = __ffs(front) - 1;
                    front &= front - 1u;
                    const int v = v0 + u;
                    const Proj p = project_one(s_cams[v], mx, my, mz, S, a.q_cut, rb, a.TW, a.TH);
                    const size_t r = (size_t)v * (size_t)a.n + (size_t)g;
                    if (p.status != 1) {
                        if (!a.vis_words && a.counts) a.counts[r] = 0u;
                    } else {
                        vis |= 1u << u;
                        const uint32_t nt = (uint32_t)((p.x1 - p.x0 + 1) * (p.y1 - p.y0 + 1));
                        if (a.counts) a.counts[r] = nt;
                        ntiles += nt;
                        a.rect[r] = make_uint2((uint32_t)p.x0 | ((uint32_t)p.x1 << 16),
                                               (uint32_t)p.y0 | ((uint32_t)p.y1 << 16));
                        zlo = min(zlo, __float_as_uint(p.z));
                        zhi = max(zhi, __float_as_uint(p.z));
                        ++nvis;
                        GeoRec gr;
                        gr.a = make_float4(p.u, p.v, p.A, fa(p.B, p.B));
                        const uint32_t ext = (uint32_t)__half_as_ushort(__float2half_ru(p.ex)) |
                                             ((uint32_t)__half_as_ushort(__float2half_ru(p.ey)) << 16);
                        gr.b = make_float4(p.C, lop, p.z, __uint_as_float(ext));
                        a.geo[r] = gr;
                        if (a.zrec) a.zrec[r] = p.z;
                    }
                }
            }
        }
        if (a.vis_words) {   // one visibility word per warp (32 consecutive Gaussians) and view
            for (int u = 0; u < nu; ++u) {
                const unsigned bal = __ballot_sync(am0, (vis >> u) & 1u);
                if (lane == 0 && gw0 < a.n)   // a warp wholly past the last Gaussian owns no word
                    a.vis_words[(size_t)(v0 + u) * nw + (size_t)(gw0 >> 5)] = bal;
            }
        }
        if (UA) pend = vis;
        if (UA) {
            while (__any_sync(am0, pend != 0u)) {
                if (pend) {
                    const int v = v0 + __ffs(pend) - 1;
                    pend &= pend - 1u;
                    const gavis_camera &cam = s_cams[v];
                    const size_t r = (size_t)v * (size_t)a.n + (size_t)g;
                    float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
                    float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
                    float Y[KM];
                    sh_basis<LM>(dx * rn, dy * rn, dz * rn, Y);
                    float col[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int j = 0; j < KC; ++j) {
                        col[0] = fmaf(th[3 * j], Y[j], col[0]);
                        col[1] = fmaf(th[3 * j + 1], Y[j], col[1]);
                        col[2] = fmaf(th[3 * j + 2], Y[j], col[2]);
                    }
                    float V = 0.0f;
                    if (a.n_train > 0) {
                        float vt = 0.0f;
#pragma unroll
                        for (int j = 0; j < KV; ++j) vt = fmaf(gm[j], Y[j], vt);
                        vt = fminf(fmaxf(vt, 0.0f), P);
                        V = -expm1f(P * log1pf(-vt / P));
                        V = fminf(fmaxf(V, 0.0f), 1.0f);
                    }
                    const float nv1 = 1.0f - V;
                    float kc = 0.0f;   // unused by the constant-covariance composite
                    if (VAR) {
                        // FisherRF variant: Q_k(d) = sum_j Y_j(d)^2 var_jk, diagonal
                        float lq = 0.0f;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            float q = 0.0f;
#pragma unroll
                            for (int j = 0; j < KC; ++j) q = fmaf(Y[j] * Y[j], ld_coef(a.sh_var, ((size_t)g * KC + j) * 3 + k, a.sh_dtype), q);
                            lq += logf(fmaxf(q, 1e-30f));
                        }
                        kc = fmaf(0.5f, lq, 4.256815599614018f);   // + 3/2 log(2 pi e)
                    }
                    UaRec ur;
                    ur.a = make_float4(V + a.beta * nv1, a.o0 * (1.0f - a.beta) * nv1, V, col[0]);
                    ur.b = make_float4(col[1], col[2], kc, 0.0f);
                    a.ua[r] = ur;
                }
            }
        }
    }
    // depth range of the batch, one atomic per warp
    const unsigned am = __activemask();
    const uint32_t wlo = __reduce_min_sync(am, zlo), whi = __reduce_max_sync(am, zhi);
    const uint32_t wvis = __reduce_add_sync(am, nvis);
    const uint32_t wtiles = __reduce_add_sync(am, ntiles);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(am) - 1) && wlo <= whi) {
        atomicMin(&a.zrange[0], wlo);
        atomicMax(&a.zrange[1], whi);
        atomicAdd(a.visible, (unsigned long long)wvis);
        atomicAdd(a.total, (unsigned long long)wtiles);
    }
}

template <int LV>
__global__ void __launch_bounds__(128) k_query(QueryArgs a)
{
    extern __shared__ gavis_camera s_cams[];
    for (int i = threadIdx.x; i < a.nv; i += blockDim.x) s_cams[i] = a.cams[i];
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    constexpr int KV = (LV + 1) * (LV + 1);
    float gm[KV];
#pragma unroll
    for (int j = 0; j < KV; ++j) gm[j] = a.gamma ? ld_coef(a.gamma, (size_t)g * KV + j, a.vf_dtype) : 0.0f;
    const float mx = a.means[3 * g], my = a.means[3 * g + 1], mz = a.means[3 * g + 2];
    const float P = (float)a.n_train;
    for (int v = 0; v < a.nv; ++v) {
        const gavis_camera &cam = s_cams[v];
        float V = 0.0f;
        if (a.n_train > 0) {
            float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
            float rn = rsqrtf(dx * dx + dy * dy + dz * dz);
            float Y[KV];
            sh_basis<LV>(dx * rn, dy * rn, dz * rn, Y);
            float vt = 0.0f;
#pragma unroll
            for (int j = 0; j < KV; ++j) vt = fmaf(gm[j], Y[j], vt);
            vt = fminf(fmaxf(vt, 0.0f), P);
            V = fminf(fmaxf(-expm1f(P * log1pf(-vt / P)), 0.0f), 1.0f);
        }
        a.V[(size_t)v * a.n + g] = V;
    }
}

template <int LC, int LV>
cudaError_t launch_ua(const ProjectArgs &a, cudaStream_t s, int blocks, size_t smem)
{
    if (a.sh_var) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_project<LC, LV, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_project<LC, LV, true, true><<<blocks, 128, smem, s>>>(a);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_project<LC, LV, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_project<LC, LV, true, false><<<blocks, 128, smem, s>>>(a);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_project(const ProjectArgs &a, cudaStream_t s)
{
    if (a.n == 0 || a.nv == 0) return cudaSuccess;
    if (a.nv > kMaxBatchViews) return cudaErrorInvalidValue;
    const int blocks = (int)((a.n + 127) / 128);
    const size_t smem = (sizeof(gavis_camera) + sizeof(ScreenBound)) * (size_t)a.nv;
    if (smem > 48 * 1024) {
        // opt in to larger dynamic shared memory for big batches
        cudaFuncSetAttribute(k_project<0, 0, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (!a.ua) {
        k_project<0, 0, false, false><<<blocks, 128, smem, s>>>(a); count_launch();
        return cudaGetLastError();
    }
#define GAVIS_UA_CASE(LC, LV)                                                                            \
    if (a.sh_degree == LC && a.vf_degree == LV) {                                                        \
        return launch_ua<LC, LV>(a, s, blocks, smem);                                                    \
    }
    GAVIS_UA_CASE(0, 0) GAVIS_UA_CASE(0, 1) GAVIS_UA_CASE(0, 2) GAVIS_UA_CASE(0, 3)
    GAVIS_UA_CASE(1, 0) GAVIS_UA_CASE(1, 1) GAVIS_UA_CASE(1, 2) GAVIS_UA_CASE(1, 3)
    GAVIS_UA_CASE(2, 0) GAVIS_UA_CASE(2, 1) GAVIS_UA_CASE(2, 2) GAVIS_UA_CASE(2, 3)
    GAVIS_UA_CASE(3, 0) GAVIS_UA_CASE(3, 1) GAVIS_UA_CASE(3, 2) GAVIS_UA_CASE(3, 3)
    GAVIS_UA_CASE(0, 4) GAVIS_UA_CASE(1, 4) GAVIS_UA_CASE(2, 4) GAVIS_UA_CASE(3, 4)
    GAVIS_UA_CASE(0, 5) GAVIS_UA_CASE(1, 5) GAVIS_UA_CASE(2, 5) GAVIS_UA_CASE(3, 5)
#undef GAVIS_UA_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_query(const QueryArgs &a, cudaStream_t s)
{
    if (a.n == 0 || a.nv == 0) return cudaSuccess;
    if (a.nv > kMaxBatchViews) return cudaErrorInvalidValue;
    const int blocks = (int)((a.n + 127) / 128);
    const size_t smem = sizeof(gavis_camera) * (size_t)a.nv;
    switch (a.vf_degree) {
#define GAVIS_Q_CASE(L)                                                                                      \
    case L:                                                                                                  \
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_query<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_query<L><<<blocks, 128, smem, s>>>(a); count_launch(); break;
        GAVIS_Q_CASE(0) GAVIS_Q_CASE(1) GAVIS_Q_CASE(2) GAVIS_Q_CASE(3) GAVIS_Q_CASE(4) GAVIS_Q_CASE(5)
#undef GAVIS_Q_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gavis
