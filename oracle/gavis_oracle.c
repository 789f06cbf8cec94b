/*
 * gavis_oracle.c -- plain CPU oracle for the GAVIS uncertainty-scoring hot
 * path (arxiv 2605.30342).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
 * library that only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load.  It shares no code, header or table with the CUDA library:
 * every formula here is written out again from the paper.
 *
 * Precision: image-space geometry (projection, conic, tile rectangles, the
 * per-pixel footprint value q) is evaluated in float32 with one rounding per
 * operation, in the fixed order written below, so that bins and sort keys can
 * be compared bit for bit.  Everything the method computes from that geometry
 * (spherical harmonics, visibility field, alpha compositing, entropies) is
 * float64.
 *
 * What follows the paper, by function:
 *   oracle_bessel_i      modified spherical Bessel i_l (Sec. "Derivation of
 *                        the vMF coefficients", eq:bl), power series.
 *   oracle_sh_complex    complex SH Y_l^m with the Condon-Shortley phase.
 *   oracle_sh_real       real SH built from the complex ones exactly as the
 *                        paper defines the real basis (same section).
 *   oracle_vf_build      Alg. "Anisotropic Visibility Field Construction"
 *                        with Alg. "Single-view Particle Visibility" per view
 *                        (eq:vis_gamma).
 *   oracle_vf_query      Alg. "Query Anisotropic Visibility Field"
 *                        (eq:vis_sh then the AM-GM bound eq:vis_bound).
 *   oracle_vf_exact      eq:vis_all, the exact multi-view visibility, from
 *                        stored per-view visibilities (for the AM-GM pin).
 *   oracle_render_view   Alg. "3DGS Uncertainty Quantification with
 *                        Visibility Field" (eq:alpha_comp, eq:huber) plus the
 *                        plain 3DGS colour of eq:orig_vr, on untiled
 *                        per-pixel depth-sorted lists; optionally the
 *                        per-pixel expected depth d of eq:id, summed over
 *                        the colour weights alpha_i T_c,i (background 0).
 *   oracle_bins          the (view, tile, depth) keys a tile rasterizer sorts
 *                        by, in canonical order (stable, ties by index).
 *   oracle_composite     one pixel's compositing over a given list (pins).
 *   (colour covariance)  with per-Gaussian coefficient variances, the
 *                        FisherRF variant Q_c,k(d) = sum_j Y_j(d)^2 var_jk
 *                        (Sec. "Integration with FisherRF") replaces the
 *                        constant sigma_c^2 I in eq:huber.
 *   oracle_visibility_view  Alg. "Single-view Particle Visibility" alone.
 *   oracle_density_control  Alg. "Visibility Field Density Control": virtual
 *                        particles, product visibility over views, pruning.
 *
 * Readings of the paper used here (the paper is silent or loose on these):
 *   - the footprint exponent is -q/2 with q = d^T Sigma2D^{-1} d (3DGS), and a
 *     Gaussian overlaps a pixel iff q <= q_cut (default 9), whatever its
 *     opacity;
 *   - the termination test comes after the update, as printed;
 *   - phi(x) = -x ln x with phi(0) = 0;
 *   - the integrated visibility is clamped to [0, |P|] before the bound, and
 *     V = 0 when |P| = 0;
 *   - the view direction of a Gaussian is normalize(x_g - campos);
 *   - the RGB output is the plain 3DGS colour (uncompensated alpha, its own
 *     transmittance), colour = sum_j theta_j Y_j(d) with no offset or clamp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* camera record (24 floats): W H fx fy cx cy tanhx tanhy R[9] t[3] pos[3] zn */
enum { C_W = 0, C_H, C_FX, C_FY, C_CX, C_CY, C_THX, C_THY, C_R = 8, C_T = 17, C_POS = 20, C_ZN = 23, C_LEN = 24 };

/* parameter record (doubles) */
enum { P_KAPPA = 0, P_EPS_T, P_QCUT, P_BETA, P_O0, P_SIGMA_C2, P_LOGDET_Q0, P_TILE, P_MARGIN, P_LEN };

/* ------------------------------------------------------------------------ */
/* special functions                                                        */
/* ------------------------------------------------------------------------ */

/* i_l(x) = x^l sum_k (x^2/2)^k / (k! (2l+2k+1)!!)   (DLMF 10.53.1 form) */
double oracle_bessel_i(int l, double x)
{
    double df = 1.0;                       /* (2l+1)!! */
    for (int k = 1; k <= 2 * l + 1; k += 2) df *= (double)k;
    double term = pow(x, (double)l) / df;  /* k = 0 */
    double sum = term;
    double h = 0.5 * x * x;
    for (int k = 1; k < 400; ++k) {
        term *= h / ((double)k * (double)(2 * l + 2 * k + 1));
        sum += term;
        if (fabs(term) <= 1e-18 * fabs(sum)) break;
    }
    return sum;
}

static double factorial(int n)
{
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= (double)k;
    return r;
}

/* associated Legendre P_l^m(x), m >= 0, with the Condon-Shortley phase */
static double assoc_legendre(int l, int m, double x)
{
    double pmm = 1.0;
    double s = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    for (int k = 1; k <= m; ++k) pmm *= -(double)(2 * k - 1) * s;
    if (l == m) return pmm;
    double pm1 = x * (double)(2 * m + 1) * pmm;
    if (l == m + 1) return pm1;
    double p2 = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        p2 = ((double)(2 * ll - 1) * x * pm1 - (double)(ll + m - 1) * pmm) / (double)(ll - m);
        pmm = pm1;
        pm1 = p2;
    }
    return p2;
}

/* complex Y_l^m(d) for unit d, -l <= m <= l, physics convention */
void oracle_sh_complex(int l, int m, const double *d, double *re, double *im)
{
    double ct = d[2];
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double phi = atan2(d[1], d[0]);
    int am = m < 0 ? -m : m;
    double nrm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
    double p = assoc_legendre(l, am, ct);
    double r = nrm * p * cos(am * phi), i = nrm * p * sin(am * phi);
    if (m < 0) {   /* Y_l^{-m} = (-1)^m conj(Y_l^m) */
        double sg = (am % 2) ? -1.0 : 1.0;
        r = sg * r;
        i = -sg * i;
    }
    *re = r;
    *im = i;
}

/* real SH, index j = l*l + l + m, as the paper defines the real basis:
 *   m < 0: sqrt2 (-1)^m Im Y_l^{|m|};  m = 0: Y_l^0;  m > 0: sqrt2 (-1)^m Re Y_l^m */
void oracle_sh_real(int L, const double *d, double *Y)
{
    for (int l = 0; l <= L; ++l) {
        for (int m = -l; m <= l; ++m) {
            double re, im;
            int am = m < 0 ? -m : m;
            oracle_sh_complex(l, am, d, &re, &im);
            double sg = (am % 2) ? -1.0 : 1.0;
            double y;
            if (m < 0) y = sqrt(2.0) * sg * im;
            else if (m == 0) y = re;
            else y = sqrt(2.0) * sg * re;
            Y[l * l + l + m] = y;
        }
    }
}

/* a_l = 4 pi zeta i_l(kappa), zeta = exp(-kappa)   (eq:vis_gamma) */
static void vmf_coeffs(int L, double kappa, double *a)
{
    double zeta = exp(-kappa);
    for (int l = 0; l <= L; ++l) a[l] = 4.0 * M_PI * zeta * oracle_bessel_i(l, kappa);
}

void oracle_vmf_coeffs(int L, double kappa, double *a) { vmf_coeffs(L, kappa, a); }

/* ------------------------------------------------------------------------ */
/* float32 image-space geometry, one rounding per operation                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    float z, u, v, A, B, C, a, c; /* depth, centre, conic, Sigma2D diagonal */
    float ex, ey;                 /* inflated footprint half-extents */
    int x0, x1, y0, y1;           /* tile rectangle (inclusive) */
    int status;                   /* 0 culled, 1 tiles, 2 valid but no tiles */
} oproj;

static void project_fp32(const float *cam, const float *mean, const float *scale,
                         const float *rot, float qcut, int tile, oproj *o)
{
    const float fx = cam[C_FX], fy = cam[C_FY], cx = cam[C_CX], cy = cam[C_CY];
    const float *R = cam + C_R, *t = cam + C_T;
    const int W = (int)cam[C_W], H = (int)cam[C_H];
    const float x = mean[0], y = mean[1], z = mean[2];
    memset(o, 0, sizeof(*o));

    /* camera space */
    float tx = ((R[0] * x + R[1] * y) + R[2] * z) + t[0];
    float ty = ((R[3] * x + R[4] * y) + R[5] * z) + t[1];
    float tz = ((R[6] * x + R[7] * y) + R[8] * z) + t[2];
    o->z = tz;
    if (!(tz > cam[C_ZN])) { o->status = 0; return; }

    /* rotation of the Gaussian from its (normalised) quaternion w,x,y,z */
    float qw = rot[0], qx = rot[1], qy = rot[2], qz = rot[3];
    float qn = sqrtf(((qw * qw + qx * qx) + qy * qy) + qz * qz);
    qw = qw / qn; qx = qx / qn; qy = qy / qn; qz = qz / qn;
    float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float G[9];
    G[0] = 1.0f - 2.0f * (yy + zz); G[1] = 2.0f * (xy - wz);        G[2] = 2.0f * (xz + wy);
    G[3] = 2.0f * (xy + wz);        G[4] = 1.0f - 2.0f * (xx + zz); G[5] = 2.0f * (yz - wx);
    G[6] = 2.0f * (xz - wy);        G[7] = 2.0f * (yz + wx);        G[8] = 1.0f - 2.0f * (xx + yy);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = G[3 * i + j] * scale[j];
    /* Sigma3D = M M^T (symmetric, 6 entries) */
    float S00 = (M[0] * M[0] + M[1] * M[1]) + M[2] * M[2];
    float S01 = (M[0] * M[3] + M[1] * M[4]) + M[2] * M[5];
    float S02 = (M[0] * M[6] + M[1] * M[7]) + M[2] * M[8];
    float S11 = (M[3] * M[3] + M[4] * M[4]) + M[5] * M[5];
    float S12 = (M[3] * M[6] + M[4] * M[7]) + M[5] * M[8];
    float S22 = (M[6] * M[6] + M[7] * M[7]) + M[8] * M[8];

    /* local affine (EWA) Jacobian with the 1.3 x tan(fov/2) clamp */
    float limx = 1.3f * cam[C_THX], limy = 1.3f * cam[C_THY];
    float txz = tx / tz, tyz = ty / tz;
    float ctx = fminf(limx, fmaxf(-limx, txz)) * tz;
    float cty = fminf(limy, fmaxf(-limy, tyz)) * tz;
    float tz2 = tz * tz;
    float J00 = fx / tz, J02 = -((fx * ctx) / tz2);
    float J11 = fy / tz, J12 = -((fy * cty) / tz2);
    /* T = J Rc */
    float T00 = J00 * R[0] + J02 * R[6], T01 = J00 * R[1] + J02 * R[7], T02 = J00 * R[2] + J02 * R[8];
    float T10 = J11 * R[3] + J12 * R[6], T11 = J11 * R[4] + J12 * R[7], T12 = J11 * R[5] + J12 * R[8];
    /* U = T Sigma3D */
    float U00 = (T00 * S00 + T01 * S01) + T02 * S02;
    float U01 = (T00 * S01 + T01 * S11) + T02 * S12;
    float U02 = (T00 * S02 + T01 * S12) + T02 * S22;
    float U10 = (T10 * S00 + T11 * S01) + T12 * S02;
    float U11 = (T10 * S01 + T11 * S11) + T12 * S12;
    float U12 = (T10 * S02 + T11 * S12) + T12 * S22;
    /* Sigma2D = U T^T + 0.3 I */
    float a = ((U00 * T00 + U01 * T01) + U02 * T02) + 0.3f;
    float b = (U00 * T10 + U01 * T11) + U02 * T12;
    float c = ((U10 * T10 + U11 * T11) + U12 * T12) + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) { o->status = 0; return; }
    o->A = c / det;
    o->B = -b / det;
    o->C = a / det;
    o->a = a;
    o->c = c;
    o->u = fx * txz + cx;
    o->v = fy * tyz + cy;

    /* tile rectangle from inflated footprint half-extents */
    float ex = sqrtf(qcut * a) * 1.0009765625f + 0.0009765625f;
    float ey = sqrtf(qcut * c) * 1.0009765625f + 0.0009765625f;
    o->ex = ex;
    o->ey = ey;
    float rb = 1.0f / (float)tile;  /* tile is a power of two: exact */
    float x0 = floorf(((o->u - ex) - 0.5f) * rb), x1 = floorf(((o->u + ex) - 0.5f) * rb);
    float y0 = floorf(((o->v - ey) - 0.5f) * rb), y1 = floorf(((o->v + ey) - 0.5f) * rb);
    int TW = (W + tile - 1) / tile, TH = (H + tile - 1) / tile;
    x0 = fmaxf(x0, 0.0f); y0 = fmaxf(y0, 0.0f);
    x1 = fminf(x1, (float)(TW - 1)); y1 = fminf(y1, (float)(TH - 1));
    if (!(x0 <= x1) || !(y0 <= y1)) { o->status = 2; return; }
    o->x0 = (int)x0; o->x1 = (int)x1; o->y0 = (int)y0; o->y1 = (int)y1;
    o->status = 1;
}

/* footprint value at pixel (i,j), float32, fixed order */
static float footprint_q(const oproj *p, int i, int j)
{
    float px = (float)i + 0.5f, py = (float)j + 0.5f;
    float dx = px - p->u, dy = py - p->v;
    float B2 = p->B + p->B;
    float qa = p->A * dx;
    float qb = fmaf(B2, dy, qa);
    float qc = p->C * dy;
    float qd = qc * dy;
    return fmaf(qb, dx, qd);
}

static uint32_t fbits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Geometry of every Gaussian in one view.  out: n x 12 floats
 * (z, u, v, A, B, C, x0, x1, y0, y1, ex, ey), status: n ints. */
void oracle_project(int64_t n, const float *cam, const float *means, const float *scales,
                    const float *rots, double qcut, int tile, float *out, int32_t *status)
{
    #pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        oproj p;
        project_fp32(cam, means + 3 * g, scales + 3 * g, rots + 4 * g, (float)qcut, tile, &p);
        float *o = out + 12 * g;
        o[0] = p.z; o[1] = p.u; o[2] = p.v; o[3] = p.A; o[4] = p.B; o[5] = p.C;
        o[6] = (float)p.x0; o[7] = (float)p.x1; o[8] = (float)p.y0; o[9] = (float)p.y1;
        o[10] = p.ex; o[11] = p.ey;
        status[g] = p.status;
    }
}

/* ------------------------------------------------------------------------ */
/* bins: keys (view * tiles + tile) << 32 | depth bits, values = index      */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; uint32_t val; } kv;

static int kv_cmp(const void *pa, const void *pb)
{
    const kv *a = (const kv *)pa, *b = (const kv *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

/* Returns the number of keys M; writes min(M, cap) sorted pairs. */
int64_t oracle_bins(int nview, const float *cams, int64_t n, const float *means, const float *scales,
                    const float *rots, double qcut, int tile, uint64_t *keys, uint32_t *vals, int64_t cap)
{
    int64_t M = 0;
    oproj *P = (oproj *)malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    kv *buf = NULL;
    int64_t bcap = 0;
    for (int v = 0; v < nview; ++v) {
        const float *cam = cams + (size_t)C_LEN * v;
        int W = (int)cam[C_W], H = (int)cam[C_H];
        int TW = (W + tile - 1) / tile, TH = (H + tile - 1) / tile;
        #pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < n; ++g)
            project_fp32(cam, means + 3 * g, scales + 3 * g, rots + 4 * g, (float)qcut, tile, &P[g]);
        for (int64_t g = 0; g < n; ++g) {
            if (P[g].status != 1) continue;
            for (int ty = P[g].y0; ty <= P[g].y1; ++ty)
                for (int tx = P[g].x0; tx <= P[g].x1; ++tx) {
                    if (M >= bcap) {
                        bcap = bcap ? 2 * bcap : 1 << 16;
                        buf = (kv *)realloc(buf, sizeof(kv) * (size_t)bcap);
                    }
                    uint64_t tileid = (uint64_t)v * (uint64_t)(TW * TH) + (uint64_t)(ty * TW + tx);
                    buf[M].key = (tileid << 32) | (uint64_t)fbits(P[g].z);
                    buf[M].val = (uint32_t)g;
                    ++M;
                }
        }
    }
    if (M > 0) qsort(buf, (size_t)M, sizeof(kv), kv_cmp);
    for (int64_t i = 0; i < M && i < cap; ++i) {
        keys[i] = buf[i].key;
        vals[i] = buf[i].val;
    }
    free(buf);
    free(P);
    return M;
}

/* [start, end) of every tile id in sorted keys; ranges: 2 * ntiles, zeroed here */
void oracle_ranges(int64_t M, const uint64_t *keys, int64_t ntiles, uint32_t *ranges)
{
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)ntiles);
    for (int64_t i = 0; i < M; ++i) {
        uint64_t t = keys[i] >> 32;
        if (i == 0 || (keys[i - 1] >> 32) != t) ranges[2 * t] = (uint32_t)i;
        if (i == M - 1 || (keys[i + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* untiled per-pixel lists                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t *start;     /* npix + 1 */
    uint64_t *ent;      /* (depth bits << 32) | index, sorted per pixel */
    float *q;           /* footprint value of each entry */
} plist;

static int u64_cmp(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Pixel range a Gaussian may touch: the exact ellipse box of its (float)
 * conic, in float64, widened by one pixel; the whole image when brute. */
static void pixel_box(const oproj *p, double qcut, int W, int H, int brute, int *i0, int *i1, int *j0, int *j1)
{
    *i0 = 0; *i1 = W - 1; *j0 = 0; *j1 = H - 1;
    if (brute) return;
    double A = p->A, B = p->B, C = p->C;
    double dc = A * C - B * B;
    if (!(dc > 0.0)) return;
    double hx = sqrt(qcut * C / dc) + 1.0, hy = sqrt(qcut * A / dc) + 1.0;
    double lo_i = ceil((double)p->u - hx - 0.5), hi_i = floor((double)p->u + hx - 0.5);
    double lo_j = ceil((double)p->v - hy - 0.5), hi_j = floor((double)p->v + hy - 0.5);
    if (lo_i < 0) lo_i = 0;
    if (lo_j < 0) lo_j = 0;
    if (hi_i > W - 1) hi_i = W - 1;
    if (hi_j > H - 1) hi_j = H - 1;
    *i0 = (int)lo_i; *i1 = (int)hi_i; *j0 = (int)lo_j; *j1 = (int)hi_j;
    if (lo_i > hi_i || lo_j > hi_j) { *i0 = 1; *i1 = 0; }
}

static void build_lists(const float *cam, int64_t n, const oproj *P, double qcut, int brute, plist *L)
{
    int W = (int)cam[C_W], H = (int)cam[C_H];
    int64_t npix = (int64_t)W * H;
    int64_t *cnt = (int64_t *)calloc((size_t)npix + 1, sizeof(int64_t));
    float fq = (float)qcut;
    /* pass 1: count */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < n; ++g) {
        if (P[g].status == 0) continue;
        int i0, i1, j0, j1;
        pixel_box(&P[g], qcut, W, H, brute, &i0, &i1, &j0, &j1);
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i)
                if (footprint_q(&P[g], i, j) <= fq) {
                    #pragma omp atomic
                    cnt[(int64_t)j * W + i] += 1;
                }
    }
    L->start = (int64_t *)malloc(sizeof(int64_t) * ((size_t)npix + 1));
    L->start[0] = 0;
    for (int64_t p = 0; p < npix; ++p) L->start[p + 1] = L->start[p] + cnt[p];
    int64_t tot = L->start[npix];
    L->ent = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(tot > 0 ? tot : 1));
    L->q = NULL;
    memset(cnt, 0, sizeof(int64_t) * (size_t)npix);
    /* pass 2: fill */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < n; ++g) {
        if (P[g].status == 0) continue;
        int i0, i1, j0, j1;
        pixel_box(&P[g], qcut, W, H, brute, &i0, &i1, &j0, &j1);
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i)
                if (footprint_q(&P[g], i, j) <= fq) {
                    int64_t pix = (int64_t)j * W + i, slot;
                    #pragma omp atomic capture
                    slot = cnt[pix]++;
                    L->ent[L->start[pix] + slot] = ((uint64_t)fbits(P[g].z) << 32) | (uint64_t)g;
                }
    }
    free(cnt);
    /* sort each pixel's list by (depth bits, index) */
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        int64_t s = L->start[p], e = L->start[p + 1];
        if (e - s > 1) qsort(L->ent + s, (size_t)(e - s), sizeof(uint64_t), u64_cmp);
    }
}

static void free_lists(plist *L)
{
    free(L->start);
    free(L->ent);
    free(L->q);
}

/* Test hook: pixel list lengths and entries for one view (brute = 1 scans the
 * whole image for every Gaussian). Returns total entries; fills start (npix+1)
 * and up to cap entries. */
int64_t oracle_pixel_lists(const float *cam, int64_t n, const float *means, const float *scales,
                           const float *rots, double qcut, int tile, int brute,
                           int64_t *start, uint64_t *ent, int64_t cap)
{
    oproj *P = (oproj *)malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    for (int64_t g = 0; g < n; ++g)
        project_fp32(cam, means + 3 * g, scales + 3 * g, rots + 4 * g, (float)qcut, tile, &P[g]);
    plist L;
    build_lists(cam, n, P, qcut, brute, &L);
    int64_t npix = (int64_t)cam[C_W] * (int64_t)cam[C_H];
    int64_t tot = L.start[npix];
    memcpy(start, L.start, sizeof(int64_t) * ((size_t)npix + 1));
    for (int64_t i = 0; i < tot && i < cap; ++i) ent[i] = L.ent[i];
    free_lists(&L);
    free(P);
    return tot;
}

/* ------------------------------------------------------------------------ */
/* compositing (float64)                                                    */
/* ------------------------------------------------------------------------ */

static double phi(double x) { return x > 0.0 ? -x * log(x) : 0.0; }

static int near_thresh(double T, double eps, double margin)
{
    return fabs(T - eps) <= margin * eps;
}

/* One pixel of Alg. "3DGS Uncertainty Quantification with Visibility Field"
 * together with the plain colour of eq:orig_vr.
 * in:  n entries with alpha[i] (effective opacity o*exp(-q/2)), V[i], col[3i..],
 *      kc_each[i] (optional) = 1/2 log((2 pi e)^3 |Q_c|) of entry i, else the
 *      constant Q_c = sigma_c2 I_3
 * out: res[0] = H, res[1..3] = rgb, res[4] = T_end, res[5] = Tc_end,
 *      res[6] = sum of w*, res[7] = sum of colour weights, res[8] = w0bar,
 *      res[9] = entries consumed, res[10] = 1 if a transmittance test landed
 *      within margin*eps of eps, res[11] = expected depth.
 *      res[12], res[13]: the least and greatest H, res[14..16], res[17..19]:
 *      the least and greatest rgb, res[20], res[21]: the least and greatest
 *      expected depth over every place where the run could have stopped had
 *      each transmittance test inside [eps(1-margin), eps(1+margin)] gone
 *      either way: each accumulator stops no earlier than its first test
 *      below eps(1+margin) and no later than its first test below
 *      eps(1-margin) (or the end of the list).  A transmittance computed with
 *      a relative error below margin stops inside that range, so these are
 *      bounds on its outputs; where no test falls in the band, lo = hi = the
 *      value above. */
void oracle_composite(int64_t n, const double *alpha, const double *V, const double *col, const double *z,
                      const double *prm, const double *kc_each, double *res)
{
    const double eps = prm[P_EPS_T], beta = prm[P_BETA], o0 = prm[P_O0];
    const double kc_const = 0.5 * 3.0 * log(prm[P_SIGMA_C2]) + 1.5 * (log(2.0 * M_PI) + 1.0);
    const double k0 = 0.5 * prm[P_LOGDET_Q0] + 1.5 * (log(2.0 * M_PI) + 1.0);
    const double margin = prm[P_MARGIN];
    const double band_hi = eps * (1.0 + margin), band_lo = eps * (1.0 - margin);
    double T = 1.0, Tc = 1.0, Hv = 0.0, w0 = 0.0, sw = 0.0, swc = 0.0, D = 0.0;
    double C[3] = {0, 0, 0};
    /* the oracle's own decisions (test after the update, as printed) */
    int ua_on = 1, rgb_on = 1, amb = 0;
    int64_t used = 0;
    double oH = 0.0, oT = 1.0, osw = 0.0, ow0 = 0.0, oC[3] = {0, 0, 0}, oD = 0.0, oTc = 1.0, oswc = 0.0;
    /* bounds: 2 = before the earliest possible stop, 1 = inside the range of
     * possible stops, 0 = past the latest */
    int ua_b = 2, rgb_b = 2;
    double Hlo = 0.0, Hhi = 0.0, Clo[3] = {0, 0, 0}, Chi[3] = {0, 0, 0}, Dlo = 0.0, Dhi = 0.0;
    for (int64_t i = 0; i < n && (ua_b || rgb_b); ++i) {
        double a = alpha[i];
        if (ua_on || rgb_on) used = i + 1;
        if (rgb_b) {
            double w = a * Tc;
            C[0] += w * col[3 * i]; C[1] += w * col[3 * i + 1]; C[2] += w * col[3 * i + 2];
            if (z) D += w * z[i];            /* expected depth, background at 0 */
            swc += w;
            Tc = Tc * (1.0 - a);
            if (rgb_on) {
                if (near_thresh(Tc, eps, margin)) amb = 1;
                if (Tc < eps) {
                    rgb_on = 0;
                    oC[0] = C[0]; oC[1] = C[1]; oC[2] = C[2]; oD = D; oTc = Tc; oswc = swc;
                }
            }
            if (rgb_b == 2 && Tc < band_hi) {
                rgb_b = 1;
                for (int k = 0; k < 3; ++k) Clo[k] = Chi[k] = C[k];
                Dlo = Dhi = D;
            } else if (rgb_b == 1) {
                for (int k = 0; k < 3; ++k) { Clo[k] = fmin(Clo[k], C[k]); Chi[k] = fmax(Chi[k], C[k]); }
                Dlo = fmin(Dlo, D); Dhi = fmax(Dhi, D);
            }
            if (rgb_b == 1 && Tc < band_lo) rgb_b = 0;
        }
        if (ua_b) {
            double v = V[i];
            double as = (v + beta * (1.0 - v)) * a + o0 * (1.0 - beta) * (1.0 - v);  /* eq:alpha_comp */
            double w = as * T;
            double wv = w * v;
            double kc = kc_each ? kc_each[i] : kc_const;   /* 1/2 log((2 pi e)^3 |Q_c|) */
            if (wv > 0.0) Hv += phi(wv) + wv * kc;         /* visible component of eq:huber */
            w0 += w * (1.0 - v);             /* mass of the prior component */
            sw += w;
            T = T * (1.0 - as);
            double Hstop = Hv + (phi(w0) + w0 * k0);   /* H if the run stops here */
            if (ua_on) {
                if (near_thresh(T, eps, margin)) amb = 1;
                if (T < eps) {
                    ua_on = 0;
                    oH = Hstop; oT = T; osw = sw; ow0 = w0;
                }
            }
            if (ua_b == 2 && T < band_hi) {
                ua_b = 1;
                Hlo = Hhi = Hstop;
            } else if (ua_b == 1) {
                Hlo = fmin(Hlo, Hstop); Hhi = fmax(Hhi, Hstop);
            }
            if (ua_b == 1 && T < band_lo) ua_b = 0;
        }
    }
    /* runs still going stop at the end of the list */
    if (rgb_on) { oC[0] = C[0]; oC[1] = C[1]; oC[2] = C[2]; oD = D; oTc = Tc; oswc = swc; }
    if (rgb_b == 2) { for (int k = 0; k < 3; ++k) Clo[k] = Chi[k] = C[k]; Dlo = Dhi = D; }
    {
        double Hend = Hv + (phi(w0) + w0 * k0);   /* invisible component added at the stop */
        if (ua_on) { oH = Hend; oT = T; osw = sw; ow0 = w0; }
        if (ua_b == 2) Hlo = Hhi = Hend;
    }
    res[0] = oH; res[1] = oC[0]; res[2] = oC[1]; res[3] = oC[2];
    res[4] = oT; res[5] = oTc; res[6] = osw; res[7] = oswc; res[8] = ow0;
    res[9] = (double)used; res[10] = (double)amb; res[11] = oD;
    res[12] = Hlo; res[13] = Hhi;
    res[14] = Clo[0]; res[15] = Clo[1]; res[16] = Clo[2];
    res[17] = Chi[0]; res[18] = Chi[1]; res[19] = Chi[2];
    res[20] = Dlo; res[21] = Dhi;
}

/* ------------------------------------------------------------------------ */
/* visibility field query (Alg. Query Anisotropic Visibility Field)         */
/* ------------------------------------------------------------------------ */

static double ipow(double b, int64_t e)
{
    double r = 1.0;
    while (e > 0) {
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
    }
    return r;
}

static void unit_dir(const float *xg, const float *pos, double *d)
{
    double dx = (double)xg[0] - (double)pos[0];
    double dy = (double)xg[1] - (double)pos[1];
    double dz = (double)xg[2] - (double)pos[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r > 0) { d[0] = dx / r; d[1] = dy / r; d[2] = dz / r; }
    else { d[0] = 0; d[1] = 0; d[2] = 1; }
}

/* V[g] for a view at campos: Vt = sum_j gamma_j Y_j(d); V = 1 - (1 - Vt/P)^P.
 * vt_out (optional) receives the unclamped Vt. */
void oracle_vf_query(int64_t n, const double *gamma, int L, int64_t P, const float *campos,
                     const float *means, double *V, double *vt_out)
{
    int K = (L + 1) * (L + 1);
    #pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        double d[3], Y[64];
        unit_dir(means + 3 * g, campos, d);
        oracle_sh_real(L, d, Y);
        double vt = 0.0;
        for (int j = 0; j < K; ++j) vt += gamma[(size_t)g * K + j] * Y[j];
        if (vt_out) vt_out[g] = vt;
        if (P <= 0) { V[g] = 0.0; continue; }
        double c = vt;
        if (c < 0.0) c = 0.0;
        if (c > (double)P) c = (double)P;
        V[g] = 1.0 - ipow(1.0 - c / (double)P, P);
    }
}

/* eq:vis_all: V(d) = 1 - prod_p (1 - v_p nu(d; d_p)), nu = exp(kappa (d.d_p - 1)).
 * vis: nview x n per-view particle visibilities; dirs: nview x n x 3. */
void oracle_vf_exact(int64_t n, int nview, const double *vis, const double *dirs, double kappa,
                     const double *d, double *V)
{
    for (int64_t g = 0; g < n; ++g) {
        double pr = 1.0;
        for (int p = 0; p < nview; ++p) {
            const double *dp = dirs + ((size_t)p * n + g) * 3;
            double nu = exp(kappa * (d[3 * g] * dp[0] + d[3 * g + 1] * dp[1] + d[3 * g + 2] * dp[2] - 1.0));
            pr *= 1.0 - vis[(size_t)p * n + g] * nu;
        }
        V[g] = 1.0 - pr;
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. Single-view Particle Visibility                                      */
/* ------------------------------------------------------------------------ */

/* sumT, cnt: per Gaussian (float64, int64), overwritten.  amb (optional):
 * set to 1 for Gaussians that follow a near-threshold transmittance test in
 * some pixel's list (their inclusion depends on rounding).
 * bnd (optional): per Gaussian, the sums a run could take when each test
 * inside [eps(1-margin), eps(1+margin)] may go either way: every pixel stops
 * no earlier than its first test below eps(1+margin) and no later than its
 * first test below eps(1-margin).  sum_early / cnt_early: T summed and
 * entries counted up to the earliest stops; cnt_late: entries counted up to
 * the latest stops.  The entries between the two stops (cnt_late -
 * cnt_early of them) each carry a transmittance in
 * [eps(1-margin), eps(1+margin)].  Returns pairs. */
typedef struct { double *sum_early; int64_t *cnt_early, *cnt_late; } vis_bounds;

int64_t oracle_visibility_view_b(const float *cam, int64_t n, const float *means, const float *scales,
                                 const float *rots, const float *opac, const double *prm,
                                 double *sumT, int64_t *cnt, uint8_t *amb, const vis_bounds *bnd)
{
    const double eps = prm[P_EPS_T], qcut = prm[P_QCUT], margin = prm[P_MARGIN];
    const double band_hi = eps * (1.0 + margin), band_lo = eps * (1.0 - margin);
    const int tile = (int)prm[P_TILE];
    oproj *P = (oproj *)malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    #pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g)
        project_fp32(cam, means + 3 * g, scales + 3 * g, rots + 4 * g, (float)qcut, tile, &P[g]);
    plist Lst;
    build_lists(cam, n, P, qcut, 0, &Lst);
    memset(sumT, 0, sizeof(double) * (size_t)n);
    memset(cnt, 0, sizeof(int64_t) * (size_t)n);
    if (bnd) {
        memset(bnd->sum_early, 0, sizeof(double) * (size_t)n);
        memset(bnd->cnt_early, 0, sizeof(int64_t) * (size_t)n);
        memset(bnd->cnt_late, 0, sizeof(int64_t) * (size_t)n);
    }
    int W = (int)cam[C_W], H = (int)cam[C_H];
    int64_t npix = (int64_t)W * H, pairs = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(+ : pairs)
    for (int64_t p = 0; p < npix; ++p) {
        int i = (int)(p % W), j = (int)(p / W);
        double T = 1.0;
        int on = 1, early = 1;       /* the oracle's own run; before the earliest stop */
        int64_t s = Lst.start[p], e = Lst.start[p + 1];
        for (int64_t k = s; k < e; ++k) {
            uint32_t g = (uint32_t)(Lst.ent[k] & 0xffffffffu);
            double q = (double)footprint_q(&P[g], i, j);
            double a = (double)opac[g] * exp(-0.5 * q);
            if (on) {
                #pragma omp atomic
                sumT[g] += T;
                #pragma omp atomic
                cnt[g] += 1;
                ++pairs;
            }
            if (bnd) {
                if (early) {
                    #pragma omp atomic
                    bnd->sum_early[g] += T;
                    #pragma omp atomic
                    bnd->cnt_early[g] += 1;
                }
                #pragma omp atomic
                bnd->cnt_late[g] += 1;
            }
            T = T * (1.0 - a);
            if (on && amb && near_thresh(T, eps, margin)) {
                for (int64_t r = k + 1; r < e; ++r) amb[(uint32_t)(Lst.ent[r] & 0xffffffffu)] = 1;
            }
            if (T < eps) on = 0;
            if (T < band_hi) early = 0;
            if (!bnd && !on) break;
            if (T < band_lo) break;
        }
    }
    free_lists(&Lst);
    free(P);
    return pairs;
}

int64_t oracle_visibility_view(const float *cam, int64_t n, const float *means, const float *scales,
                               const float *rots, const float *opac, const double *prm,
                               double *sumT, int64_t *cnt, uint8_t *amb, double *sum_early,
                               int64_t *cnt_early, int64_t *cnt_late)
{
    vis_bounds b = {sum_early, cnt_early, cnt_late};
    return oracle_visibility_view_b(cam, n, means, scales, rots, opac, prm, sumT, cnt, amb,
                                    sum_early ? &b : NULL);
}

/* Range [v_lo, v_hi] of v = sumT / cnt over the runs vis_bounds allows, for
 * one Gaussian: k of its late entries beyond the early ones (0 <= k <= K)
 * each add a transmittance t; the other pass's own float32 transmittance may
 * differ by a further factor (1 +- margin), so t lies in
 * [eps (1-margin)^2, eps (1+margin)^2].  (S + k t) / (C + k) is monotone in k
 * and in t, so its extremes sit at k in {0, K} and the ends of t's range. */
static void visibility_range(double S, int64_t C, int64_t Cl, double eps, double margin, double *vlo, double *vhi)
{
    const double tlo = eps * (1.0 - margin) * (1.0 - margin), thi = eps * (1.0 + margin) * (1.0 + margin);
    const int64_t K = Cl - C;
    const double v0 = C > 0 ? S / (double)C : 0.0;
    *vlo = *vhi = v0;
    if (K > 0) {
        double a = (S + (double)K * tlo) / (double)(C + K), b = (S + (double)K * thi) / (double)(C + K);
        *vlo = fmin(v0, a);
        *vhi = fmax(v0, b);
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. Anisotropic Visibility Field Construction                           */
/* ------------------------------------------------------------------------ */

/* gamma: n x (L+1)^2 float64, overwritten.  vis_out (optional): nview x n
 * per-view visibilities v_p[g].  amb (optional, n): union over views.
 * gamma_rad (optional, n x (L+1)^2): sum over views of
 * r_p |a_l Y_j(d_p)|, where r_p is the largest distance from v_p to the ends
 * of its range under rounding-sensitive terminations (visibility_range):
 * a bound on how far a field built with such terminations can lie from
 * gamma, coefficient by coefficient. */
void oracle_vf_build(int nview, const float *cams, int64_t n, const float *means, const float *scales,
                     const float *rots, const float *opac, int L, const double *prm,
                     double *gamma, double *vis_out, uint8_t *amb, double *gamma_rad)
{
    int K = (L + 1) * (L + 1);
    double a[64];
    vmf_coeffs(L, prm[P_KAPPA], a);
    memset(gamma, 0, sizeof(double) * (size_t)n * K);
    if (gamma_rad) memset(gamma_rad, 0, sizeof(double) * (size_t)n * K);
    if (amb) memset(amb, 0, (size_t)n);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    double *sumT = (double *)malloc(sizeof(double) * nn);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * nn);
    vis_bounds b = {NULL, NULL, NULL};
    if (gamma_rad) {
        b.sum_early = (double *)malloc(sizeof(double) * nn);
        b.cnt_early = (int64_t *)malloc(sizeof(int64_t) * nn);
        b.cnt_late = (int64_t *)malloc(sizeof(int64_t) * nn);
    }
    for (int p = 0; p < nview; ++p) {
        const float *cam = cams + (size_t)C_LEN * p;
        oracle_visibility_view_b(cam, n, means, scales, rots, opac, prm, sumT, cnt, amb, gamma_rad ? &b : NULL);
        #pragma omp parallel for schedule(static)
        for (int64_t g = 0; g < n; ++g) {
            double v = cnt[g] > 0 ? sumT[g] / (double)cnt[g] : 0.0;
            if (vis_out) vis_out[(size_t)p * n + g] = v;
            double r = 0.0;
            if (gamma_rad) {
                double vlo, vhi;
                visibility_range(b.sum_early[g], b.cnt_early[g], b.cnt_late[g], prm[P_EPS_T], prm[P_MARGIN], &vlo, &vhi);
                r = fmax(vhi - v, v - vlo);
            }
            if (v == 0.0 && r == 0.0) continue;
            double d[3], Y[64];
            unit_dir(means + 3 * g, cam + C_POS, d);
            oracle_sh_real(L, d, Y);
            for (int l = 0; l <= L; ++l)
                for (int m = -l; m <= l; ++m) {
                    int j = l * l + l + m;
                    gamma[(size_t)g * K + j] += v * a[l] * Y[j];
                    if (gamma_rad) gamma_rad[(size_t)g * K + j] += r * fabs(a[l] * Y[j]);
                }
        }
    }
    free(sumT);
    free(cnt);
    free(b.sum_early);
    free(b.cnt_early);
    free(b.cnt_late);
}

/* ------------------------------------------------------------------------ */
/* one candidate view: VF query + UQ rasterization + colour                 */
/* ------------------------------------------------------------------------ */

/* rgb: 3 x H x W planar; unc: H x W; amb: H x W (0/1); used: H x W entries
 * consumed.  V: per-Gaussian visibility for this view (from oracle_vf_query).
 * sh: n x (Lc+1)^2 x 3 colour coefficients.  bounds (optional): 10 planes of
 * H x W, the least and greatest value each output can take when the
 * transmittance tests near eps_T go either way (see oracle_composite):
 * unc_lo, unc_hi, r_lo, g_lo, b_lo, r_hi, g_hi, b_hi, depth_lo, depth_hi. */
void oracle_render_view(const float *cam, int64_t n, const float *means, const float *scales,
                        const float *rots, const float *opac, const double *sh, const double *sh_var, int Lc,
                        const double *V, const double *prm, double *rgb, double *unc, double *depth,
                        uint8_t *amb, int32_t *used, double *bounds)
{
    const double qcut = prm[P_QCUT];
    const int tile = (int)prm[P_TILE];
    const int Kc = (Lc + 1) * (Lc + 1);
    oproj *P = (oproj *)malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    double *col = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *kcg = sh_var ? (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1)) : NULL;
    #pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        project_fp32(cam, means + 3 * g, scales + 3 * g, rots + 4 * g, (float)qcut, tile, &P[g]);
        double d[3], Y[64];
        unit_dir(means + 3 * g, cam + C_POS, d);
        oracle_sh_real(Lc, d, Y);
        for (int k = 0; k < 3; ++k) {
            double c = 0.0;
            for (int j = 0; j < Kc; ++j) c += sh[((size_t)g * Kc + j) * 3 + k] * Y[j];   /* eq:rgb_sh */
            col[3 * g + k] = c;
        }
        if (kcg) {
            /* FisherRF variant: Q_c,k(d) = sum_j Y_j(d)^2 var_jk (diagonal) */
            double lq = 0.0;
            for (int k = 0; k < 3; ++k) {
                double q = 0.0;
                for (int j = 0; j < Kc; ++j) q += Y[j] * Y[j] * sh_var[((size_t)g * Kc + j) * 3 + k];
                lq += log(q);
            }
            kcg[g] = 0.5 * lq + 1.5 * (log(2.0 * M_PI) + 1.0);
        }
    }
    plist Lst;
    build_lists(cam, n, P, qcut, 0, &Lst);
    int W = (int)cam[C_W], H = (int)cam[C_H];
    int64_t npix = (int64_t)W * H;
    #pragma omp parallel
    {
        int64_t capn = 0;
        double *al = NULL, *vv = NULL, *cc = NULL, *kk = NULL, *zz = NULL;
        #pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < npix; ++p) {
            int i = (int)(p % W), j = (int)(p / W);
            int64_t s = Lst.start[p], e = Lst.start[p + 1], m = e - s;
            if (m > capn) {
                capn = m * 2;
                al = (double *)realloc(al, sizeof(double) * (size_t)capn);
                vv = (double *)realloc(vv, sizeof(double) * (size_t)capn);
                cc = (double *)realloc(cc, sizeof(double) * 3 * (size_t)capn);
                kk = (double *)realloc(kk, sizeof(double) * (size_t)capn);
                zz = (double *)realloc(zz, sizeof(double) * (size_t)capn);
            }
            for (int64_t k = 0; k < m; ++k) {
                uint32_t g = (uint32_t)(Lst.ent[s + k] & 0xffffffffu);
                double q = (double)footprint_q(&P[g], i, j);
                al[k] = (double)opac[g] * exp(-0.5 * q);
                vv[k] = V[g];
                cc[3 * k] = col[3 * g]; cc[3 * k + 1] = col[3 * g + 1]; cc[3 * k + 2] = col[3 * g + 2];
                if (kcg) kk[k] = kcg[g];
                zz[k] = (double)P[g].z;
            }
            double res[24];
            oracle_composite(m, al, vv, cc, zz, prm, kcg ? kk : NULL, res);
            if (bounds) {
                bounds[p] = res[12];
                bounds[npix + p] = res[13];
                for (int k = 0; k < 6; ++k) bounds[(2 + k) * npix + p] = res[14 + k];
                bounds[8 * npix + p] = res[20];
                bounds[9 * npix + p] = res[21];
            }
            unc[p] = res[0];
            rgb[p] = res[1];
            rgb[npix + p] = res[2];
            rgb[2 * npix + p] = res[3];
            if (depth) depth[p] = res[11];
            if (amb) amb[p] = (uint8_t)res[10];
            if (used) used[p] = (int32_t)res[9];
        }
        free(al); free(vv); free(cc); free(kk); free(zz);
    }
    free_lists(&Lst);
    free(col);
    free(kcg);
    free(P);
}

/* ------------------------------------------------------------------------ */
/* Alg. Visibility Field Density Control                                    */
/* ------------------------------------------------------------------------ */

/* Virtual particles: centres x_j (caller-drawn, uniform in the scene),
 * identity rotation, isotropic scale s with (4/3) pi s^3 rho = 1 + eta,
 * opacity 0.  Their multi-view visibility 1 - prod_p (1 - v_p[j]) is
 * computed with Alg. Single-view Particle Visibility on the union of the
 * scene and the virtual particles; a particle is kept (under-explored) iff
 * that visibility is <= eps_v.
 *   vis_out: n_virt (float64); keep: n_virt (0/1); amb (optional): n_virt,
 *   set when a rounding-sensitive transmittance test touched the particle;
 *   vis_lo, vis_hi (optional): n_virt, the range of the multi-view
 *   visibility when those tests go either way (per-view ranges from
 *   visibility_range; 1 - prod(1 - v) is increasing in every v).
 * Returns the number kept. */
int64_t oracle_density_control(int nview, const float *cams, int64_t n, const float *means, const float *scales,
                               const float *rots, const float *opac, int64_t n_virt, const float *vmeans,
                               double rho, double eta, double eps_v, const double *prm, double *vis_out,
                               uint8_t *keep, uint8_t *amb, double *vis_lo, double *vis_hi)
{
    const int64_t na = n + n_virt;
    const double s = cbrt(3.0 * (1.0 + eta) / (4.0 * M_PI * rho));
    float *am = (float *)malloc(sizeof(float) * 3 * (size_t)(na > 0 ? na : 1));
    float *as = (float *)malloc(sizeof(float) * 3 * (size_t)(na > 0 ? na : 1));
    float *ar = (float *)malloc(sizeof(float) * 4 * (size_t)(na > 0 ? na : 1));
    float *ao = (float *)malloc(sizeof(float) * (size_t)(na > 0 ? na : 1));
    memcpy(am, means, sizeof(float) * 3 * (size_t)n);
    memcpy(as, scales, sizeof(float) * 3 * (size_t)n);
    memcpy(ar, rots, sizeof(float) * 4 * (size_t)n);
    memcpy(ao, opac, sizeof(float) * (size_t)n);
    for (int64_t j = 0; j < n_virt; ++j) {
        for (int k = 0; k < 3; ++k) {
            am[3 * (n + j) + k] = vmeans[3 * j + k];
            as[3 * (n + j) + k] = (float)s;
        }
        ar[4 * (n + j)] = 1.0f;
        ar[4 * (n + j) + 1] = ar[4 * (n + j) + 2] = ar[4 * (n + j) + 3] = 0.0f;
        ao[n + j] = 0.0f;
    }
    const size_t nv1 = (size_t)(n_virt > 0 ? n_virt : 1), na1 = (size_t)(na > 0 ? na : 1);
    double *prod = (double *)malloc(sizeof(double) * nv1);
    double *plo = (double *)malloc(sizeof(double) * nv1);   /* product with every v at its low end */
    double *phi_ = (double *)malloc(sizeof(double) * nv1);  /* ... at its high end */
    for (int64_t j = 0; j < n_virt; ++j) prod[j] = plo[j] = phi_[j] = 1.0;
    double *sumT = (double *)malloc(sizeof(double) * na1);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * na1);
    uint8_t *ab = (uint8_t *)calloc(na1, 1);
    vis_bounds b = {(double *)malloc(sizeof(double) * na1), (int64_t *)malloc(sizeof(int64_t) * na1),
                    (int64_t *)malloc(sizeof(int64_t) * na1)};
    for (int p = 0; p < nview; ++p) {
        oracle_visibility_view_b(cams + (size_t)C_LEN * p, na, am, as, ar, ao, prm, sumT, cnt, ab, &b);
        for (int64_t j = 0; j < n_virt; ++j) {
            double v = cnt[n + j] > 0 ? sumT[n + j] / (double)cnt[n + j] : 0.0;
            double vlo, vhi;
            visibility_range(b.sum_early[n + j], b.cnt_early[n + j], b.cnt_late[n + j], prm[P_EPS_T],
                             prm[P_MARGIN], &vlo, &vhi);
            prod[j] *= 1.0 - v;
            plo[j] *= 1.0 - vlo;
            phi_[j] *= 1.0 - vhi;
        }
    }
    int64_t kept = 0;
    for (int64_t j = 0; j < n_virt; ++j) {
        double vt = 1.0 - prod[j];
        if (vis_out) vis_out[j] = vt;
        if (vis_lo) vis_lo[j] = 1.0 - plo[j];
        if (vis_hi) vis_hi[j] = 1.0 - phi_[j];
        keep[j] = (uint8_t)(vt <= eps_v);
        kept += keep[j];
        if (amb) amb[j] = ab[n + j];
    }
    free(am); free(as); free(ar); free(ao); free(prod); free(plo); free(phi_); free(sumT); free(cnt); free(ab);
    free(b.sum_early); free(b.cnt_early); free(b.cnt_late);
    return kept;
}
