// sh_basis.cuh -- real spherical harmonics up to degree 5 as polynomials of a
// unit direction (x, y, z): degrees 0..3 written out, degrees 4 and 5 by the
// recurrences below.
//
// Basis: the paper's real SH (derivation of the vMF coefficients): for m < 0
// sqrt2 (-1)^m Im Y_l^{|m|}, for m = 0 Y_l^0, for m > 0 sqrt2 (-1)^m Re Y_l^m,
// with Y_l^m the complex SH carrying the Condon-Shortley phase.  The (-1)^m
// cancels that phase, which gives the polynomials below, index j = l^2 + l + m.
// Constants: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt2 for m != 0 and
// the integer factor of the associated Legendre polynomial.
#pragma once

namespace gavis {

constexpr int kMaxVfDegree = 5;   // largest visibility-field degree the kernels take

// compile-time constants of the basis (Newton's iteration for the square root)
constexpr double cx_sqrt(double x)
{
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 80; ++i) r = 0.5 * (r + x / r);
    return r;
}
constexpr double cx_fact(int n)
{
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= (double)k;
    return r;
}
// sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), times sqrt2 for m > 0
constexpr double sh_norm(int l, int m)
{
    return cx_sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * cx_fact(l - m) / cx_fact(l + m)) *
           (m > 0 ? cx_sqrt(2.0) : 1.0);
}

// Degrees 4..L.  With Q_l^m(z) = d^m P_l(z) / dz^m (the associated Legendre
// function without the Condon-Shortley phase, divided by sin^m theta) and
// C_m + i S_m = (x + i y)^m = sin^m theta e^{i m phi}:
//   Y_l0 = N_l0 Q_l^0,  Y_l,m = N_lm Q_l^m C_m,  Y_l,-m = N_lm Q_l^m S_m.
// Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) z Q_m^m and
// (l - m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m.
template <int L>
__device__ __forceinline__ void sh_basis_high(float x, float y, float z, float *Y)
{
    float C[L + 1], S[L + 1];
    C[0] = 1.0f;
    S[0] = 0.0f;
#pragma unroll
    for (int m = 1; m <= L; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
    float Q[L + 1][L + 1];
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        float dfact = 1.0f;   // (2m-1)!!
#pragma unroll
        for (int k = 1; k < 2 * m; k += 2) dfact *= (float)k;
        Q[m][m] = dfact;
        if (m + 1 <= L) Q[m + 1][m] = (float)(2 * m + 1) * z * Q[m][m];
#pragma unroll
        for (int l = m + 2; l <= L; ++l)
            Q[l][m] = ((float)(2 * l - 1) * z * Q[l - 1][m] - (float)(l + m - 1) * Q[l - 2][m]) / (float)(l - m);
    }
#pragma unroll
    for (int l = 4; l <= L; ++l) {
        Y[l * l + l] = (float)sh_norm(l, 0) * Q[l][0];
#pragma unroll
        for (int m = 1; m <= l; ++m) {
            const float nq = (float)sh_norm(l, m) * Q[l][m];
            Y[l * l + l + m] = nq * C[m];
            Y[l * l + l - m] = nq * S[m];
        }
    }
}

template <int L>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    static_assert(L >= 0 && L <= kMaxVfDegree, "SH degree out of range");
    Y[0] = 0.28209479177387814f;
    if (L >= 1) {
        Y[1] = 0.4886025119029199f * y;
        Y[2] = 0.4886025119029199f * z;
        Y[3] = 0.4886025119029199f * x;
    }
    if (L >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = 1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
        Y[7] = 1.0925484305920792f * x * z;
        Y[8] = 0.5462742152960396f * (xx - yy);
        if (L >= 3) {
            Y[9] = 0.5900435899266435f * y * (3.0f * xx - yy);
            Y[10] = 2.890611442640554f * x * y * z;
            Y[11] = 0.4570457994644658f * y * (5.0f * zz - 1.0f);
            Y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
            Y[13] = 0.4570457994644658f * x * (5.0f * zz - 1.0f);
            Y[14] = 1.445305721320277f * z * (xx - yy);
            Y[15] = 0.5900435899266435f * x * (xx - 3.0f * yy);
        }
    }
    if (L >= 4) sh_basis_high<L>(x, y, z, Y);
}

}  // namespace gavis
