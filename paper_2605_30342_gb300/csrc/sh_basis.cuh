// sh_basis.cuh -- real spherical harmonics up to degree 3 as polynomials of a
// unit direction (x, y, z).
//
// Basis: the paper's real SH (derivation of the vMF coefficients): for m < 0
// sqrt2 (-1)^m Im Y_l^{|m|}, for m = 0 Y_l^0, for m > 0 sqrt2 (-1)^m Re Y_l^m,
// with Y_l^m the complex SH carrying the Condon-Shortley phase.  The (-1)^m
// cancels that phase, which gives the polynomials below, index j = l^2 + l + m.
// Constants: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt2 for m != 0 and
// the integer factor of the associated Legendre polynomial.
#pragma once

namespace gavis {

template <int L>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
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
}

}  // namespace gavis
