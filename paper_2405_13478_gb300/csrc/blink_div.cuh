// blink_div.cuh -- correctly rounded FP64 division by a reused divisor.
//
// The cell assignment divides every baseline component by the channel's
// wavelength and cell size (Sec. 5.2.1); with the divisor's correctly rounded
// reciprocal y = RN(1/b) computed once, a / b takes one multiply and four
// fused multiply-adds instead of a full division each time.
//
// Method (P. Markstein, "Computation of elementary functions on the IBM RISC
// System/6000 processor", IBM J. Res. Develop. 34(1), 1990): q0 = RN(a y) is
// within two ulps of a/b; the residual r0 = a - b q0 is exact in an FMA and
// q1 = RN(q0 + r0 y) is within one ulp; by Markstein's theorem (y within half
// an ulp of 1/b, q1 within one ulp of a/b) RN(q1 + (a - b q1) y) is the
// correctly rounded quotient RN(a/b), bit-identical to IEEE division.  The
// theorem needs every intermediate in the normal range: outside
// 2^-900 < |a| < 2^900 (and a = 0) the plain division is used.
#pragma once

#include <cmath>

namespace blink {

__host__ __device__ inline double div_by(double a, double b, double y) {
    const double m = fabs(a);
    if (!(m > 0x1p-900 && m < 0x1p900)) return a / b;
    const double q0 = a * y;
    const double r0 = fma(-q0, b, a);
    const double q1 = fma(r0, y, q0);
    const double r1 = fma(-q1, b, a);
    return fma(r1, y, q1);
}

}  // namespace blink
