// blink_div.cuh -- correctly rounded FP64 division by a reused divisor, and
// the grid-cell index of one baseline axis built on it.
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
#include <cstdint>

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

// One axis of the cell assignment: k = round half away from zero of
// t = RN(RN(d / lambda) / delta_u), the paper's FP64 arithmetic (d: antenna
// offset, m); false if the baseline leaves the grid (|k| > N/2 - 1) or t is not
// finite.  Fast path: tf = d * s32 in FP32, s32 = 1 / (lambda delta_u), lies
// within 1.8e-7 |t| of t (three FP32 roundings, two FP64 ones); when tf is
// more than 4e-7 |tf| + 1e-6 away from every half-integer and well inside 2N,
// t rounds to the same integer, so the FP64 quotients (correctly rounded,
// div_by) are computed only for the few baselines near a cell edge.  The FP64
// pipe of this part is narrow: the quotients bound the kernel otherwise.
__host__ __device__ inline bool axis_cell(double d, double lambda, double inv_lambda, double delta_u, double inv_du,
                                          float s32, int n_px, int &k) {
    const float tf = float(d) * s32;
    const float af = fabsf(tf);
    const float whole = truncf(af), fr = af - whole;
    long long r;
    if (af < 2.0f * float(n_px) - 1.0f && fabsf(fr - 0.5f) > fmaf(af, 4e-7f, 1e-6f)) {
        r = (long long)(fr > 0.5f ? whole + 1.0f : whole);
        if (tf < 0.f) r = -r;
    } else {
        const double t = div_by(div_by(d, lambda, inv_lambda), delta_u, inv_du);
        if (!(fabs(t) <= 2.0 * double(n_px))) return false;
        r = std::llround(t);
    }
    const long long kmax = n_px / 2 - 1;
    if (r > kmax || r < -kmax) return false;
    k = int(r);
    return true;
}

}  // namespace blink
