// blink_fft.cuh -- in-register DFT codelets and four-step size plans.
//
// The inverse 2-D transform of the imager (Sec. 5.2.2) is done as two batches of
// 1-D transforms.  A 1-D transform of length N = N1 * N2 is split four-step
// (Cooley-Tukey with one twiddle stage): N2 transforms of length N1 along
// stride N2, a twiddle multiply by W_N^(n2 k1), then N1 transforms of length
// N2 on contiguous runs.  Each short transform (N1, N2 <= 32) runs entirely in
// one thread's registers; shared memory only carries the exchange between the
// two steps.
//
// Roots of unity are computed at compile time from their Taylor series after
// an exact integer reduction of the angle to the first octant, so the short
// transforms get their twiddles as immediate operands.  The four-step
// twiddles, whose exponent depends on the lane, come from a transposed table
// in global memory (FourStepTable), read with coalesced loads or staged in
// shared memory: lanes reading distinct constant-memory addresses would be
// serialised.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace blink {

struct c32 {
    float x, y;
};
struct c64d {
    double x, y;
};

// ------------------------------------------------------- compile-time roots
constexpr double kHalfPi = 1.57079632679489661923132169163975144;

constexpr double taylor_sin(double a) {
    double a2 = a * a, term = a, sum = a;
    for (int i = 1; i < 14; ++i) {
        term *= -a2 / double((2 * i) * (2 * i + 1));
        sum += term;
    }
    return sum;
}
constexpr double taylor_cos(double a) {
    double a2 = a * a, term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) {
        term *= -a2 / double((2 * i - 1) * (2 * i));
        sum += term;
    }
    return sum;
}

// exp(+2 pi i k / n) for integers k, n > 0.
constexpr c64d unit_root(long long k, long long n) {
    k %= n;
    if (k < 0) k += n;
    const long long q = (4 * k) / n;      // quadrant 0..3
    const long long r = 4 * k - q * n;    // angle within quadrant = (pi/2) r / n
    double c = 0.0, s = 0.0;
    if (2 * r <= n) {
        const double a = kHalfPi * double(r) / double(n);
        c = taylor_cos(a);
        s = taylor_sin(a);
    } else {
        const double a = kHalfPi * double(n - r) / double(n);
        c = taylor_sin(a);
        s = taylor_cos(a);
    }
    switch (q) {
        case 0: return c64d{c, s};
        case 1: return c64d{-s, c};
        case 2: return c64d{-c, -s};
        default: return c64d{s, -c};
    }
}

// ----------------------------------------------------------- complex helpers
// Complex sums as paired FP32 adds on the GPU: one instruction for both
// components, each rounded like a scalar add (the butterflies are most of the
// transforms' FP32 instructions, and the large transforms are issue-bound).
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, c32 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by S*i
template <int S>
__host__ __device__ __forceinline__ float2 mul_si(float2 a) {
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// --------------------------------------------------------- in-register DFTs
// Compile-time loop: f(std::integral_constant<int, i>) for i in [B, E).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// z * W_N^(S e) with e a compile-time exponent: the root is an immediate.
template <int N, int S, int E>
__host__ __device__ __forceinline__ float2 twiddle(float2 z) {
    constexpr int e = ((E % N) + N) % N;
    if constexpr (e == 0) {
        return z;
    } else if constexpr (4 * e == N) {
        return mul_si<S>(z);
    } else if constexpr (2 * e == N) {
        return make_float2(-z.x, -z.y);
    } else if constexpr (4 * e == 3 * N) {
        return mul_si<-S>(z);
    } else {
        constexpr c64d w = unit_root(e, N);
        constexpr float wx = float(w.x), wy = float(S * w.y);
        return make_float2(fmaf(z.x, wx, -z.y * wy), fmaf(z.x, wy, z.y * wx));
    }
}

// X[k] = sum_j x[j] W_N^(S j k), in place, natural order in and out.
template <int N>
constexpr int first_radix() {
    return (N % 4 == 0) ? 4 : (N % 2 == 0) ? 2 : (N % 3 == 0) ? 3 : (N % 5 == 0) ? 5 : N;
}

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// Largest factor A of N with gcd(A, N / A) == 1 and 1 < A < N (0 if none):
// such N take the prime-factor (Good-Thomas) split, which needs no twiddles.
template <int N>
constexpr int coprime_factor() {
    int best = 0;
    for (int a = 2; a < N; ++a)
        if (N % a == 0 && gcd_c(a, N / a) == 1) best = a;
    return best;
}

// (a^-1) mod m for gcd(a, m) == 1, m >= 1.
constexpr int inv_mod(int a, int m) {
    for (int x = 0; x < m; ++x)
        if ((a % m) * x % m == 1 % m) return x;
    return 0;
}

template <int N, int S>
__host__ __device__ __forceinline__ void dft(float2 (&x)[N]);

template <int S>
__host__ __device__ __forceinline__ void bfly2(float2 &a, float2 &b) {
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int S>
__host__ __device__ __forceinline__ void bfly3(float2 (&x)[3]) {
    constexpr float h = 0.866025403784438646763723170752936f;  // sin(2 pi / 3) = sqrt(3)/2
    const float2 t1 = cadd(x[1], x[2]);
    const float2 t2 = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
    const float2 d = csub(x[1], x[2]);
    const float2 t3 = mul_si<S>(make_float2(h * d.x, h * d.y));
    x[0] = cadd(x[0], t1);
    x[1] = cadd(t2, t3);
    x[2] = csub(t2, t3);
}

template <int S>
__host__ __device__ __forceinline__ void bfly4(float2 (&x)[4]) {
    const float2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    const float2 s13 = cadd(x[1], x[3]), d13 = mul_si<S>(csub(x[1], x[3]));
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, d13);
    x[3] = csub(d02, d13);
}

template <int S>
__host__ __device__ __forceinline__ void bfly5(float2 (&x)[5]) {
    // cos/sin of 2 pi/5 and 4 pi/5 from their closed forms in sqrt(5)
    constexpr float c1 = 0.309016994374947424102293417182819f;   // (sqrt5 - 1) / 4
    constexpr float c2 = -0.809016994374947424102293417182819f;  // -(sqrt5 + 1) / 4
    constexpr float s1 = 0.951056516295153572116439333379382f;   // sqrt(10 + 2 sqrt5) / 4
    constexpr float s2 = 0.587785252292473129168705954639073f;   // sqrt(10 - 2 sqrt5) / 4
    const float2 a = x[0];
    const float2 p14 = cadd(x[1], x[4]), m14 = csub(x[1], x[4]);
    const float2 p23 = cadd(x[2], x[3]), m23 = csub(x[2], x[3]);
    const float2 r1 = make_float2(fmaf(c1, p14.x, fmaf(c2, p23.x, a.x)), fmaf(c1, p14.y, fmaf(c2, p23.y, a.y)));
    const float2 r2 = make_float2(fmaf(c2, p14.x, fmaf(c1, p23.x, a.x)), fmaf(c2, p14.y, fmaf(c1, p23.y, a.y)));
    const float2 i1 = mul_si<S>(make_float2(fmaf(s1, m14.x, s2 * m23.x), fmaf(s1, m14.y, s2 * m23.y)));
    const float2 i2 = mul_si<S>(make_float2(fmaf(s2, m14.x, -s1 * m23.x), fmaf(s2, m14.y, -s1 * m23.y)));
    x[0] = cadd(a, cadd(p14, p23));
    x[1] = cadd(r1, i1);
    x[4] = csub(r1, i1);
    x[2] = cadd(r2, i2);
    x[3] = csub(r2, i2);
}

// Plain DFT for a prime radix without a dedicated butterfly.
template <int P, int S>
__host__ __device__ __forceinline__ void dft_prime(float2 (&x)[P]) {
    float2 y[P];
    static_for<0, P>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        float2 acc = x[0];
        static_for<1, P>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            acc = cadd(acc, twiddle<P, S, (j * k) % P>(x[j]));
        });
        y[k] = acc;
    });
#pragma unroll
    for (int k = 0; k < P; ++k) x[k] = y[k];
}

template <int N, int S>
__host__ __device__ __forceinline__ void dft(float2 (&x)[N]) {
    if constexpr (N == 1) {
        return;
    } else if constexpr (N == 2) {
        bfly2<S>(x[0], x[1]);
    } else if constexpr (N == 3) {
        bfly3<S>(x);
    } else if constexpr (N == 4) {
        bfly4<S>(x);
    } else if constexpr (N == 5) {
        bfly5<S>(x);
    } else if constexpr (first_radix<N>() == N) {
        dft_prime<N, S>(x);
    } else if constexpr (coprime_factor<N>() != 0) {
        // Prime-factor split N = A B, gcd(A, B) = 1: input n = (B a + A b) mod
        // N, length-A transforms over a, length-B transforms over b, output
        // k = CRT(k_a, k_b) with W_N^(n k) = W_A^(a k_a) W_B^(b k_b).
        constexpr int A = coprime_factor<N>(), B = N / A;
        constexpr int eA = B * inv_mod(B, A), eB = A * inv_mod(A, B);  // k = (k_a eA + k_b eB) mod N
        float2 t[B][A];
#pragma unroll
        for (int b = 0; b < B; ++b) {
#pragma unroll
            for (int a = 0; a < A; ++a) t[b][a] = x[(B * a + A * b) % N];
            dft<A, S>(t[b]);
        }
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
            float2 u[B];
#pragma unroll
            for (int b = 0; b < B; ++b) u[b] = t[b][ka];
            dft<B, S>(u);
#pragma unroll
            for (int kb = 0; kb < B; ++kb) x[(ka * eA + kb * eB) % N] = u[kb];
        }
    } else {
        // Decimation in time: residue classes j mod P, length-M transforms,
        // twiddles W_N^(r k), then length-P transforms across the classes.
        constexpr int P = first_radix<N>();
        constexpr int M = N / P;
        float2 a[P][M];
#pragma unroll
        for (int r = 0; r < P; ++r)
#pragma unroll
            for (int j = 0; j < M; ++j) a[r][j] = x[j * P + r];
#pragma unroll
        for (int r = 0; r < P; ++r) dft<M, S>(a[r]);
        static_for<0, M>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            float2 t[P];
            static_for<0, P>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                t[r] = twiddle<N, S, r * k>(a[r][k]);
            });
            dft<P, S>(t);
#pragma unroll
            for (int q = 0; q < P; ++q) x[k + q * M] = t[q];
        });
    }
}

// ---------------------------------------------------------------- size plans
// Supported image sizes and their four-step split N = N1 * N2.
template <int N>
struct Plan;
#define BLINK_PLAN(N_, N1_, N2_)                                 \
    template <>                                                  \
    struct Plan<N_> {                                            \
        static constexpr int N = N_, N1 = N1_, N2 = N2_;         \
        static_assert(N1 * N2 == N, "four-step split mismatch"); \
    };
BLINK_PLAN(16, 4, 4)
BLINK_PLAN(20, 4, 5)
BLINK_PLAN(24, 4, 6)
BLINK_PLAN(32, 4, 8)
BLINK_PLAN(36, 6, 6)
BLINK_PLAN(48, 6, 8)
BLINK_PLAN(64, 8, 8)
BLINK_PLAN(96, 8, 12)
BLINK_PLAN(120, 10, 12)
BLINK_PLAN(128, 8, 16)
BLINK_PLAN(160, 10, 16)
BLINK_PLAN(180, 12, 15)
BLINK_PLAN(192, 12, 16)
BLINK_PLAN(256, 16, 16)
BLINK_PLAN(360, 18, 20)
BLINK_PLAN(384, 16, 24)
BLINK_PLAN(512, 16, 32)
BLINK_PLAN(768, 24, 32)
BLINK_PLAN(1024, 32, 32)
#undef BLINK_PLAN

// Four-step twiddles W_N^(n2 k1) (inverse direction) in transposed order,
// index k1 N2 + n2: copied to shared memory they are read by lanes running
// along n2 without bank conflicts (the constant cache would serialise the 32
// distinct addresses of such a warp).
template <int N>
struct FourStepTable {
    c32 v[N];
    constexpr FourStepTable() : v{} {
        for (int k1 = 0; k1 < Plan<N>::N1; ++k1)
            for (int n2 = 0; n2 < Plan<N>::N2; ++n2) {
                const c64d w = unit_root((n2 * k1) % N, N);
                v[k1 * Plan<N>::N2 + n2] = c32{float(w.x), float(w.y)};
            }
    }
};

template <int N>
__device__ FourStepTable<N> g_four_step = FourStepTable<N>();

}  // namespace blink
