// Host check of the in-register DFT codelets (blink_fft.cuh): every codelet
// length the four-step plans use, both directions, against the direct sum
// X[k] = sum_j x[j] exp(S 2 pi i j k / N) in double precision.  Prints "ok"
// and the worst error relative to the largest output magnitude.
#include <cmath>
#include <cstdio>
#include <random>

#include "blink_fft.cuh"

using namespace blink;

template <int N, int S>
double check(std::mt19937_64 &rng) {
    std::normal_distribution<double> nd(0.0, 1.0);
    double worst = 0.0;
    for (int trial = 0; trial < 50; ++trial) {
        float2 x[N];
        double xr[N], xi[N];
        for (int j = 0; j < N; ++j) {
            xr[j] = float(nd(rng));
            xi[j] = float(nd(rng));
            x[j] = make_float2(float(xr[j]), float(xi[j]));
        }
        dft<N, S>(x);
        double peak = 0.0, err = 0.0;
        for (int k = 0; k < N; ++k) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < N; ++j) {
                const double a = S * 2.0 * M_PI * double((long long)j * k % N) / N;
                sr += xr[j] * std::cos(a) - xi[j] * std::sin(a);
                si += xr[j] * std::sin(a) + xi[j] * std::cos(a);
            }
            peak = std::fmax(peak, std::hypot(sr, si));
            err = std::fmax(err, std::hypot(double(x[k].x) - sr, double(x[k].y) - si));
        }
        worst = std::fmax(worst, err / peak);
    }
    return worst;
}

template <int N>
double both(std::mt19937_64 &rng) {
    return std::fmax(check<N, +1>(rng), check<N, -1>(rng));
}

int main() {
    std::mt19937_64 rng(12345);
    const int sizes[] = {2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 18, 20, 24, 32};
    const double errs[] = {both<2>(rng),  both<3>(rng),  both<4>(rng),  both<5>(rng),  both<6>(rng),
                           both<8>(rng),  both<10>(rng), both<12>(rng), both<15>(rng), both<16>(rng),
                           both<18>(rng), both<20>(rng), both<24>(rng), both<32>(rng)};
    double worst = 0.0;
    for (int i = 0; i < 14; ++i) {
        if (!(errs[i] < 1e-6)) {
            std::printf("FAIL N=%d relative error %.3e\n", sizes[i], errs[i]);
            return 1;
        }
        worst = std::fmax(worst, errs[i]);
    }
    std::printf("ok %.3e\n", worst);
    return 0;
}
