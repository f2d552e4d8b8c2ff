// Host check of blink::div_by (blink_div.cuh) against IEEE division: random
// quotients over wide exponent ranges, the wavelength and cell-size ranges
// of the cell assignment, exact and near-halfway quotients.  Prints "ok N".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#define __host__
#define __device__
#include "blink_div.cuh"

static uint64_t bits(double x) {
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
}

int main() {
    std::mt19937_64 rng(2405);
    std::uniform_real_distribution<double> unit(1.0, 2.0), sgn(-1.0, 1.0);
    std::uniform_int_distribution<int> ex(-300, 300);
    long long n = 0;
    auto check = [&](double a, double b) {
        const double y = 1.0 / b;
        const double got = blink::div_by(a, b, y), want = a / b;
        ++n;
        if (bits(got) != bits(want)) {
            std::printf("FAIL a=%.17g b=%.17g got=%.17g want=%.17g\n", a, b, got, want);
            return false;
        }
        return true;
    };
    for (int i = 0; i < 4000000; ++i) {  // random significands and exponents
        const double a = std::ldexp(unit(rng), ex(rng)) * (sgn(rng) < 0 ? -1 : 1);
        const double b = std::ldexp(unit(rng), ex(rng)) * (sgn(rng) < 0 ? -1 : 1);
        if (!check(a, b)) return 1;
    }
    std::uniform_real_distribution<double> base(-2.0e5, 2.0e5), lam(0.05, 30.0), du(1e-3, 50.0);
    for (int i = 0; i < 4000000; ++i) {  // baseline / wavelength, then / cell size
        const double a = base(rng), b = lam(rng), c = du(rng);
        if (!check(a, b) || !check(a / b, c)) return 1;
    }
    std::uniform_int_distribution<int64_t> qi(-(int64_t(1) << 40), int64_t(1) << 40);
    for (int i = 0; i < 2000000; ++i) {  // exact and near-halfway quotients
        const double b = lam(rng), q = double(qi(rng)) + 0.5;
        const double a = q * b;
        if (!check(a, b) || !check(std::nextafter(a, 1e300), b) || !check(std::nextafter(a, -1e300), b)) return 1;
        const double c = du(rng), k = double(qi(rng) % 4096) + 0.5;
        if (!check(k * c, c) || !check(std::nextafter(k * c, 1e300), c) || !check(std::nextafter(k * c, -1e300), c))
            return 1;
    }
    const double edge[] = {0.0, -0.0, 1e-310, -1e-310, 1e300, 3.0, 7.0, 0.1, 299792458.0};
    for (double a : edge)
        for (double b : {3.0, 0.1, 1.7, 1e-5, 2.0})
            if (!check(a, b)) return 1;
    std::printf("ok %lld\n", n);
    return 0;
}
