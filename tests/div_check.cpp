// Host check of blink::div_by (blink_div.cuh) against IEEE division: random
// quotients over wide exponent ranges, the wavelength and cell-size ranges
// of the cell assignment, exact and near-halfway quotients; then
// blink::axis_cell (FP32 estimate, exact FP64 fallback near cell edges)
// against its definition on 20 M offsets, most of them within 10^-12 to
// 10^-1 cells of a cell edge or of the grid border.  Prints "ok ...".
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

    // axis_cell (FP32 fast path + exact fallback) against its definition:
    // k = llround(RN(RN(d / lambda) / delta_u)), dropped beyond 2N or N/2 - 1
    long long nc = 0, slow = 0;
    const int sizes[] = {16, 20, 24, 32, 36, 48, 64, 96, 120, 128, 160, 180, 192, 256, 360, 384, 512, 768, 1024};
    std::uniform_real_distribution<double> fr(50e6, 350e6), dul(-3.0, 1.0), off(-1e-2, 1e-2);
    std::uniform_int_distribution<int> si(0, 18), lg(-12, -1);
    auto cell_check = [&](double d, double lambda, double du, int n) {
        const double il = 1.0 / lambda, idu = 1.0 / du;
        const float s32 = float(il * idu);
        int k = 12345;
        const bool got = blink::axis_cell(d, lambda, il, du, idu, s32, n, k);
        const double t = (d / lambda) / du;
        bool want = std::fabs(t) <= 2.0 * n;
        long long r = 0;
        if (want) {
            r = std::llround(t);
            want = r <= n / 2 - 1 && r >= -(n / 2 - 1);
        }
        ++nc;
        const float tf = float(d) * s32;
        if (!(std::fabs(tf) < 2.0f * float(n) - 1.0f) ||
            !(std::fabs(std::fabs(tf) - std::trunc(std::fabs(tf)) - 0.5f) > std::fma(std::fabs(tf), 4e-7f, 1e-6f)))
            ++slow;
        if (got != want || (got && k != r)) {
            std::printf("FAIL cell d=%.17g lambda=%.17g du=%.17g n=%d got=%d/%d want=%d/%lld\n", d, lambda, du, n,
                        int(got), k, int(want), r);
            return false;
        }
        return true;
    };
    for (int i = 0; i < 4000000; ++i) {
        const double lambda = 299792458.0 / fr(rng), du = std::pow(10.0, dul(rng));
        const int n = sizes[si(rng)];
        // a quotient near a half-integer (or the grid edge), offset by 10^-12 .. 10^-1 cells
        const double half = std::floor(sgn(rng) * (n / 2 + 2)) + 0.5;
        const double eps = (sgn(rng) < 0 ? -1 : 1) * std::pow(10.0, double(lg(rng)));
        const double d1 = (half + eps) * lambda * du;
        const double d2 = base(rng) * 1e-2;  // anywhere
        if (!cell_check(d1, lambda, du, n) || !cell_check(d2, lambda, du, n)) return 1;
        if (!cell_check(std::nextafter(half * lambda * du, 1e300), lambda, du, n) ||
            !cell_check(std::nextafter(half * lambda * du, -1e300), lambda, du, n) ||
            !cell_check(half * lambda * du, lambda, du, n))
            return 1;
    }
    std::printf("ok %lld quotients, %lld cells (%lld on the exact path)\n", n, nc, slow);
    return 0;
}
