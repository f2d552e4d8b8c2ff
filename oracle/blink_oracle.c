/*
 * blink_oracle.c -- plain FP64 CPU reference for the BLINK dirty-image path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) includes, links or calls this file.  Only tests/, the smoke
 * check in __graft_entry__.py and the cpu_baseline / reference leg of bench.py
 * may load it.  It shares no code, header, table or constant with the GPU path.
 *
 * What it computes (paper: Sokolowski et al., "BLINK", arXiv 2405.13478):
 *
 *   (1) baseline (u,v) in wavelengths: difference of antenna positions divided
 *       by lambda = c / nu, in FP64 (Sec. 5.2.1 step 1; the Fig. 7 listing
 *       computes the wavelength from the channel frequency in double).  The
 *       array is coplanar and phased at zenith, so w is dropped (Sec. 4.3,
 *       Eqs. 4-5).
 *   (2) grid cell: k = round(u / delta_u) with delta_u = 1/(N_px dx)
 *       (Sec. 4.4.1, Eq. 9); cells are indexed so that the centre bin is zero
 *       spatial frequency (Sec. 5.2.1 step 1).
 *   (3) gridding: every visibility is added to its cell and its Hermitian
 *       conjugate to the mirrored cell, with a per-cell counter
 *       (Sec. 5.2.1 steps 2-3; the correlation matrix holds both V_ij and
 *       V_ji = conj(V_ij)).
 *   (4) weighting: natural = plain sum; uniform = each cell divided by its
 *       count (Sec. 4.4.2; Sec. 5.2.1, weighting applied after gridding).
 *   (5) dirty image = real part of the inverse 2-D Fourier transform of the
 *       gridded visibilities, with the FFT shifts that put the phase centre in
 *       the middle of the image (Sec. 4.3, Eq. 6; Sec. 5.2.2).
 *
 * Readings where the paper is silent:
 *   - u = x_j - x_i for the pair (i < j), baselines in lexicographic order;
 *   - round half away from zero (C lround), so cell(-u) = -cell(u);
 *   - a cell is kept iff |k_u| <= N/2-1 and |k_v| <= N/2-1 (the -N/2 bin has
 *     no mirrored partner and is dropped together with anything beyond it);
 *   - uniform weight of a cell = 1/n, n counting both the V and conj(V) entries;
 *   - the inverse transform is unnormalised (exp(+2 pi i ...), no 1/N^2), so a
 *     unit source at the phase centre gives a centre pixel equal to the summed
 *     weight;
 *   - image row y <-> m (v axis), column x <-> l (u axis), centre (N/2, N/2).
 *
 * Two independent evaluations of step 5 are provided: orc_image_direct (the
 * double sum of the definition over occupied cells, with exact integer phase
 * reduction) and orc_image_fft (an FP64 mixed-radix FFT, the way the paper
 * computes it).  Both are pinned in tests/ against closed forms, brute force
 * and numpy.fft.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC.
 * -ffp-contract=off keeps every step 1-2 operation a single IEEE rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C_LIGHT 299792458.0 /* m/s, exact by SI definition */
#define ORC_DROPPED INT32_MIN   /* cell index of a baseline that is not gridded */

int orc_version(void) { return 1; }

int64_t orc_n_baselines(int n_ant) {
    /* cross-correlations only: N_ant (N_ant - 1) / 2 (Table 3, Sec. 5.2.1) */
    return (int64_t)n_ant * (int64_t)(n_ant - 1) / 2;
}

/* ----------------------------------------------------------- 1: (u,v) */
/* ant_xyz: [n_ant][3] metres; u, v: [B] wavelengths, b over pairs (i<j). */
void orc_uv(const double *ant_xyz, int n_ant, double freq_hz, double *u, double *v) {
    const double lambda = ORC_C_LIGHT / freq_hz;
    int64_t b = 0;
    for (int i = 0; i < n_ant; ++i) {
        for (int j = i + 1; j < n_ant; ++j) {
            const double dx = ant_xyz[3 * j + 0] - ant_xyz[3 * i + 0];
            const double dy = ant_xyz[3 * j + 1] - ant_xyz[3 * i + 1];
            u[b] = dx / lambda;
            v[b] = dy / lambda;
            ++b;
        }
    }
}

/* ----------------------------------------------------------- 2: cells */
/* One axis: k = round-half-away(t), t = w / delta_u; returns 0 if dropped. */
static int orc_axis_cell(double w, double delta_u, int n_px, int32_t *k) {
    const double t = w / delta_u;
    const int32_t kmax = n_px / 2 - 1;
    if (!(fabs(t) <= 2.0 * (double)n_px)) return 0; /* far outside (or NaN) */
    const long r = lround(t);
    if (r > kmax || r < -kmax) return 0;
    *k = (int32_t)r;
    return 1;
}

/* ku, kv: [B] signed cell offsets from the centre; ORC_DROPPED when dropped.
 * Returns the number of baselines kept. */
int64_t orc_cells(const double *u, const double *v, int64_t nb, double delta_u, int n_px,
                  int32_t *ku, int32_t *kv) {
    int64_t kept = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int32_t a = 0, c = 0;
        if (orc_axis_cell(u[b], delta_u, n_px, &a) && orc_axis_cell(v[b], delta_u, n_px, &c)) {
            ku[b] = a;
            kv[b] = c;
            ++kept;
        } else {
            ku[b] = ORC_DROPPED;
            kv[b] = ORC_DROPPED;
        }
    }
    return kept;
}

/* ------------------------------------------------------- 3-4: grid */
/* vis: [B] complex64 (re, im interleaved floats).
 * grid: [N][N] complex128 (re, im interleaved doubles), row y = k_v + N/2,
 *       column x = k_u + N/2 (zero spatial frequency in the centre bin).
 * count: [N][N] number of entries per cell (may be NULL).
 * weighting: 0 natural, 1 uniform.  *wsum = summed weight of all entries.
 * Returns 0, or -1 on a bad argument. */
static int orc_grid_any(const int32_t *ku, const int32_t *kv, const float *vis32, const double *vis64,
                        int64_t nb, int n_px, int weighting, double *grid, int32_t *count,
                        double *wsum);

int orc_grid(const int32_t *ku, const int32_t *kv, const float *vis, int64_t nb, int n_px,
             int weighting, double *grid, int32_t *count, double *wsum) {
    return orc_grid_any(ku, kv, vis, NULL, nb, n_px, weighting, grid, count, wsum);
}

/* Same with complex128 visibilities (used by the finite-difference pins). */
int orc_grid_c128(const int32_t *ku, const int32_t *kv, const double *vis, int64_t nb, int n_px,
                  int weighting, double *grid, int32_t *count, double *wsum) {
    return orc_grid_any(ku, kv, NULL, vis, nb, n_px, weighting, grid, count, wsum);
}

static int orc_grid_any(const int32_t *ku, const int32_t *kv, const float *vis32, const double *vis64,
                        int64_t nb, int n_px, int weighting, double *grid, int32_t *count,
                        double *wsum) {
    if (n_px < 4 || (n_px & 1) || (weighting != 0 && weighting != 1)) return -1;
    const int64_t npix = (int64_t)n_px * n_px;
    int32_t *cnt = count ? count : (int32_t *)malloc(sizeof(int32_t) * (size_t)npix);
    if (!cnt) return -1;
    memset(grid, 0, sizeof(double) * 2 * (size_t)npix);
    memset(cnt, 0, sizeof(int32_t) * (size_t)npix);
    const int h = n_px / 2;
    int64_t entries = 0;
    for (int64_t b = 0; b < nb; ++b) {
        if (ku[b] == ORC_DROPPED) continue;
        const double re = vis32 ? (double)vis32[2 * b] : vis64[2 * b];
        const double im = vis32 ? (double)vis32[2 * b + 1] : vis64[2 * b + 1];
        /* V_ij at (u, v) */
        const int64_t p = (int64_t)(kv[b] + h) * n_px + (ku[b] + h);
        grid[2 * p] += re;
        grid[2 * p + 1] += im;
        cnt[p] += 1;
        /* V_ji = conj(V_ij) at (-u, -v) */
        const int64_t q = (int64_t)(-kv[b] + h) * n_px + (-ku[b] + h);
        grid[2 * q] += re;
        grid[2 * q + 1] -= im;
        cnt[q] += 1;
        entries += 2;
    }
    if (weighting == 1) {
        int64_t occupied = 0;
        for (int64_t p = 0; p < npix; ++p) {
            if (cnt[p] > 0) {
                grid[2 * p] /= (double)cnt[p];
                grid[2 * p + 1] /= (double)cnt[p];
                ++occupied;
            }
        }
        *wsum = (double)occupied; /* every occupied cell carries weight 1 */
    } else {
        *wsum = (double)entries; /* every entry carries weight 1 */
    }
    if (!count) free(cnt);
    return 0;
}

/* ---------------------------------------------------------- twiddle table */
/* tw[2m], tw[2m+1] = cos, sin of 2 pi m / n, m = 0..n-1. */
static double *orc_twiddles(int n) {
    double *tw = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!tw) return NULL;
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < n; ++m) {
        tw[2 * m] = cos(two_pi * (double)m / (double)n);
        tw[2 * m + 1] = sin(two_pi * (double)m / (double)n);
    }
    return tw;
}

/* ------------------------------------------ 5: direct definition */
/* image[py][px] = Re sum_k G[k] exp(+2 pi i (k_u (px - N/2) + k_v (py - N/2)) / N)
 * summed over every non-zero cell; the phase is reduced modulo N in integers
 * before the table lookup, so no large-argument trigonometry is involved.
 * *max_abs_imag receives max |Im| over the image (0 for a Hermitian grid). */
int orc_image_direct(const double *grid, int n_px, double *image, double *max_abs_imag) {
    if (n_px < 4 || (n_px & 1)) return -1;
    const int n = n_px, h = n_px / 2;
    const int64_t npix = (int64_t)n * n;
    int64_t nocc = 0;
    for (int64_t p = 0; p < npix; ++p)
        if (grid[2 * p] != 0.0 || grid[2 * p + 1] != 0.0) ++nocc;
    int32_t *ck = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(nocc + 1));
    double *cg = (double *)malloc(sizeof(double) * 2 * (size_t)(nocc + 1));
    double *tw = orc_twiddles(n);
    if (!ck || !cg || !tw) { free(ck); free(cg); free(tw); return -1; }
    int64_t c = 0;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            const int64_t p = (int64_t)y * n + x;
            if (grid[2 * p] != 0.0 || grid[2 * p + 1] != 0.0) {
                ck[2 * c] = x - h; /* k_u */
                ck[2 * c + 1] = y - h; /* k_v */
                cg[2 * c] = grid[2 * p];
                cg[2 * c + 1] = grid[2 * p + 1];
                ++c;
            }
        }
    double worst = 0.0;
    for (int py = 0; py < n; ++py) {
        for (int px = 0; px < n; ++px) {
            double re = 0.0, im = 0.0;
            for (int64_t j = 0; j < nocc; ++j) {
                int64_t e = (int64_t)ck[2 * j] * (px - h) + (int64_t)ck[2 * j + 1] * (py - h);
                e %= n;
                if (e < 0) e += n;
                const double cs = tw[2 * e], sn = tw[2 * e + 1];
                re += cg[2 * j] * cs - cg[2 * j + 1] * sn;
                im += cg[2 * j] * sn + cg[2 * j + 1] * cs;
            }
            image[(int64_t)py * n + px] = re;
            if (fabs(im) > worst) worst = fabs(im);
        }
    }
    if (max_abs_imag) *max_abs_imag = worst;
    free(ck); free(cg); free(tw);
    return 0;
}

/* --------------------------------------------------- FP64 mixed-radix FFT */
static int orc_smallest_factor(int n) {
    if (n % 2 == 0) return 2;
    for (int p = 3; p * p <= n; p += 2)
        if (n % p == 0) return p;
    return n;
}

/* out[k] = sum_{j<n} in[j*stride] exp(sign 2 pi i j k / n), complex interleaved.
 * Decimation in time: n = p*m, input split by residue r = j mod p, each
 * residue class transformed recursively, then combined with
 * X[k + q m] = sum_r W_n^{r(k + q m)} Y_r[k].  tw holds W_ntot; W_n^e is
 * W_ntot^{e*ntot/n}. */
static void orc_fft_rec(const double *in, int64_t stride, int n, double *out, int sign,
                        const double *tw, int ntot, double *tmp) {
    if (n == 1) {
        out[0] = in[0];
        out[1] = in[1];
        return;
    }
    const int p = orc_smallest_factor(n), m = n / p;
    for (int r = 0; r < p; ++r)
        orc_fft_rec(in + 2 * (int64_t)r * stride, stride * p, m, out + 2 * (int64_t)r * m, sign, tw,
                    ntot, tmp);
    const int scale = ntot / n;
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) {
            tmp[2 * r] = out[2 * ((int64_t)r * m + k)];
            tmp[2 * r + 1] = out[2 * ((int64_t)r * m + k) + 1];
        }
        for (int q = 0; q < p; ++q) {
            const int64_t kk = (int64_t)k + (int64_t)q * m;
            double re = 0.0, im = 0.0;
            for (int r = 0; r < p; ++r) {
                const int64_t e = ((int64_t)r * kk) % n * scale;
                const double cs = tw[2 * e], sn = sign * tw[2 * e + 1];
                re += tmp[2 * r] * cs - tmp[2 * r + 1] * sn;
                im += tmp[2 * r] * sn + tmp[2 * r + 1] * cs;
            }
            tmp[2 * (p + q)] = re;
            tmp[2 * (p + q) + 1] = im;
        }
        for (int q = 0; q < p; ++q) {
            out[2 * ((int64_t)k + (int64_t)q * m)] = tmp[2 * (p + q)];
            out[2 * ((int64_t)k + (int64_t)q * m) + 1] = tmp[2 * (p + q) + 1];
        }
    }
}

/* 1-D transform of a complex vector (exported for the FFT pins). */
int orc_fft1d(const double *in, int n, int sign, double *out) {
    if (n < 1 || (sign != 1 && sign != -1)) return -1;
    double *tw = orc_twiddles(n);
    double *tmp = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    if (!tw || !tmp) { free(tw); free(tmp); return -1; }
    orc_fft_rec(in, 1, n, out, sign, tw, n, tmp);
    free(tw); free(tmp);
    return 0;
}

/* -------------------------------------------- 5: FFT with shifts */
/* ifftshift (centre bin -> index 0), unnormalised inverse 2-D FFT, fftshift
 * (index 0 -> centre pixel), real part (Sec. 5.2.2). */
int orc_image_fft(const double *grid, int n_px, double *image, double *max_abs_imag) {
    if (n_px < 4 || (n_px & 1)) return -1;
    const int n = n_px, h = n_px / 2;
    const size_t npix = (size_t)n * n;
    double *a = (double *)malloc(sizeof(double) * 2 * npix);
    double *col = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    double *tw = orc_twiddles(n);
    double *tmp = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    if (!a || !col || !tw || !tmp) { free(a); free(col); free(tw); free(tmp); return -1; }
    /* ifftshift: a[y'][x'] = G[(y'+h) mod n][(x'+h) mod n] */
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            const size_t src = (size_t)((y + h) % n) * n + (size_t)((x + h) % n);
            a[2 * ((size_t)y * n + x)] = grid[2 * src];
            a[2 * ((size_t)y * n + x) + 1] = grid[2 * src + 1];
        }
    /* rows (u axis) */
    for (int y = 0; y < n; ++y) {
        orc_fft_rec(a + 2 * (size_t)y * n, 1, n, col, +1, tw, n, tmp);
        memcpy(a + 2 * (size_t)y * n, col, sizeof(double) * 2 * (size_t)n);
    }
    /* columns (v axis) */
    for (int x = 0; x < n; ++x) {
        orc_fft_rec(a + 2 * (size_t)x, n, n, col, +1, tw, n, tmp);
        for (int y = 0; y < n; ++y) {
            a[2 * ((size_t)y * n + x)] = col[2 * y];
            a[2 * ((size_t)y * n + x) + 1] = col[2 * y + 1];
        }
    }
    /* fftshift + real part */
    double worst = 0.0;
    for (int py = 0; py < n; ++py)
        for (int px = 0; px < n; ++px) {
            const size_t src = (size_t)((py + h) % n) * n + (size_t)((px + h) % n);
            image[(size_t)py * n + px] = a[2 * src];
            if (fabs(a[2 * src + 1]) > worst) worst = fabs(a[2 * src + 1]);
        }
    if (max_abs_imag) *max_abs_imag = worst;
    free(a); free(col); free(tw); free(tmp);
    return 0;
}

/* ------------------------------------------------- adjoint (degridding) */
/* Gradient of a real loss L(image) with respect to the visibilities.  The
 * image is linear in V: I[p] = sum_b w_b 2 Re(V_b E(k_b, p)) with
 * E(k, p) = exp(+2 pi i k.(p - N/2) / N) (Sec. 4.3 Eq. 6 with the gridding of
 * Sec. 5.2.1; w_b = 1 natural, 1/n(cell) uniform).  With R = dL/dI, the
 * gradient in the convention dL/dRe V + i dL/dIm V is
 *     gamma_b = 2 w_b H[k_b],  H[k] = sum_p R[p] exp(-2 pi i k.(p - N/2) / N),
 * and zero for baselines that are not gridded (the paper does not
 * differentiate the imager; this is the adjoint of the map above). */
static int orc_entry_weights(const int32_t *ku, const int32_t *kv, int64_t nb, int n_px,
                             int weighting, double *w) {
    const int h = n_px / 2;
    int32_t *cnt = (int32_t *)calloc((size_t)n_px * n_px, sizeof(int32_t));
    if (!cnt) return -1;
    for (int64_t b = 0; b < nb; ++b) {
        if (ku[b] == ORC_DROPPED) continue;
        cnt[(int64_t)(kv[b] + h) * n_px + (ku[b] + h)] += 1;
        cnt[(int64_t)(-kv[b] + h) * n_px + (-ku[b] + h)] += 1;
    }
    for (int64_t b = 0; b < nb; ++b) {
        if (ku[b] == ORC_DROPPED) {
            w[b] = 0.0;
        } else if (weighting == 1) {
            w[b] = 1.0 / (double)cnt[(int64_t)(kv[b] + h) * n_px + (ku[b] + h)];
        } else {
            w[b] = 1.0;
        }
    }
    free(cnt);
    return 0;
}

/* Direct sum over pixels (small images).  resid: [N][N]; gamma: [B] complex. */
int orc_degrid_direct(const int32_t *ku, const int32_t *kv, int64_t nb, int n_px, int weighting,
                      const double *resid, double *gamma) {
    if (n_px < 4 || (n_px & 1)) return -1;
    const int n = n_px, h = n_px / 2;
    double *w = (double *)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    double *tw = orc_twiddles(n);
    if (!w || !tw || orc_entry_weights(ku, kv, nb, n, weighting, w)) { free(w); free(tw); return -1; }
    for (int64_t b = 0; b < nb; ++b) {
        double re = 0.0, im = 0.0;
        if (ku[b] != ORC_DROPPED) {
            for (int py = 0; py < n; ++py)
                for (int px = 0; px < n; ++px) {
                    int64_t e = (int64_t)ku[b] * (px - h) + (int64_t)kv[b] * (py - h);
                    e %= n;
                    if (e < 0) e += n;
                    const double r = resid[(int64_t)py * n + px];
                    re += r * tw[2 * e];
                    im -= r * tw[2 * e + 1]; /* exp(-i theta) */
                }
        }
        gamma[2 * b] = 2.0 * w[b] * re;
        gamma[2 * b + 1] = 2.0 * w[b] * im;
    }
    free(w); free(tw);
    return 0;
}

/* Same through an FP64 forward 2-D FFT of the ifftshifted residual. */
int orc_degrid_fft(const int32_t *ku, const int32_t *kv, int64_t nb, int n_px, int weighting,
                   const double *resid, double *gamma) {
    if (n_px < 4 || (n_px & 1)) return -1;
    const int n = n_px, h = n_px / 2;
    const size_t npix = (size_t)n * n;
    double *a = (double *)malloc(sizeof(double) * 2 * npix);
    double *col = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    double *tw = orc_twiddles(n);
    double *tmp = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    if (!a || !col || !tw || !tmp || !w || orc_entry_weights(ku, kv, nb, n, weighting, w)) {
        free(a); free(col); free(tw); free(tmp); free(w);
        return -1;
    }
    /* a[n_y][n_x] = R[(n_y + h) mod n][(n_x + h) mod n]: pixel offset p - N/2 in FFT order */
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            a[2 * ((size_t)y * n + x)] = resid[(size_t)((y + h) % n) * n + (size_t)((x + h) % n)];
            a[2 * ((size_t)y * n + x) + 1] = 0.0;
        }
    for (int y = 0; y < n; ++y) {
        orc_fft_rec(a + 2 * (size_t)y * n, 1, n, col, -1, tw, n, tmp);
        memcpy(a + 2 * (size_t)y * n, col, sizeof(double) * 2 * (size_t)n);
    }
    for (int x = 0; x < n; ++x) {
        orc_fft_rec(a + 2 * (size_t)x, n, n, col, -1, tw, n, tmp);
        for (int y = 0; y < n; ++y) {
            a[2 * ((size_t)y * n + x)] = col[2 * y];
            a[2 * ((size_t)y * n + x) + 1] = col[2 * y + 1];
        }
    }
    for (int64_t b = 0; b < nb; ++b) {
        if (ku[b] == ORC_DROPPED) {
            gamma[2 * b] = gamma[2 * b + 1] = 0.0;
            continue;
        }
        const size_t y = (size_t)((kv[b] % n + n) % n), x = (size_t)((ku[b] % n + n) % n);
        gamma[2 * b] = 2.0 * w[b] * a[2 * (y * n + x)];
        gamma[2 * b + 1] = 2.0 * w[b] * a[2 * (y * n + x) + 1];
    }
    free(a); free(col); free(tw); free(tmp); free(w);
    return 0;
}

/* Chain rule to per-antenna gains for V_ij = g_i conj(g_j) M_ij (i < j):
 * gamma(g_i) += sum_{j>i} gamma(V_ij) g_j conj(M_ij)
 *             + sum_{k<i} conj(gamma(V_ki)) g_k M_ki          (accumulates). */
void orc_gain_grad(int n_ant, const double *gamma_v, const double *gains, const double *model,
                   double *gamma_g) {
    int64_t b = 0;
    for (int i = 0; i < n_ant; ++i) {
        for (int j = i + 1; j < n_ant; ++j, ++b) {
            const double gr = gamma_v[2 * b], gi = gamma_v[2 * b + 1];
            const double mr = model[2 * b], mi = model[2 * b + 1];
            /* term for g_i: gamma * g_j * conj(M) */
            const double tr = gains[2 * j] * mr + gains[2 * j + 1] * mi;  /* g_j conj(M) */
            const double ti = gains[2 * j + 1] * mr - gains[2 * j] * mi;
            gamma_g[2 * i] += gr * tr - gi * ti;
            gamma_g[2 * i + 1] += gr * ti + gi * tr;
            /* term for g_j: conj(gamma) * g_i * M */
            const double ur = gains[2 * i] * mr - gains[2 * i + 1] * mi;  /* g_i M */
            const double ui = gains[2 * i] * mi + gains[2 * i + 1] * mr;
            gamma_g[2 * j] += gr * ur + gi * ui;
            gamma_g[2 * j + 1] += gr * ui - gi * ur;
        }
    }
}

/* ----------------------------------- calibration gains (Sec. 4.2, step ii) */
/* Antenna-based complex gains applied after correlation: the visibility of
 * the pair (i < j) becomes g_i conj(g_j) V_ij.  gains: [n_ant] complex128;
 * vis: [B] complex64; out: [B] complex128 (re, im interleaved).  To remove a
 * calibration solution pass its reciprocal gains. */
void orc_apply_gains(int n_ant, const double *gains, const float *vis, double *out) {
    int64_t b = 0;
    for (int i = 0; i < n_ant; ++i) {
        const double ar = gains[2 * i], ai = gains[2 * i + 1];
        for (int j = i + 1; j < n_ant; ++j, ++b) {
            const double cr = gains[2 * j], ci = gains[2 * j + 1];
            /* g_i conj(g_j) = (ar + i ai)(cr - i ci) */
            const double pr = ar * cr + ai * ci;
            const double pi = ai * cr - ar * ci;
            const double vr = vis[2 * b], vi = vis[2 * b + 1];
            out[2 * b] = pr * vr - pi * vi;
            out[2 * b + 1] = pr * vi + pi * vr;
        }
    }
}

/* --------------------------------------------------- whole path, batched */
/* One layer = one (time step, channel) image (Sec. 5.2.4).  Layer l reads
 * B = n_ant(n_ant-1)/2 complex64 visibilities at vis + 2*vis_off[l] and writes
 * n_px[l]^2 doubles at images + out_off[l]; wsum[l] gets the summed weight.
 * mode 0: FFT route, mode 1: direct route.  n_threads <= 0: all cores.
 * Returns 0 or the first non-zero layer status. */
int orc_image_batch_ex(const double *ant_xyz, int n_ant, int n_layers, const int32_t *n_px,
                       const int32_t *weighting, const double *freq_hz, const double *delta_u,
                       const int64_t *vis_off, const int64_t *out_off, const float *vis,
                       const double *gains, int64_t gain_stride, int64_t gain_period,
                       const double *ref, double *images, double *wsum, int mode, int n_threads);

int orc_image_batch(const double *ant_xyz, int n_ant, int n_layers, const int32_t *n_px,
                    const int32_t *weighting, const double *freq_hz, const double *delta_u,
                    const int64_t *vis_off, const int64_t *out_off, const float *vis,
                    double *images, double *wsum, int mode, int n_threads) {
    return orc_image_batch_ex(ant_xyz, n_ant, n_layers, n_px, weighting, freq_hz, delta_u, vis_off,
                              out_off, vis, NULL, 0, 0, NULL, images, wsum, mode, n_threads);
}

/* The same with the two optional steps around the imager that transient
 * searches use:
 *   gains (may be NULL): layer l's visibilities are first multiplied by
 *     g_i conj(g_j) with the gain row gains + 2 * r * gain_stride, r = l mod
 *     gain_period (r = l when gain_period <= 0), complex128 [n_ant];
 *     gain_stride 0 = one row for every layer; gain_period = number of
 *     channels gives per-channel gains for time-major layers (Sec. 4.2,
 *     step ii);
 *   ref (may be NULL): a reference image is subtracted from each dirty image,
 *     image = dirty - ref, ref read at the layer's out_off like the output
 *     (Sec. 2 and Sec. 4.3 after Eq. 6: side-lobes of a transient search are
 *     removed by subtracting a reference image of the same field). */
int orc_image_batch_ex(const double *ant_xyz, int n_ant, int n_layers, const int32_t *n_px,
                       const int32_t *weighting, const double *freq_hz, const double *delta_u,
                       const int64_t *vis_off, const int64_t *out_off, const float *vis,
                       const double *gains, int64_t gain_stride, int64_t gain_period,
                       const double *ref, double *images, double *wsum, int mode, int n_threads) {
    const int64_t nb = orc_n_baselines(n_ant);
    int status = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_num_procs();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int l = 0; l < n_layers; ++l) {
        const int n = n_px[l];
        double *u = (double *)malloc(sizeof(double) * (size_t)nb);
        double *v = (double *)malloc(sizeof(double) * (size_t)nb);
        int32_t *ku = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
        int32_t *kv = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
        double *g = (double *)malloc(sizeof(double) * 2 * (size_t)n * n);
        double *vg = gains ? (double *)malloc(sizeof(double) * 2 * (size_t)nb) : NULL;
        int st = (!u || !v || !ku || !kv || !g || (gains && !vg)) ? -1 : 0;
        if (!st) {
            orc_uv(ant_xyz, n_ant, freq_hz[l], u, v);
            orc_cells(u, v, nb, delta_u[l], n, ku, kv);
            if (gains) {
                const int64_t row = gain_period > 0 ? l % gain_period : l;
                orc_apply_gains(n_ant, gains + 2 * gain_stride * row, vis + 2 * vis_off[l], vg);
                st = orc_grid_c128(ku, kv, vg, nb, n, weighting[l], g, NULL, &wsum[l]);
            } else {
                st = orc_grid(ku, kv, vis + 2 * vis_off[l], nb, n, weighting[l], g, NULL, &wsum[l]);
            }
        }
        if (!st) {
            double mi = 0.0;
            st = mode == 1 ? orc_image_direct(g, n, images + out_off[l], &mi)
                           : orc_image_fft(g, n, images + out_off[l], &mi);
        }
        if (!st && ref) {
            double *img = images + out_off[l];
            const double *rf = ref + out_off[l];
            for (int64_t p = 0; p < (int64_t)n * n; ++p) img[p] -= rf[p];
        }
        free(u); free(v); free(ku); free(kv); free(g); free(vg);
        if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
            if (!status) status = st;
        }
    }
    return status;
}
