"""The oracle pins must catch plausible mistakes.

Each case copies the oracle source, plants one mistake by a textual edit,
compiles the mutant with gcc (CPU only), points the oracle wrapper at it and
runs the pins: at least one pin has to fail for every mutant.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle_adjoint as adj
from tests import test_oracle_epilogue as epi
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "blink_oracle.c")

MUTANTS = {
    # a dropped Hermitian conjugate entry
    "no_conjugate_entry": ("        grid[2 * q] += re;\n        grid[2 * q + 1] -= im;\n",
                           ""),
    # conjugate entry without the conjugation
    "conjugate_not_conjugated": ("grid[2 * q + 1] -= im;", "grid[2 * q + 1] += im;"),
    # rounding half up instead of half away from zero
    "round_half_up": ("const long r = lround(t);", "const long r = (long)floor(t + 0.5);"),
    # wrong baseline sign convention (i - j)
    "baseline_sign": ("const double dx = ant_xyz[3 * j + 0] - ant_xyz[3 * i + 0];",
                      "const double dx = ant_xyz[3 * i + 0] - ant_xyz[3 * j + 0];"),
    # u and v swapped (transposed image)
    "uv_swapped": ("u[b] = dx / lambda;\n            v[b] = dy / lambda;",
                   "u[b] = dy / lambda;\n            v[b] = dx / lambda;"),
    # forward instead of inverse transform in the direct route
    "direct_wrong_sign": ("im += cg[2 * j] * sn + cg[2 * j + 1] * cs;",
                          "im += -cg[2 * j] * sn + cg[2 * j + 1] * cs;\n"
                          "                re += 2 * cg[2 * j + 1] * sn;"),
    # forward instead of inverse transform in the FFT route
    "fft_wrong_sign": ("orc_fft_rec(a + 2 * (size_t)y * n, 1, n, col, +1, tw, n, tmp);",
                       "orc_fft_rec(a + 2 * (size_t)y * n, 1, n, col, -1, tw, n, tmp);"),
    # missing output fftshift
    "no_output_shift": ("const size_t src = (size_t)((py + h) % n) * n + (size_t)((px + h) % n);",
                        "const size_t src = (size_t)py * n + (size_t)px;"),
    # edge rule one cell too tight (drops valid |k| = N/2 - 1 cells)
    "edge_too_tight": ("const int32_t kmax = n_px / 2 - 1;", "const int32_t kmax = n_px / 2 - 2;"),
    # uniform weight counting only one of the two entries
    "uniform_half_count": ("        cnt[q] += 1;\n", ""),
    # summed weight of natural weighting counting baselines, not entries
    "natural_wsum": ("entries += 2;", "entries += 1;"),
    # adjoint with the inverse instead of the forward kernel (direct route)
    "degrid_wrong_sign": ("im -= r * tw[2 * e + 1]; /* exp(-i theta) */",
                          "im += r * tw[2 * e + 1];"),
    # adjoint missing the factor 2 of V and conj(V) (FFT route)
    "degrid_no_factor_two": ("gamma[2 * b] = 2.0 * w[b] * a[2 * (y * n + x)];",
                             "gamma[2 * b] = w[b] * a[2 * (y * n + x)];"),
    # adjoint ignoring the uniform weights
    "degrid_no_uniform_weight": ("w[b] = 1.0 / (double)cnt[(int64_t)(kv[b] + h) * n_px + (ku[b] + h)];",
                                 "w[b] = 1.0;"),
    # gain chain rule without the conjugate on the second antenna's term
    "gain_grad_conjugate": ("gamma_g[2 * j + 1] += gr * ui - gi * ur;",
                            "gamma_g[2 * j + 1] += gr * ui + gi * ur;"),
    # gain product with the conjugate on the first antenna: conj(g_i) g_j
    "gain_conjugate_swapped": ("const double pi = ai * cr - ar * ci;", "const double pi = ar * ci - ai * cr;"),
    # reference image added instead of subtracted
    "reference_added": ("for (int64_t p = 0; p < (int64_t)n * n; ++p) img[p] -= rf[p];",
                        "for (int64_t p = 0; p < (int64_t)n * n; ++p) img[p] += rf[p];"),
    # every layer reads the first gain row
    "gain_stride_ignored": ("orc_apply_gains(n_ant, gains + 2 * gain_stride * row,",
                            "orc_apply_gains(n_ant, gains,"),
    # gain period ignored (rows run on past the period)
    "gain_period_ignored": ("const int64_t row = gain_period > 0 ? l % gain_period : l;",
                            "const int64_t row = l;"),
}

PINS = [
    pins.test_cells_bruteforce_integer_construction,
    pins.test_cells_round_half_away_from_zero,
    pins.test_grid_uniform_unit_cells,
    pins.test_grid_is_hermitian,
    lambda: pins.test_on_grid_image_equals_direct_dft_sum(0, "direct"),
    lambda: pins.test_on_grid_image_equals_direct_dft_sum(1, "fft"),
    lambda: pins.test_unit_source_at_phase_centre_gives_summed_weight(0),
    pins.test_offcentre_point_source_peaks_at_its_pixel,
    pins.test_single_cell_shift_theorem,
    lambda: pins.test_image_fft_matches_numpy_shifted_ifft2(16),
    lambda: pins.test_grid_counts_match_bruteforce_histogram(5),
    lambda: adj.test_adjoint_dot_product_identity(1, "direct"),
    lambda: adj.test_adjoint_dot_product_identity(0, "fft"),
    lambda: adj.test_visibility_gradient_matches_finite_differences(1),
    adj.test_gain_gradient_matches_finite_differences,
    lambda: epi.test_phase_ramp_gains_move_a_source(0),
    lambda: epi.test_gains_match_bruteforce_direct_sum(1),
    epi.test_gain_rows_follow_the_stride,
    epi.test_reference_subtraction_is_dirty_minus_reference,
]


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="orc_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, workdir, monkeypatch):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = src.replace(old, new, 1)
    c_path = os.path.join(workdir, f"{name}.c")
    so_path = os.path.join(workdir, f"lib{name}.so")
    open(c_path, "w").write(mut)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared",
                    "-fPIC", c_path, "-o", so_path, "-lm"], check=True)
    real = oracle._load()
    mlib = ctypes.CDLL(so_path)
    for fn in ("orc_version", "orc_n_baselines", "orc_uv", "orc_cells", "orc_grid",
               "orc_image_direct", "orc_image_fft", "orc_fft1d", "orc_image_batch",
               "orc_grid_c128", "orc_degrid_direct", "orc_degrid_fft", "orc_gain_grad",
               "orc_apply_gains", "orc_image_batch_ex"):
        getattr(mlib, fn).restype = getattr(real, fn).restype
        getattr(mlib, fn).argtypes = getattr(real, fn).argtypes
    monkeypatch.setattr(oracle, "_lib", mlib)
    failed = 0
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0, f"no pin caught mutant {name}"
