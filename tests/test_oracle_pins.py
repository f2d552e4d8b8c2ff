"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself or with the GPU path.  Each test
uses an independent route: exact integer arithmetic, closed forms, brute force
on tiny inputs, numpy.fft, or a golden value printed in the paper.  Every
plausible slip in the oracle (a dropped conjugate term, a flipped exponent
sign, transposed axes, a wrong shift, a wrong rounding rule, a wrong weight or
summed weight) makes at least one of these fail.
"""
import math
import os

import numpy as np
import pytest

import oracle

C = oracle.C_LIGHT
NU_LAMBDA2 = C / 2.0  # 149896229 Hz: lambda = c / nu = 2 m exactly
HERE = os.path.dirname(os.path.abspath(__file__))


def int_array(n_ant, lo, hi, seed):
    rng = np.random.default_rng(seed)
    xyz = np.zeros((n_ant, 3))
    xyz[:, :2] = rng.integers(lo, hi, size=(n_ant, 2))
    return xyz


def brute_pairs(n_ant):
    return [(i, j) for i in range(n_ant) for j in range(i + 1, n_ant)]


# ------------------------------------------------------ uv and cells
def test_lambda_is_exact():
    assert C / NU_LAMBDA2 == 2.0


def test_uv_exact_on_integer_positions():
    xyz = int_array(9, -40, 40, 1)
    u, v = oracle.uv(xyz, NU_LAMBDA2)
    for b, (i, j) in enumerate(brute_pairs(9)):
        assert u[b] == (xyz[j, 0] - xyz[i, 0]) / 2.0
        assert v[b] == (xyz[j, 1] - xyz[i, 1]) / 2.0


def test_cells_bruteforce_integer_construction():
    # lambda = 2 m and delta_u = 0.5 -> u / delta_u = dx exactly, so k = dx.
    n_px = 64
    xyz = int_array(24, -40, 40, 2)
    u, v = oracle.uv(xyz, NU_LAMBDA2)
    ku, kv = oracle.cells(u, v, 0.5, n_px)
    kmax = n_px // 2 - 1
    n_drop = 0
    for b, (i, j) in enumerate(brute_pairs(24)):
        dx = int(xyz[j, 0] - xyz[i, 0])
        dy = int(xyz[j, 1] - xyz[i, 1])
        if abs(dx) <= kmax and abs(dy) <= kmax:
            assert (ku[b], kv[b]) == (dx, dy)
        else:
            assert ku[b] == oracle.DROPPED and kv[b] == oracle.DROPPED
            n_drop += 1
    assert n_drop > 0  # the edge rule was exercised


def test_cells_round_half_away_from_zero():
    # delta_u = 1, lambda = 2: t = dx / 2, so odd dx sits exactly on a tie.
    xyz = np.zeros((2, 3))
    for dx in range(-9, 10):
        xyz[1, 0] = dx
        xyz[1, 1] = -dx
        u, v = oracle.uv(xyz, NU_LAMBDA2)
        ku, kv = oracle.cells(u, v, 1.0, 64)
        want = int(math.copysign(math.floor(abs(dx) / 2 + 0.5), dx))
        assert ku[0] == want and kv[0] == -want


def test_cells_mirror_symmetry():
    # Reflecting the array through the origin reverses every baseline.
    rng = np.random.default_rng(3)
    xyz = np.zeros((30, 3))
    xyz[:, :2] = rng.uniform(-1500, 1500, (30, 2))
    u, v = oracle.uv(xyz, 160e6)
    ur, vr = oracle.uv(-xyz, 160e6)
    du = np.abs(np.concatenate([u, v])).max() / 60
    ku, kv = oracle.cells(u, v, du, 128)
    kur, kvr = oracle.cells(ur, vr, du, 128)
    keep = ku != oracle.DROPPED
    assert np.array_equal(ku[keep], -kur[keep]) and np.array_equal(kv[keep], -kvr[keep])
    assert np.array_equal(kur[~keep], ku[~keep])


# -------------------------------------------------- grid and weights
def tiny_case(n_ant=6, n_px=16, seed=5, lo=-6, hi=7):
    xyz = int_array(n_ant, lo, hi, seed)
    u, v = oracle.uv(xyz, NU_LAMBDA2)
    ku, kv = oracle.cells(u, v, 0.5, n_px)
    return xyz, u, v, ku, kv


def histogram(ku, kv, n_px):
    h = n_px // 2
    cnt = {}
    for a, c in zip(ku, kv):
        if a == oracle.DROPPED:
            continue
        for s in (1, -1):
            key = (s * c + h, s * a + h)
            cnt[key] = cnt.get(key, 0) + 1
    return cnt


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_grid_counts_match_bruteforce_histogram(seed):
    n_px = 16
    _, _, _, ku, kv = tiny_case(8, n_px, seed)
    g, cnt, ws = oracle.grid(ku, kv, np.ones(ku.size, np.complex64), n_px, 0)
    ref = histogram(ku, kv, n_px)
    dense = np.zeros((n_px, n_px), np.int64)
    for (y, x), c in ref.items():
        dense[y, x] = c
    assert np.array_equal(cnt, dense)
    # natural weighting with V = 1: the grid IS the weight map
    assert np.array_equal(g.real, dense.astype(float)) and not g.imag.any()
    assert ws == 2 * int((ku != oracle.DROPPED).sum()) == dense.sum()


def test_grid_uniform_unit_cells():
    n_px = 16
    _, _, _, ku, kv = tiny_case(9, n_px, 11)
    g, cnt, ws = oracle.grid(ku, kv, np.ones(ku.size, np.complex64), n_px, 1)
    occ = cnt > 0
    assert np.all(g[occ] == 1.0) and not g[~occ].any()
    assert ws == occ.sum()


def test_grid_is_hermitian():
    n_px = 32
    rng = np.random.default_rng(8)
    _, _, _, ku, kv = tiny_case(12, n_px, 9, -12, 13)
    vis = (rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)).astype(np.complex64)
    for w in (0, 1):
        g, _, _ = oracle.grid(ku, kv, vis, n_px, w)
        # G[-k] = conj(G[k]); index of -k is (n - y, n - x) for y, x >= 1
        inner = g[1:, 1:]
        assert np.allclose(inner[::-1, ::-1], np.conj(inner), rtol=0, atol=1e-12)
        assert not g[0, :].any() and not g[:, 0].any()  # the -N/2 bins stay empty


# ------------------------------------------------------------ image
def direct_baseline_sum(u, v, vis, weights, delta_u, n_px):
    """sum_b w_b 2 Re(V_b exp(+2 pi i (u_b l + v_b m))) on the pixel grid."""
    p = (np.arange(n_px) - n_px // 2) / (n_px * delta_u)
    L = p[None, :]          # column <-> l
    M = p[:, None]          # row    <-> m
    img = np.zeros((n_px, n_px))
    for b in range(u.size):
        ph = 2 * np.pi * (u[b] * L + v[b] * M)
        img += weights[b] * 2 * np.real(vis[b] * np.exp(1j * ph))
    return img


@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("mode", ["direct", "fft"])
def test_on_grid_image_equals_direct_dft_sum(weighting, mode):
    n_px, du = 16, 0.5
    xyz, u, v, ku, kv = tiny_case(6, n_px, 21)
    rng = np.random.default_rng(22)
    vis = (rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)).astype(np.complex64)
    img, ws, mi = oracle.image(xyz, NU_LAMBDA2, du, n_px, weighting, vis, mode)
    keep = ku != oracle.DROPPED
    if weighting == 0:
        w = keep.astype(float)
    else:
        cnt = histogram(ku, kv, n_px)
        h = n_px // 2
        w = np.array([1.0 / cnt[(c + h, a + h)] if a != oracle.DROPPED else 0.0
                      for a, c in zip(ku, kv)])
    ref = direct_baseline_sum(u, v, vis.astype(np.complex128), w, du, n_px)
    assert np.abs(img - ref).max() <= 1e-12 * np.abs(ref).max()
    assert mi <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("weighting", [0, 1])
def test_unit_source_at_phase_centre_gives_summed_weight(weighting):
    xyz = int_array(20, -30, 31, 4)
    n_px = 64
    u, v = oracle.uv(xyz, NU_LAMBDA2)
    ku, _ = oracle.cells(u, v, 0.5, n_px)
    vis = np.ones(ku.size, np.complex64)
    for mode in ("direct", "fft"):
        img, ws, _ = oracle.image(xyz, NU_LAMBDA2, 0.5, n_px, weighting, vis, mode)
        assert img[n_px // 2, n_px // 2] == pytest.approx(ws, rel=1e-13)
        assert img.max() == pytest.approx(ws, rel=1e-13)


def test_offcentre_point_source_peaks_at_its_pixel():
    # On-grid uv and a source exactly on pixel (py0, px0) != transposed pixel:
    # every term is in phase there, so the peak equals the summed weight.
    n_px, du = 32, 0.5
    xyz = int_array(10, -14, 15, 31)
    u, v = oracle.uv(xyz, NU_LAMBDA2)
    ku, kv = oracle.cells(u, v, du, n_px)
    px0, py0 = 21, 9
    l0 = (px0 - n_px // 2) / (n_px * du)
    m0 = (py0 - n_px // 2) / (n_px * du)
    vis = np.exp(-2j * np.pi * (u * l0 + v * m0)).astype(np.complex64)
    for mode in ("direct", "fft"):
        img, ws, _ = oracle.image(xyz, NU_LAMBDA2, du, n_px, 0, vis, mode)
        assert np.unravel_index(np.argmax(img), img.shape) == (py0, px0)
        assert img[py0, px0] == pytest.approx(ws, rel=1e-6)


def test_single_cell_shift_theorem():
    # One baseline on cell k0 with V = a + ib: the image is the closed form
    # 2 Re((a + ib) exp(2 pi i k0.(p - N/2) / N)).
    n_px = 24
    h = n_px // 2
    ku = np.array([5], np.int32)
    kv = np.array([-3], np.int32)
    V = np.array([0.75 - 0.5j], np.complex64)
    g, _, ws = oracle.grid(ku, kv, V, n_px, 0)
    p = np.arange(n_px) - h
    ref = 2 * np.real(complex(V[0]) * np.exp(2j * np.pi * (5 * p[None, :] - 3 * p[:, None]) / n_px))
    for f in (oracle.image_direct, oracle.image_fft):
        img, _ = f(g)
        assert np.abs(img - ref).max() < 1e-13
    assert ws == 2


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 12, 18, 49, 180, 256, 1024])
def test_fft1d_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    assert np.allclose(oracle.fft1d(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-11 * n)
    assert np.allclose(oracle.fft1d(x, -1), np.fft.fft(x), rtol=0, atol=1e-11 * n)


@pytest.mark.parametrize("n_px", [16, 18, 180, 256])
def test_image_fft_matches_numpy_shifted_ifft2(n_px):
    rng = np.random.default_rng(n_px)
    nb = 200
    ku = rng.integers(-(n_px // 2 - 1), n_px // 2, nb).astype(np.int32)
    kv = rng.integers(-(n_px // 2 - 1), n_px // 2, nb).astype(np.int32)
    vis = (rng.normal(size=nb) + 1j * rng.normal(size=nb)).astype(np.complex64)
    g, _, _ = oracle.grid(ku, kv, vis, n_px, 1)
    ref = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g))) * n_px * n_px
    img, mi = oracle.image_fft(g)
    peak = np.abs(ref).max()
    assert np.abs(img - ref.real).max() <= 1e-12 * peak
    assert np.abs(ref.imag).max() <= 1e-12 * peak and mi <= 1e-12 * peak
    if n_px <= 180:
        img_d, _ = oracle.image_direct(g)
        assert np.abs(img_d - ref.real).max() <= 1e-12 * peak


def test_parseval_and_linearity():
    n_px = 48
    rng = np.random.default_rng(41)
    xyz = int_array(16, -20, 21, 41)
    u, v = oracle.uv(xyz, NU_LAMBDA2)
    ku, kv = oracle.cells(u, v, 0.5, n_px)
    v1 = (rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)).astype(np.complex64)
    v2 = (rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)).astype(np.complex64)
    for w in (0, 1):
        g1, _, _ = oracle.grid(ku, kv, v1, n_px, w)
        g2, _, _ = oracle.grid(ku, kv, v2, n_px, w)
        i1, _ = oracle.image_fft(g1)
        i2, _ = oracle.image_fft(g2)
        # Parseval for the unnormalised inverse transform of a Hermitian grid
        assert (i1 ** 2).sum() == pytest.approx(n_px ** 2 * (np.abs(g1) ** 2).sum(), rel=1e-12)
        # linearity in the visibilities (weights depend only on the cells)
        a, b = 0.25, -1.5
        g12, _, _ = oracle.grid(ku, kv, (a * v1.astype(np.complex128) + b * v2).astype(
            np.complex64), n_px, w)
        i12, _ = oracle.image_fft(g12)
        # exact linearity up to the complex64 rounding of the combined input
        gref = a * g1 + b * g2
        assert np.abs(g12 - gref).max() <= 1e-6 * np.abs(gref).max() + 1e-12
        assert np.abs(i12 - (a * i1 + b * i2)).max() <= 1e-5 * np.abs(i12).max()


def test_batch_matches_single_layers():
    xyz = int_array(12, -10, 11, 51)
    rng = np.random.default_rng(52)
    nb = oracle.n_baselines(12)
    vis = (rng.normal(size=3 * nb) + 1j * rng.normal(size=3 * nb)).astype(np.complex64)
    layers = [dict(n_px=32, weighting=0, freq_hz=NU_LAMBDA2, delta_u=0.5, vis_offset=0),
              dict(n_px=16, weighting=1, freq_hz=1.1 * NU_LAMBDA2, delta_u=0.7, vis_offset=nb),
              dict(n_px=24, weighting=0, freq_hz=0.9 * NU_LAMBDA2, delta_u=0.4,
                   vis_offset=2 * nb)]
    imgs, ws = oracle.image_batch(xyz, layers, vis, "fft", n_threads=2)
    for k, L in enumerate(layers):
        img, w, _ = oracle.image(xyz, L["freq_hz"], L["delta_u"], L["n_px"], L["weighting"],
                                 vis[L["vis_offset"]:L["vis_offset"] + nb], "direct")
        assert ws[k] == w
        assert np.abs(imgs[k] - img).max() <= 1e-11 * max(1.0, np.abs(img).max())


def test_table3_operation_counts_golden():
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(HERE, "golden",
            "table3_operation_counts.txt")) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for n_ant, n_px, n_corr, n_grid, n_fft, n_tot in rows:
        assert oracle.n_baselines(n_ant) == n_corr == n_grid
        assert round(n_px * n_px * math.log2(n_px * n_px)) == n_fft
        assert n_corr + n_grid + n_fft == n_tot
