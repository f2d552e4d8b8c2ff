"""Pins of the oracle's adjoint (gradients of an image loss).

The adjoint is checked against things that do not use its derivation:
FP64 central finite differences of the oracle's forward image, the
dot-product identity of a linear map and its adjoint, and numpy.fft.
"""
import numpy as np
import pytest

import oracle

NU = oracle.C_LIGHT / 2.0  # lambda = 2 m


def small_array(n_ant, seed, span=9.0):
    rng = np.random.default_rng(seed)
    xyz = np.zeros((n_ant, 3))
    xyz[:, :2] = rng.uniform(-span, span, (n_ant, 2))
    return xyz


def forward64(ku, kv, vis, n_px, weighting):
    g, _, _ = oracle.grid_c128(ku, kv, vis, n_px, weighting)
    img, _ = oracle.image_fft(g)
    return img


def lattice_array(n_side, step=2.0):
    """Antennas on a square lattice: many baselines share a cell (redundancy)."""
    g = np.arange(n_side) * step
    xyz = np.zeros((n_side * n_side, 3))
    xyz[:, 0] = np.repeat(g, n_side)
    xyz[:, 1] = np.tile(g, n_side)
    return xyz


def case(n_ant=7, n_px=24, seed=1, du=0.45, redundant=False):
    xyz = lattice_array(3) if redundant else small_array(n_ant, seed)
    u, v = oracle.uv(xyz, NU)
    ku, kv = oracle.cells(u, v, du, n_px)
    rng = np.random.default_rng(seed + 100)
    vis = rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)
    return ku, kv, vis, rng


@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("mode", ["direct", "fft"])
def test_adjoint_dot_product_identity(weighting, mode):
    ku, kv, vis, rng = case(seed=2, redundant=weighting == 1, du=0.9 if weighting else 0.45)
    if weighting == 0:
        assert (ku == oracle.DROPPED).any()  # dropped baselines get a zero gradient
    n_px = 24
    img = forward64(ku, kv, vis, n_px, weighting)
    r = rng.normal(size=(n_px, n_px))
    gam = oracle.degrid(ku, kv, r, weighting, mode)
    lhs = (r * img).sum()
    rhs = np.real(vis * np.conj(gam)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-11)
    assert not gam[ku == oracle.DROPPED].any()


@pytest.mark.parametrize("weighting", [0, 1])
def test_degrid_routes_agree_and_match_numpy(weighting):
    ku, kv, _, rng = case(n_ant=9, n_px=20, seed=3, du=0.6)
    n_px = 20
    r = rng.normal(size=(n_px, n_px))
    a = oracle.degrid(ku, kv, r, weighting, "direct")
    b = oracle.degrid(ku, kv, r, weighting, "fft")
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()
    # H = forward FFT of the shifted residual, read at each baseline's cell
    H = np.fft.fft2(np.fft.ifftshift(r))
    keep = ku != oracle.DROPPED
    _, cnt, _ = oracle.grid(ku, kv, np.ones(ku.size, np.complex64), n_px, weighting)
    w = np.ones(ku.size)
    if weighting == 1:
        w = np.array([1.0 / cnt[c + n_px // 2, a_ + n_px // 2] if a_ != oracle.DROPPED else 0.0
                      for a_, c in zip(ku, kv)])
    want = np.where(keep, 2 * w * H[np.where(keep, kv, 0) % n_px, np.where(keep, ku, 0) % n_px], 0)
    assert np.abs(b - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("weighting", [0, 1])
def test_visibility_gradient_matches_finite_differences(weighting):
    n_px = 16
    ku, kv, vis, rng = case(n_ant=6, n_px=n_px, seed=4, du=0.8, redundant=weighting == 1)
    if weighting == 1:  # shared cells, so uniform weights differ from 1
        _, cnt, _ = oracle.grid(ku, kv, np.ones(ku.size, np.complex64), n_px, 1)
        assert cnt.max() >= 3
    target = rng.normal(size=(n_px, n_px))

    def loss(v):
        return ((forward64(ku, kv, v, n_px, weighting) - target) ** 2).sum()

    img = forward64(ku, kv, vis, n_px, weighting)
    gam = oracle.degrid(ku, kv, 2 * (img - target), weighting, "fft")
    h = 1e-6
    for b in rng.choice(np.nonzero(ku != oracle.DROPPED)[0], 6, replace=False):
        for part, unit in ((0, 1.0), (1, 1j)):
            vp, vm = vis.copy(), vis.copy()
            vp[b] += h * unit
            vm[b] -= h * unit
            fd = (loss(vp) - loss(vm)) / (2 * h)
            an = gam[b].real if part == 0 else gam[b].imag
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-6 * np.abs(gam).max())


def test_gain_gradient_matches_finite_differences():
    # V_ij = g_i conj(g_j) M_ij; loss = sum (image - model image)^2 (station-gains form)
    n_px, n_ant = 16, 8
    xyz = small_array(n_ant, 5)
    u, v = oracle.uv(xyz, NU)
    ku, kv = oracle.cells(u, v, 0.8, n_px)
    rng = np.random.default_rng(6)
    model = rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)
    gains = np.abs(rng.normal(1.0, 0.1, n_ant)) * np.exp(1j * rng.uniform(-np.pi, np.pi, n_ant))
    i, j = np.triu_indices(n_ant, 1)
    target = forward64(ku, kv, model, n_px, 0)

    def loss(g):
        return ((forward64(ku, kv, g[i] * np.conj(g[j]) * model, n_px, 0) - target) ** 2).sum()

    vis = gains[i] * np.conj(gains[j]) * model
    img = forward64(ku, kv, vis, n_px, 0)
    gam_v = oracle.degrid(ku, kv, 2 * (img - target), 0, "fft")
    gam_g = oracle.gain_grad(n_ant, gam_v, gains, model)
    h = 1e-6
    for a in range(n_ant):  # 16 perturbed gain components (real and imaginary parts)
        for unit in (1.0, 1j):
            gp, gm = gains.copy(), gains.copy()
            gp[a] += h * unit
            gm[a] -= h * unit
            fd = (loss(gp) - loss(gm)) / (2 * h)
            an = gam_g[a].real if unit == 1.0 else gam_g[a].imag
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-6 * np.abs(gam_g).max())
