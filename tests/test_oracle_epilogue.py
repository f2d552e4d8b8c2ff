"""Pins of the oracle's fused-epilogue steps: antenna gains applied to the
visibilities (Sec. 4.2, calibration step ii) and a reference image subtracted
from the dirty image (Sec. 2; Sec. 4.3 after Eq. 6).

Each pin rests on something other than the oracle's own arithmetic: the
shift theorem (a gain phase ramp moves a point source to a known pixel with
a known peak), scaling (real gains c give c^2 times the image), a numpy
brute-force sum over baselines, and the linearity of the imager (subtracting
the image of W equals imaging V - W).
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import NU_LAMBDA2, direct_baseline_sum, int_array, tiny_case

LAM = 2.0  # metres at NU_LAMBDA2


def layers_for(n_px, du, weighting, n, nb):
    return [dict(n_px=n_px, weighting=weighting, freq_hz=NU_LAMBDA2, delta_u=du,
                 vis_offset=k * nb) for k in range(n)]


def test_unit_gains_are_the_identity():
    xyz = int_array(12, -20, 21, 3)
    nb = oracle.n_baselines(12)
    rng = np.random.default_rng(1)
    vis = (rng.normal(size=2 * nb) + 1j * rng.normal(size=2 * nb)).astype(np.complex64)
    lay = layers_for(48, 0.5, 1, 2, nb)
    plain, ws0 = oracle.image_batch(xyz, lay, vis)
    ones, ws1 = oracle.image_batch(xyz, lay, vis, gains=np.ones(12, np.complex128))
    for a, b in zip(plain, ones):
        assert np.array_equal(a, b)
    assert np.array_equal(ws0, ws1)


@pytest.mark.parametrize("weighting", [0, 1])
def test_phase_ramp_gains_move_a_source(weighting):
    # V = 1 (unit source at the phase centre).  Gains g_a = exp(2 pi i (x_a l0 +
    # y_a m0) / lambda) give g_i conj(g_j) = exp(-2 pi i (u l0 + v m0)): the
    # visibilities of a unit source at (l0, m0).  With on-grid cells and (l0, m0)
    # on a pixel, every term is in phase there: peak = summed weight.
    n_px, du = 32, 0.5
    xyz = int_array(10, -14, 15, 31)
    nb = oracle.n_baselines(10)
    px0, py0 = 22, 7
    l0 = (px0 - n_px // 2) / (n_px * du)
    m0 = (py0 - n_px // 2) / (n_px * du)
    g = np.exp(2j * np.pi * (xyz[:, 0] * l0 + xyz[:, 1] * m0) / LAM)
    vis = np.ones(nb, np.complex64)
    for mode in ("direct", "fft"):
        (img,), ws = oracle.image_batch(xyz, layers_for(n_px, du, weighting, 1, nb), vis, mode,
                                        gains=g)
        assert np.unravel_index(np.argmax(img), img.shape) == (py0, px0)
        assert img[py0, px0] == pytest.approx(ws[0], rel=1e-12)


@pytest.mark.parametrize("weighting", [0, 1])
def test_real_gains_scale_the_image(weighting):
    xyz = int_array(9, -12, 13, 8)
    nb = oracle.n_baselines(9)
    rng = np.random.default_rng(9)
    vis = (rng.normal(size=nb) + 1j * rng.normal(size=nb)).astype(np.complex64)
    lay = layers_for(32, 0.5, weighting, 1, nb)
    (plain,), _ = oracle.image_batch(xyz, lay, vis)
    (scaled,), _ = oracle.image_batch(xyz, lay, vis, gains=np.full(9, 1.5 + 0j))
    assert np.abs(scaled - 2.25 * plain).max() <= 1e-12 * np.abs(plain).max()


@pytest.mark.parametrize("weighting", [0, 1])
def test_gains_match_bruteforce_direct_sum(weighting):
    n_px, du = 16, 0.5
    xyz, u, v, ku, kv = tiny_case(6, n_px, 21)
    rng = np.random.default_rng(23)
    vis = (rng.normal(size=ku.size) + 1j * rng.normal(size=ku.size)).astype(np.complex64)
    g = rng.normal(1.0, 0.2, 6) * np.exp(1j * rng.uniform(-np.pi, np.pi, 6))
    # brute force: pair list, product, direct sum over baselines
    pairs = [(i, j) for i in range(6) for j in range(i + 1, 6)]
    vg = np.array([g[i] * np.conj(g[j]) * complex(vis[b]) for b, (i, j) in enumerate(pairs)])
    keep = ku != oracle.DROPPED
    if weighting == 0:
        w = keep.astype(float)
    else:
        h = n_px // 2
        cnt = {}
        for a, c in zip(ku[keep], kv[keep]):
            cnt[(c + h, a + h)] = cnt.get((c + h, a + h), 0) + 1
            cnt[(h - c, h - a)] = cnt.get((h - c, h - a), 0) + 1
        w = np.array([1.0 / cnt[(c + h, a + h)] if a != oracle.DROPPED else 0.0
                      for a, c in zip(ku, kv)])
    want = direct_baseline_sum(u, v, vg, w, du, n_px)
    for mode in ("direct", "fft"):
        (img,), _ = oracle.image_batch(xyz, layers_for(n_px, du, weighting, 1, ku.size), vis,
                                       mode, gains=g)
        assert np.abs(img - want).max() <= 1e-12 * np.abs(want).max()


def test_gain_rows_follow_the_stride():
    xyz = int_array(8, -10, 11, 14)
    nb = oracle.n_baselines(8)
    rng = np.random.default_rng(14)
    vis = (rng.normal(size=3 * nb) + 1j * rng.normal(size=3 * nb)).astype(np.complex64)
    rows = np.exp(1j * rng.uniform(-np.pi, np.pi, (3, 8))) * rng.uniform(0.5, 1.5, (3, 8))
    lay = layers_for(32, 0.5, 0, 3, nb)
    together, _ = oracle.image_batch(xyz, lay, vis, gains=rows.reshape(-1), gain_stride=8)
    for k in range(3):
        (alone,), _ = oracle.image_batch(xyz, [dict(lay[k], vis_offset=0)],
                                         vis[k * nb:(k + 1) * nb], gains=rows[k])
        assert np.array_equal(together[k], alone)
    shared, _ = oracle.image_batch(xyz, lay, vis, gains=rows[0], gain_stride=0)
    (first,), _ = oracle.image_batch(xyz, [dict(lay[2], vis_offset=0)], vis[2 * nb:],
                                     gains=rows[0])
    assert np.array_equal(shared[2], first)
    # period 2: layer 2 wraps around to row 0 (all three rows passed, so a
    # wrong row index reads valid memory)
    per, _ = oracle.image_batch(xyz, lay, vis, gains=rows.reshape(-1), gain_stride=8,
                                gain_period=2)
    assert np.array_equal(per[2], first)
    assert np.array_equal(per[1], together[1])


def test_reference_subtraction_is_dirty_minus_reference():
    # linearity: image(V) - image(W) == image(V - W); subtracting the image of
    # the visibilities themselves leaves exactly zero
    xyz = int_array(11, -16, 17, 5)
    nb = oracle.n_baselines(11)
    rng = np.random.default_rng(6)
    V = (rng.normal(size=2 * nb) + 1j * rng.normal(size=2 * nb)).astype(np.complex64)
    W = (rng.normal(size=2 * nb) + 1j * rng.normal(size=2 * nb)).astype(np.complex64)
    lay = [dict(n_px=n, weighting=1, freq_hz=NU_LAMBDA2, delta_u=0.5, vis_offset=k * nb)
           for k, n in enumerate((32, 48))]
    img_w, _ = oracle.image_batch(xyz, lay, W)
    img_v, _ = oracle.image_batch(xyz, lay, V)
    ref = np.concatenate([x.reshape(-1) for x in img_w])
    diff, ws = oracle.image_batch(xyz, lay, V, ref=ref)
    direct, _ = oracle.image_batch(xyz, lay, V - W)
    for d, a, v_ in zip(diff, direct, img_v):
        assert np.abs(d - a).max() <= 1e-6 * np.abs(v_).max()   # V - W rounded to complex64
    self_ref = np.concatenate([x.reshape(-1) for x in img_v])
    zero, _ = oracle.image_batch(xyz, lay, V, ref=self_ref)
    assert all(not z.any() for z in zero)
    none, _ = oracle.image_batch(xyz, lay, V, ref=np.zeros_like(self_ref))
    for a, b in zip(none, img_v):
        assert np.array_equal(a, b)


def test_reference_linearity_exact_in_fp64():
    # the same linearity with W = V / 2 exactly representable in complex64:
    # image(V) - image(W) == image(W) to FP64 rounding
    xyz = int_array(7, -9, 10, 2)
    nb = oracle.n_baselines(7)
    rng = np.random.default_rng(2)
    V = (rng.normal(size=nb) + 1j * rng.normal(size=nb)).astype(np.complex64)
    W = (V / 2).astype(np.complex64)
    lay = layers_for(24, 0.5, 0, 1, nb)
    (iw,), _ = oracle.image_batch(xyz, lay, W)
    (d,), _ = oracle.image_batch(xyz, lay, V, ref=iw.reshape(-1))
    assert np.abs(d - iw).max() <= 1e-12 * np.abs(iw).max()


def test_apply_gains_matches_pairwise_product():
    rng = np.random.default_rng(4)
    n = 7
    g = rng.normal(size=n) + 1j * rng.normal(size=n)
    vis = (rng.normal(size=n * (n - 1) // 2) + 1j * rng.normal(size=n * (n - 1) // 2))
    vis = vis.astype(np.complex64)
    got = oracle.apply_gains(n, g, vis)
    b = 0
    for i in range(n):
        for j in range(i + 1, n):
            assert got[b] == pytest.approx(g[i] * np.conj(g[j]) * complex(vis[b]), rel=1e-15)
            b += 1
