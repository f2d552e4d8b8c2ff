"""GPU fused epilogue (gains applied at gridding, reference image subtracted at
the store) against the FP64 oracle, on every kernel path.

Bar: the output is dirty - ref, and the FP32 error lives in the dirty image,
so max |gpu - oracle| <= tol * (max |oracle| + max |ref|) per layer, with
tol = 1e-5 for the FP32 paths and the mode's bound for the tensor-core path
(max |dirty| <= max |dirty - ref| + max |ref|).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_2405_13478_gb300 import binding, build
    build.build()
    c = binding.Context(0)
    yield c
    c.close()


def split(flat, layers):
    return [flat[L["out_offset"]:L["out_offset"] + L["n_px"] ** 2].reshape(L["n_px"], L["n_px"])
            for L in layers]


def check(got_flat, want, ref_flat, layers, tol=TOL, what=""):
    for k, (g, w, r) in enumerate(zip(split(got_flat, layers), want, split(ref_flat, layers))):
        bound = tol * (np.abs(w).max() + np.abs(r).max())
        err = np.abs(g.astype(np.float64) - w).max()
        assert np.isfinite(g).all(), f"{what} layer {k}: non-finite"
        assert err <= bound, f"{what} layer {k}: err {err:.3e} > {bound:.3e}"


def station_case(seed, sizes, weighting=1):
    ws = synth.station_batch(seed=seed, n_times=1)
    nb = ws.n_baselines
    layers = []
    for k, n in enumerate(sizes):
        f = float(ws.freqs_hz[(5 * k) % 32])
        layers.append(dict(n_px=n, weighting=weighting, freq_hz=f, delta_u=0.5,
                           vis_offset=k * nb))
    vis = synth.noise((len(sizes) * nb,), 1.0, seed, "cpu")
    return ws, layers, vis


def gain_rows(n_rows, n_ant, seed):
    rng = np.random.default_rng(seed)
    g = np.abs(rng.normal(1.0, 0.1, (n_rows, n_ant))) * np.exp(1j * rng.uniform(-np.pi, np.pi,
                                                                              (n_rows, n_ant)))
    return g.astype(np.complex64)


def run(torch, ctx, ws, layers, vis, gains, stride, ref, flags=0, path=None):
    from paper_2405_13478_gb300 import binding
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    if path is not None:
        for g in range(len(plan.tuning())):
            try:
                plan.set_tuning(g, path)
            except binding.BlinkError:
                pass  # the group cannot take this path (shared memory); keep its default
    out = torch.full((total,), float("nan"), device="cuda")
    d_ref = None if ref is None else torch.as_tensor(ref).cuda()
    d_g = None if gains is None else torch.as_tensor(gains.reshape(-1)).cuda()
    plan.image(vis.reshape(-1).cuda(), out, flags=flags, gains=d_g, gain_stride=stride, ref=d_ref)
    torch.cuda.synchronize()
    plan.check()
    plan.close()
    return layers, total, out.cpu().numpy()


@pytest.mark.parametrize("path", [None, 1, 2, 3])
def test_gains_and_reference_every_small_path(torch, ctx, path):
    sizes = [64, 128, 180, 256]
    ws, layers, vis = station_case(31, sizes)
    from paper_2405_13478_gb300 import binding
    lay, total = binding.layer_out_offsets(layers)
    g = gain_rows(len(sizes), ws.n_ant, 5)
    ref = np.random.default_rng(7).normal(0, 50.0, total).astype(np.float32)
    lay, total, got = run(torch, ctx, ws, layers, vis, g, ws.n_ant, ref, path=path)
    want, _ = oracle.image_batch(ws.ant_xyz, lay, vis.numpy(), gains=g.astype(np.complex128),
                                 gain_stride=ws.n_ant, ref=ref.astype(np.float64))
    check(got, want, ref, lay, what=f"path {path}")


def test_gains_and_reference_large_sizes(torch, ctx):
    """Two-kernel path (512, 1024); shared gains (stride 0), natural weighting."""
    flags = 0
    from paper_2405_13478_gb300 import binding
    ws = synth.uneven_batch(seed=12, n_times=30)
    chans = [200, 300, 210]   # 512, 1024, 512
    vis = ws.vis("cpu", times=[20])[0, chans, :].contiguous()
    layers = [dict(n_px=int(ws.n_px[c]), weighting=0, freq_hz=float(ws.freqs_hz[c]),
                   delta_u=float(ws.delta_u[c]), vis_offset=k * ws.n_baselines)
              for k, c in enumerate(chans)]
    lay, total = binding.layer_out_offsets(layers)
    g = gain_rows(1, ws.n_ant, 9)
    ref = np.random.default_rng(8).normal(0, 20.0, total).astype(np.float32)
    lay, total, got = run(torch, ctx, ws, layers, vis, g, 0, ref, flags=flags)
    want, _ = oracle.image_batch(ws.ant_xyz, lay, vis.reshape(-1).numpy(),
                                 gains=g.reshape(-1).astype(np.complex128), gain_stride=0,
                                 ref=ref.astype(np.float64))
    check(got, want, ref, lay, tol=TOL, what=f"flags {flags:#x}")


def test_normalised_image_minus_reference(torch, ctx):
    ws, layers, vis = station_case(33, [180, 180])
    from paper_2405_13478_gb300 import binding
    lay, total = binding.layer_out_offsets(layers)
    ref = np.random.default_rng(3).normal(0, 1e-3, total).astype(np.float32)
    lay, total, got = run(torch, ctx, ws, layers, vis, None, 0, ref, flags=1)
    dirty, wsum = oracle.image_batch(ws.ant_xyz, lay, vis.numpy())
    want = [d / s - r for d, s, r in zip(dirty, wsum, split(ref.astype(np.float64), lay))]
    check(got, want, ref, lay)


def test_unit_gains_are_bit_identical_on_the_scheduled_path(torch, ctx):
    ws, layers, vis = station_case(34, [180, 128])
    ones = np.ones((1, ws.n_ant), np.complex64)
    _, _, plain = run(torch, ctx, ws, layers, vis, None, 0, None, path=1)
    _, _, gained = run(torch, ctx, ws, layers, vis, ones, 0, None, path=1)
    assert np.array_equal(plain, gained)


def test_reference_overlapping_the_output_is_rejected(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws, layers, vis = station_case(35, [128, 256])
    lay, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), lay)
    d_vis = vis.cuda()
    out = torch.empty(total, device="cuda")
    big = torch.zeros(total + 64, device="cuda")
    for o, r in ((out, out), (big[:total], big[32:32 + total]), (big[32:32 + total], big[:total])):
        with pytest.raises(binding.BlinkError) as ei:
            plan.image(d_vis, o, ref=r)
        assert ei.value.status == binding.ERR_INVALID
    with pytest.raises(binding.BlinkError) as ei:
        plan.image(d_vis, out, gains=torch.ones(ws.n_ant, dtype=torch.complex64, device="cuda"),
                   gain_stride=-1)
    assert ei.value.status == binding.ERR_INVALID
    # adjacent, non-overlapping buffers are fine
    both = torch.zeros(2 * total, device="cuda")
    both[total:] = torch.randn(total, generator=torch.Generator().manual_seed(1)).cuda()
    plan.image(d_vis, both[:total], ref=both[total:])
    torch.cuda.synchronize()
    want, _ = oracle.image_batch(ws.ant_xyz, lay, vis.numpy(),
                                 ref=both[total:].cpu().double().numpy())
    check(both[:total].cpu().numpy(), want, both[total:].cpu().numpy(), lay)
    plan.close()


def test_graph_replay_with_epilogue_tracks_new_reference(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws, layers, vis = station_case(36, [180, 256, 180])
    lay, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), lay)
    g = gain_rows(3, ws.n_ant, 4)
    d_g = torch.as_tensor(g.reshape(-1)).cuda()
    d_ref = torch.zeros(total, device="cuda")
    out = torch.empty(total, device="cuda")
    d_vis = vis.cuda()
    plan.capture(d_vis, out, gains=d_g, gain_stride=ws.n_ant, ref=d_ref)
    for seed in (1, 2):
        r = np.random.default_rng(seed).normal(0, 30.0, total).astype(np.float32)
        d_ref.copy_(torch.as_tensor(r))
        out.fill_(float("nan"))
        plan.replay()
        torch.cuda.synchronize()
        want, _ = oracle.image_batch(ws.ant_xyz, lay, vis.numpy(), gains=g.astype(np.complex128),
                                     gain_stride=ws.n_ant, ref=r.astype(np.float64))
        check(out.cpu().numpy(), want, r, lay, what=f"replay {seed}")
    plan.close()


@pytest.mark.parametrize("flags,tol", [(0x20, 1e-5), (0x30, 1e-3)])
def test_gains_and_reference_tensor_core_transform(torch, ctx, flags, tol):
    """Station 512^2 layers through the DFT-GEMM (BF16x3, FP16): the reference
    is subtracted in the TMEM epilogue, the gains in the row pass."""
    from paper_2405_13478_gb300 import binding
    ws = synth.station_512(seed=5, n_times=1)
    chans = [0, 9, 15]
    vis = ws.vis("cpu", times=[0])[0, chans, :].contiguous()
    layers = [dict(n_px=512, weighting=0, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=k * ws.n_baselines) for k, c in enumerate(chans)]
    lay, total = binding.layer_out_offsets(layers)
    g = gain_rows(3, ws.n_ant, 10)
    ref = np.random.default_rng(10).normal(0, 5.0, total).astype(np.float32)
    lay, total, got = run(torch, ctx, ws, layers, vis, g, ws.n_ant, ref, flags=flags)
    want, _ = oracle.image_batch(ws.ant_xyz, lay, vis.reshape(-1).numpy(),
                                 gains=g.astype(np.complex128), gain_stride=ws.n_ant,
                                 ref=ref.astype(np.float64))
    check(got, want, ref, lay, tol=tol, what=f"flags {flags:#x}")


def test_per_channel_gains_with_period(torch, ctx):
    """Time-major layers (2 steps x 3 channels) with one gain row per channel:
    gain_period = 3 wraps the rows over the time steps."""
    from paper_2405_13478_gb300 import binding
    ws = synth.station_batch(seed=37, n_times=2)
    chans = [0, 11, 31]
    vis = ws.vis("cpu", times=[0, 1])[:, chans, :].contiguous().reshape(-1)
    layers = [dict(n_px=180, weighting=1, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=(t * 3 + k) * ws.n_baselines)
              for t in range(2) for k, c in enumerate(chans)]
    lay, total = binding.layer_out_offsets(layers)
    g = gain_rows(3, ws.n_ant, 12)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), lay)
    out = torch.empty(total, device="cuda")
    plan.image(vis.cuda(), out, gains=torch.as_tensor(g.reshape(-1)).cuda(),
               gain_stride=ws.n_ant, gain_period=3)
    torch.cuda.synchronize()
    plan.close()
    want, _ = oracle.image_batch(ws.ant_xyz, lay, vis.numpy(), gains=g.astype(np.complex128),
                                 gain_stride=ws.n_ant, gain_period=3)
    check(out.cpu().numpy(), want, np.zeros(total, np.float32), lay)


@pytest.mark.parametrize("path", [None, 1, 2, 3])
def test_gains_without_product_table_large_array(torch, ctx, path):
    """2048 antennas (2,096,128 baselines) with one gain row per layer: the
    gain-product table (20 rows x B x 8 bytes = 335 MB) exceeds its cap, so
    every kernel forms g_i conj(g_j) from the antenna gains itself; this also
    runs the baseline -> antenna-pair map at a large n on the GPU."""
    from paper_2405_13478_gb300 import binding
    n_ant, n_lay, n_px = 2048, 20, 64
    xyz = synth.antennas_disk(n_ant, 38.0, 41)
    nb = n_ant * (n_ant - 1) // 2
    freqs = np.linspace(150e6, 180e6, n_lay)
    du = synth.max_uv(xyz, freqs[-1]) / (n_px / 2 - 1)
    layers = [dict(n_px=n_px, weighting=k % 2, freq_hz=float(f), delta_u=du, vis_offset=k * nb)
              for k, f in enumerate(freqs)]
    lay, total = binding.layer_out_offsets(layers)
    vis = synth.noise((n_lay * nb,), 1.0, 42, "cpu")
    g = gain_rows(n_lay, n_ant, 43)
    array = type("Array", (), {"ant_xyz": xyz})()
    lay, total, got = run(torch, ctx, array, layers, vis, g, n_ant, None, path=path)
    want, _ = oracle.image_batch(xyz, lay, vis.numpy(), gains=g.astype(np.complex128),
                                 gain_stride=n_ant)
    check(got, want, np.zeros(total, np.float32), lay, what=f"path {path}")
