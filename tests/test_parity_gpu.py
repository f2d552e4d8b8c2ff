"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: cell indices bit-exact; grid cells within the FP32 summation bound; FP32 images
within 1e-5 of the oracle image's peak (max |gpu - oracle| / max |oracle|),
per layer.  Inputs come from synth.py only; expected values from oracle/ only.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


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


def to_dev(torch, a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def gpu_images(torch, ctx, xyz, layers, vis_cpu, flags=0):
    from paper_2405_13478_gb300 import binding
    layers, total = binding.layer_out_offsets(layers)
    d_xyz = to_dev(torch, xyz)
    d_vis = vis_cpu.reshape(-1).cuda()
    out = torch.full((max(total, 1),), float("nan"), dtype=torch.float32, device="cuda")
    ws = torch.zeros(max(len(layers), 1), dtype=torch.float32, device="cuda")
    ctx.image_batch(d_xyz, layers, d_vis, out, ws, flags)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    imgs = [o[L["out_offset"]:L["out_offset"] + L["n_px"] ** 2].reshape(L["n_px"], L["n_px"])
            for L in layers]
    return imgs, ws.cpu().numpy()[:len(layers)]


def oracle_images(xyz, layers, vis_cpu):
    vis = vis_cpu.reshape(-1).numpy()
    return oracle.image_batch(xyz, layers, vis, "fft")


def assert_images_close(got, want, tol=IMG_TOL, what=""):
    for k, (g, w) in enumerate(zip(got, want)):
        peak = np.abs(w).max()
        err = np.abs(g.astype(np.float64) - w).max()
        assert np.isfinite(g).all(), f"{what} layer {k}: non-finite output"
        assert err <= tol * peak, f"{what} layer {k}: max err {err:.3e} vs peak {peak:.3e}"


def ws_sub(ws: synth.Workload, times, chans):
    """Layers and a compact vis tensor for a (times x chans) slice."""
    vis = ws.vis("cpu", times=times)[:, chans, :]  # [T'][C'][B]
    layers = ws.layers(times=range(len(times)), chans=range(len(chans)))
    for L, (t, c) in zip(layers, [(t, c) for t in range(len(times)) for c in range(len(chans))]):
        ch = chans[c]
        L.update(n_px=int(ws.n_px[ch]), freq_hz=float(ws.freqs_hz[ch]),
                 delta_u=float(ws.delta_u[ch]), vis_offset=(t * len(chans) + c) * ws.n_baselines)
    return layers, vis.contiguous()


# ------------------------------------------------------ uv and cells
def gpu_cells(torch, ctx, xyz, layers, nb):
    d = torch.empty((len(layers), nb, 2), dtype=torch.int32, device="cuda")
    ctx.cells(to_dev(torch, xyz), layers, d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("seed,name", list(enumerate(synth.WORKLOADS, start=1)))
def test_cells_bit_exact_on_every_workload(torch, ctx, seed, name):
    ws = synth.WORKLOADS[name](seed=seed)
    chans = sorted(set([0, ws.n_chan // 2, ws.n_chan - 1] + list(range(0, ws.n_chan, 97))))
    layers = [dict(n_px=int(ws.n_px[c]), weighting=ws.weighting, freq_hz=float(ws.freqs_hz[c]),
                   delta_u=float(ws.delta_u[c]), vis_offset=0) for c in chans]
    got = gpu_cells(torch, ctx, ws.ant_xyz, layers, ws.n_baselines)
    for k, L in enumerate(layers):
        u, v = oracle.uv(ws.ant_xyz, L["freq_hz"])
        ku, kv = oracle.cells(u, v, L["delta_u"], L["n_px"])
        assert np.array_equal(got[k, :, 0], ku) and np.array_equal(got[k, :, 1], kv), (name, k)


def test_cells_ties_and_edges_bit_exact(torch, ctx):
    # lambda = 2 m: integer positions put u / delta_u exactly on integers and
    # half-integers, and on the kept/dropped edge.
    nu = oracle.C_LIGHT / 2.0
    xs = np.arange(-13, 14, dtype=np.float64)
    xyz = np.zeros((xs.size, 3))
    xyz[:, 0] = xs
    xyz[:, 1] = -0.5 * xs
    layers = [dict(n_px=n, weighting=0, freq_hz=nu, delta_u=du, vis_offset=0)
              for n in (16, 20, 24) for du in (0.5, 1.0, 1.5)]
    nb = oracle.n_baselines(xs.size)
    got = gpu_cells(torch, ctx, xyz, layers, nb)
    dropped = kept = 0
    for k, L in enumerate(layers):
        u, v = oracle.uv(xyz, nu)
        ku, kv = oracle.cells(u, v, L["delta_u"], L["n_px"])
        assert np.array_equal(got[k, :, 0], ku) and np.array_equal(got[k, :, 1], kv)
        dropped += int((ku == oracle.DROPPED).sum())
        kept += int((ku != oracle.DROPPED).sum())
    assert dropped > 0 and kept > 0  # both sides of the edge rule were exercised


# -------------------------------------------------- grid and weights
def gpu_grids(torch, ctx, xyz, layers, vis_cpu):
    out_layers, off = [], 0
    for L in layers:
        L = dict(L)
        L["out_offset"] = off
        off += L["n_px"] ** 2
        out_layers.append(L)
    g = torch.zeros(2 * off, dtype=torch.float32, device="cuda")
    w = torch.zeros(len(layers), dtype=torch.float32, device="cuda")
    ctx.grid(to_dev(torch, xyz), out_layers, vis_cpu.reshape(-1).cuda(), g, w)
    torch.cuda.synchronize()
    gc = g.cpu().numpy().view(np.complex64)
    return [gc[L["out_offset"]:L["out_offset"] + L["n_px"] ** 2].reshape(L["n_px"], L["n_px"])
            for L in out_layers], w.cpu().numpy()


@pytest.mark.parametrize("weighting", [0, 1])
@pytest.mark.parametrize("n_px", [16, 180, 256])
def test_grid_matches_oracle(torch, ctx, weighting, n_px):
    # Tolerance from the arithmetic: a cell is an FP32 sum of n entries in
    # some order, so |error| <= (n - 1) u sum|V| (u = 2^-24) before the
    # weight, plus one rounding for the weight and one for the origin doubling.
    if n_px == 256:
        ws, times, chans = synth.single_image(seed=3), [0], [0]
    else:
        ws, times, chans = synth.station_batch(seed=3, n_times=2), [0, 1], [0, 31]
    ws.weighting = weighting
    ws.n_px = np.full(ws.n_chan, n_px)
    if n_px == 16:
        ws.delta_u = np.full(ws.n_chan, 4.0)  # ~300 entries per cell, some baselines dropped
    layers, vis = ws_sub(ws, times, chans)
    got, wsum = gpu_grids(torch, ctx, ws.ant_xyz, layers, vis)
    v = vis.reshape(-1).numpy()
    for k, L in enumerate(layers):
        u, vv = oracle.uv(ws.ant_xyz, L["freq_hz"])
        ku, kv = oracle.cells(u, vv, L["delta_u"], L["n_px"])
        vk = v[L["vis_offset"]:L["vis_offset"] + ws.n_baselines]
        g, cnt, w = oracle.grid(ku, kv, vk, L["n_px"], L["weighting"])
        gabs, _, _ = oracle.grid(ku, kv, np.abs(vk).astype(np.complex64), L["n_px"],
                                 L["weighting"])
        bound = (cnt + 2) * 2.0 ** -24 * np.abs(gabs) + 1e-30
        assert wsum[k] == pytest.approx(w, rel=1e-7)
        assert np.all(np.abs(got[k] - g) <= bound), (n_px, weighting, k)
        assert np.abs(got[k] - g).max() <= 1e-5 * np.abs(g).max()


# ------------------------------------------------------------------- images
@pytest.mark.parametrize("n_px", [16, 32, 64, 128, 180, 192, 256, 360, 512, 1024])
@pytest.mark.parametrize("weighting", [0, 1])
def test_images_match_oracle_across_sizes(torch, ctx, n_px, weighting):
    # A 3 km array with the cell size filling the grid: every support row is
    # populated, so both the fused path (small N) and the row/column path
    # (large N) run with several tiles and ragged tails.
    ws = synth.single_image(seed=n_px)
    ws.weighting = weighting
    ws.n_px = np.array([n_px])
    ws.delta_u = np.array([synth.max_uv(ws.ant_xyz, ws.freqs_hz[0]) / (n_px / 2 - 1)])
    layers, vis = ws_sub(ws, [0], [0])
    got, wsum = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    want, wref = oracle_images(ws.ant_xyz, layers, vis)
    assert_images_close(got, want, what=f"N={n_px} w={weighting}")
    assert np.allclose(wsum, wref, rtol=1e-7)


def test_station_batch_slice_uniform_180(torch, ctx):
    ws = synth.station_batch(seed=11, n_times=3)
    layers, vis = ws_sub(ws, [0, 2], list(range(32)))
    got, wsum = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    want, wref = oracle_images(ws.ant_xyz, layers, vis)
    assert_images_close(got, want, what="station")
    assert np.allclose(wsum, wref, rtol=1e-7)


def test_single_image_single_256(torch, ctx):
    ws = synth.single_image(seed=0)
    layers, vis = ws_sub(ws, [0], [0])
    got, _ = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    want, _ = oracle_images(ws.ant_xyz, layers, vis)
    assert_images_close(got, want, what="single")


def test_uneven_batch_mixed_sizes_in_one_call(torch, ctx):
    ws = synth.uneven_batch(seed=5, n_times=30)
    chans = [0, 100, 200, 300, 767]          # sizes 128, 256, 512, 1024, 1024
    layers, vis = ws_sub(ws, [20, 25], chans)
    got, _ = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    want, _ = oracle_images(ws.ant_xyz, layers, vis)
    assert_images_close(got, want, what="uneven")


def test_station_512_station_512(torch, ctx):
    ws = synth.station_512(seed=7, n_times=2)
    layers, vis = ws_sub(ws, [1], [0, 15])
    got, _ = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    want, _ = oracle_images(ws.ant_xyz, layers, vis)
    assert_images_close(got, want, what="station512")


def test_station_gains_station_1024_gains(torch, ctx):
    ws = synth.station_gains(seed=9, n_times=1)
    layers, vis = ws_sub(ws, [0], [3])
    got, _ = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    want, _ = oracle_images(ws.ant_xyz, layers, vis)
    assert_images_close(got, want, what="gains")


# ----------------------------------------------------------- edge cases
@pytest.mark.parametrize("weighting", [0, 1])
def test_unit_source_at_centre_gives_summed_weight_on_gpu(torch, ctx, weighting):
    ws = synth.station_batch(seed=2, n_times=1)
    B = ws.n_baselines
    layers = [dict(n_px=180, weighting=weighting, freq_hz=float(f), delta_u=0.5,
                   vis_offset=k * B) for k, f in enumerate(ws.freqs_hz[:4])]
    import torch as t
    vis = t.ones((4, B), dtype=t.complex64)
    got, wsum = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    for g, w in zip(got, wsum):
        assert g[90, 90] == pytest.approx(w, rel=2e-6)
        assert g.max() == pytest.approx(w, rel=2e-6)


def test_ragged_baselines_and_unaligned_offsets(torch, ctx):
    # 7 antennas -> 21 baselines; layers start at odd complex offsets
    rng = np.random.default_rng(4)
    xyz = np.zeros((7, 3))
    xyz[:, :2] = rng.uniform(-20, 20, (7, 2))
    B = 21
    vis = synth.noise((5 * B + 3,), 1.0, 41, "cpu")
    layers = [dict(n_px=n, weighting=w, freq_hz=1.5e8, delta_u=0.6, vis_offset=off)
              for n, w, off in ((16, 0, 1), (32, 1, B + 2), (180, 0, 3 * B + 3), (256, 1, 2 * B))]
    got, _ = gpu_images(torch, ctx, xyz, layers, vis)
    want, _ = oracle_images(xyz, layers, vis)
    assert_images_close(got, want, what="ragged")


@pytest.mark.parametrize("weighting", [0, 1])
def test_redundant_grid_array_long_schedule_blocks(torch, ctx, weighting):
    # A 12 x 12 grid of antennas at 2 m: 10296 baselines in two staging
    # chunks, the shortest spacings repeat up to 132 times, so a schedule
    # block can exceed the bank-ordered length and a cell's peak exceeds the
    # ranking's last bucket.  Images against the oracle, bits across plans.
    xyz = synth.antennas_grid(12, 2.0)
    nb = 144 * 143 // 2
    chans = (150e6, 165e6, 180e6)
    layers = [dict(n_px=n, weighting=weighting, freq_hz=f, delta_u=0.5, vis_offset=k * nb)
              for k, (n, f) in enumerate(zip((128, 180, 256), chans))]
    vis = synth.noise((len(layers) * nb,), 1.0, 43, "cpu")
    got, _ = gpu_images(torch, ctx, xyz, layers, vis)
    want, _ = oracle_images(xyz, layers, vis)
    assert_images_close(got, want, what="grid array")
    again, _ = gpu_images(torch, ctx, xyz, layers, vis)
    for a, b in zip(got, again):
        assert np.array_equal(a, b)


def test_normalize_flag(torch, ctx):
    ws = synth.station_batch(seed=8, n_times=1)
    layers, vis = ws_sub(ws, [0], [0, 31])
    raw, wsum = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    norm, _ = gpu_images(torch, ctx, ws.ant_xyz, layers, vis, flags=1)
    for r, n, w in zip(raw, norm, wsum):
        assert np.abs(n * w - r).max() <= 1e-6 * np.abs(r).max()


def test_all_baselines_dropped_gives_zero_image(torch, ctx):
    ws = synth.single_image(seed=1)
    # a cell far smaller than any baseline puts every baseline off the grid
    layers = [dict(n_px=16, weighting=1, freq_hz=160e6, delta_u=1e-9, vis_offset=0)]
    vis = synth.noise((ws.n_baselines,), 1.0, 42, "cpu")
    got, wsum = gpu_images(torch, ctx, ws.ant_xyz, layers, vis)
    assert not got[0].any() and wsum[0] == 0


def test_zero_layers_is_a_no_op(torch, ctx):
    from paper_2405_13478_gb300 import binding
    xyz = to_dev(torch, np.zeros((4, 3)))
    out = torch.zeros(1, device="cuda")
    ctx.image_batch(xyz, [], torch.zeros(2, dtype=torch.complex64, device="cuda"), out)
    torch.cuda.synchronize()
    assert binding.OK == 0


def test_invalid_arguments_are_rejected(torch, ctx):
    from paper_2405_13478_gb300 import binding
    xyz = to_dev(torch, np.zeros((4, 3)))
    vis = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(64 * 64, device="cuda")
    bad = [dict(n_px=15, weighting=0, freq_hz=1e8, delta_u=1.0, vis_offset=0),
           dict(n_px=64, weighting=3, freq_hz=1e8, delta_u=1.0, vis_offset=0),
           dict(n_px=64, weighting=0, freq_hz=-1.0, delta_u=1.0, vis_offset=0),
           dict(n_px=64, weighting=0, freq_hz=1e8, delta_u=float("nan"), vis_offset=0),
           dict(n_px=64, weighting=0, freq_hz=1e8, delta_u=1.0, vis_offset=-2)]
    for L in bad:
        with pytest.raises(binding.BlinkError) as ei:
            ctx.image_batch(xyz, [L], vis, out)
        assert ei.value.status == binding.ERR_INVALID
    with pytest.raises(binding.BlinkError) as ei:
        ctx.image_batch(xyz, [dict(n_px=58, weighting=0, freq_hz=1e8, delta_u=1.0,
                                   vis_offset=0)], vis, out)
    assert ei.value.status == binding.ERR_UNSUPPORTED


def test_plan_reuse_matches_batch(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws = synth.station_batch(seed=12, n_times=2)
    layers, vis = ws_sub(ws, [0, 1], list(range(0, 32, 5)))
    layers, total = binding.layer_out_offsets(layers)
    d_xyz = to_dev(torch, ws.ant_xyz)
    d_vis = vis.reshape(-1).cuda()
    a = torch.empty(total, device="cuda")
    b = torch.empty(total, device="cuda")
    c = torch.empty(total, device="cuda")
    ctx.image_batch(d_xyz, layers, d_vis, a)
    plan = ctx.plan(d_xyz, layers)
    plan.image(d_vis, b)
    plan.image(d_vis, c)
    torch.cuda.synchronize()
    peak = a.abs().max().item()
    assert (a - b).abs().max().item() <= 1e-6 * peak
    assert (b - c).abs().max().item() <= 1e-6 * peak
    w, nk = plan.layer_info(0)
    assert w > 0 and 0 < nk <= ws.n_baselines
    plan.close()


def test_host_buffer_path_matches_device_path(torch, ctx):
    """blink_image_batch_host: host inputs and outputs, several pipeline
    chunks (585 MB of visibilities in 128 MB chunks), mixed sizes in a chunk."""
    from paper_2405_13478_gb300 import binding
    ws = synth.station_batch(seed=15, n_times=70)          # 2240 layers, 585 MB of visibilities
    vis = ws.vis("cpu")
    layers = ws.layers()
    layers[5] = dict(layers[5], n_px=256, delta_u=0.3, weighting=0)
    layers, total = binding.layer_out_offsets(layers)
    h_vis = vis.reshape(-1).pin_memory()
    h_img = torch.empty(total, dtype=torch.float32).pin_memory()
    h_ws = torch.empty(len(layers), dtype=torch.float32)
    ctx.image_batch_host(ws.ant_xyz, layers, h_vis, h_img, h_ws)
    d_img = torch.empty(total, dtype=torch.float32, device="cuda")
    d_ws = torch.empty(len(layers), dtype=torch.float32, device="cuda")
    ctx.image_batch(to_dev(torch, ws.ant_xyz), layers, vis.reshape(-1).cuda(), d_img, d_ws)
    torch.cuda.synchronize()
    h, d = h_img.numpy(), d_img.cpu().numpy()
    for L in layers:
        o, n = L["out_offset"], L["n_px"] ** 2
        assert np.abs(h[o:o + n] - d[o:o + n]).max() <= 1e-6 * np.abs(d[o:o + n]).max()
    assert torch.equal(h_ws, d_ws.cpu())


# ------------------------------------------------- full bench configuration
def test_station_batch_full_batch_sampled_layers(torch, ctx):
    """The bench workload (32000 layers of 180^2, uniform) in one call;
    sampled layers against the oracle, every layer checked for finiteness and
    for the summed-weight identity of its channel."""
    from paper_2405_13478_gb300 import binding
    ws = synth.station_batch(seed=0)
    vis = ws.vis("cuda")                       # [1000][32][32640] complex64 on the GPU
    layers = ws.layers()
    layers, total = binding.layer_out_offsets(layers)
    out = torch.empty(total, dtype=torch.float32, device="cuda")
    wsum = torch.empty(len(layers), dtype=torch.float32, device="cuda")
    ctx.image_batch(to_dev(torch, ws.ant_xyz), layers, vis.reshape(-1), out, wsum)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all().item()
    rng = np.random.default_rng(0)
    pick = sorted(set(rng.integers(0, len(layers), 12).tolist() + [0, len(layers) - 1]))
    sub = [dict(layers[k], vis_offset=i * ws.n_baselines) for i, k in enumerate(pick)]
    vcpu = torch.stack([vis.reshape(-1)[layers[k]["vis_offset"]:layers[k]["vis_offset"] +
                                        ws.n_baselines] for k in pick]).cpu()
    want, wref = oracle.image_batch(ws.ant_xyz, sub, vcpu.reshape(-1).numpy(), "fft")
    o = out.cpu().numpy()
    got = [o[layers[k]["out_offset"]:layers[k]["out_offset"] + 180 * 180].reshape(180, 180)
           for k in pick]
    assert_images_close(got, want, what="station-full")
    w = wsum.cpu().numpy()
    assert np.allclose(w[pick], wref, rtol=1e-7)
    # summed weight depends only on the channel
    assert np.array_equal(w.reshape(1000, 32), np.broadcast_to(w[:32], (1000, 32)))
    del vis, out


def test_scheduled_gridding_is_bit_reproducible(torch, ctx):
    # The station workload uses the atomic-free register-accumulation
    # gridding: every cell sums its visibilities in a fixed order, so two runs
    # give the same bits.
    from paper_2405_13478_gb300 import binding
    ws = synth.station_batch(seed=14, n_times=2)
    layers, vis = ws_sub(ws, [0, 1], list(range(0, 32, 3)))
    layers, total = binding.layer_out_offsets(layers)
    d_xyz = to_dev(torch, ws.ant_xyz)
    d_vis = vis.reshape(-1).cuda()
    a = torch.empty(total, device="cuda")
    b = torch.empty(total, device="cuda")
    ctx.image_batch(d_xyz, layers, d_vis, a)
    ctx.image_batch(d_xyz, layers, d_vis, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
