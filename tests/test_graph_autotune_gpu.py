"""GPU: kernel-path choice, the autotuner and CUDA-graph replay of a plan.

Every kernel path a size group can take (scheduled fused, atomic fused,
two-kernel with several wave budgets) must give the oracle's images within
the same bar as the default path: max |gpu - oracle| <= 1e-5 * max |oracle|
per layer.  A replayed graph must track new visibility contents written into
the buffers it was captured with.
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


def mixed_layers(ws, times, chans):
    from paper_2405_13478_gb300 import binding
    vis = ws.vis("cpu", times=times)[:, chans, :].contiguous()
    layers = []
    for t in range(len(times)):
        for c, ch in enumerate(chans):
            layers.append(dict(n_px=int(ws.n_px[ch]), weighting=int(ws.weighting),
                               freq_hz=float(ws.freqs_hz[ch]), delta_u=float(ws.delta_u[ch]),
                               vis_offset=(t * len(chans) + c) * ws.n_baselines))
    layers, total = binding.layer_out_offsets(layers)
    return layers, total, vis


def split(out, layers):
    o = out.cpu().numpy()
    return [o[L["out_offset"]:L["out_offset"] + L["n_px"] ** 2].reshape(L["n_px"], L["n_px"])
            for L in layers]


def assert_close(got, want, what=""):
    for k, (g, w) in enumerate(zip(got, want)):
        peak = np.abs(w).max()
        err = np.abs(g.astype(np.float64) - w).max()
        assert np.isfinite(g).all(), f"{what} layer {k}: non-finite output"
        assert err <= IMG_TOL * peak, f"{what} layer {k}: max err {err:.3e} vs peak {peak:.3e}"


def small_size_workload(seed):
    """A station of station-batch shape imaged at every small size, both weightings."""
    ws = synth.station_batch(seed=seed, n_times=2)
    sizes = [16, 20, 64, 128, 180, 256]
    layers = []
    for k, n in enumerate(sizes):
        f = float(ws.freqs_hz[(7 * k) % 32])
        du = synth.max_uv(ws.ant_xyz, f) / (n / 2 - 1) * (1.3 if n <= 20 else 1.0)
        layers.append(dict(n_px=n, weighting=k % 2, freq_hz=f, delta_u=du,
                           vis_offset=k * ws.n_baselines))
    vis = synth.noise((len(sizes) * ws.n_baselines,), 1.0, seed, "cpu")
    return ws, layers, vis


@pytest.mark.parametrize("path", [1, 2, 3, 4])
def test_every_kernel_path_matches_oracle_small_sizes(torch, ctx, path):
    from paper_2405_13478_gb300 import binding
    ws, layers, vis = small_size_workload(seed=21)
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    taken = []
    for g in range(len(layers)):
        try:
            plan.set_tuning(g, path, 4 << 20 if path >= 3 else 0)
            taken.append(path)
        except binding.BlinkError as e:
            # the fused kernels are unavailable where the image's canonical
            # rows do not fit shared memory (or, scheduled, the schedule)
            assert path in (1, 2) and e.status == binding.ERR_INVALID
            taken.append(0)
    assert taken.count(path) >= len(layers) - 2
    out = torch.full((total,), float("nan"), device="cuda")
    plan.image(vis.cuda(), out)
    torch.cuda.synchronize()
    plan.check()
    want, _ = oracle.image_batch(ws.ant_xyz, layers, vis.numpy(), "fft")
    assert_close(split(out, layers), want, what=f"path {path}")
    assert [t[1] for t in plan.tuning()] == taken
    plan.close()


@pytest.mark.parametrize("path", [3, 4])
@pytest.mark.parametrize("wave_mb", [1, 12, 96])
def test_wave_budgets_match_oracle_large_sizes(torch, ctx, wave_mb, path):
    ws = synth.uneven_batch(seed=8, n_times=30)
    layers, total, vis = mixed_layers(ws, [20, 21], [200, 300, 767])   # 512, 1024, 1024
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    for g, _ in enumerate(plan.tuning()):
        plan.set_tuning(g, path, wave_mb << 20)
    out = torch.full((total,), float("nan"), device="cuda")
    plan.image(vis.reshape(-1).cuda(), out)
    torch.cuda.synchronize()
    want, _ = oracle.image_batch(ws.ant_xyz, layers, vis.reshape(-1).numpy(), "fft")
    assert_close(split(out, layers), want, what=f"path {path}, scratch {wave_mb} MB")
    plan.close()


def test_unavailable_paths_are_rejected(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws = synth.uneven_batch(seed=8, n_times=30)
    layers, total, vis = mixed_layers(ws, [20], [0, 300])   # 128, 1024
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    assert [t[0] for t in plan.tuning()] == [128, 1024]
    for bad in [(1, 1, 0), (1, 2, 0), (0, 5, 0), (0, 3, -1), (2, 3, 0), (-1, 0, 0)]:
        with pytest.raises(binding.BlinkError) as ei:
            plan.set_tuning(*bad)
        assert ei.value.status == binding.ERR_INVALID
    assert [t[1] for t in plan.tuning()] == [0, 0]
    plan.close()


def test_autotune_choice_keeps_parity(torch, ctx):
    ws = synth.uneven_batch(seed=9, n_times=30)
    layers, total, vis = mixed_layers(ws, [20, 25], [0, 100, 200, 300, 767])
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    d_vis = vis.reshape(-1).cuda()
    out = torch.full((total,), float("nan"), device="cuda")
    plan.autotune(d_vis, out)
    tune = plan.tuning()
    assert [t[0] for t in tune] == [128, 256, 512, 1024]
    assert all(t[1] in (1, 2, 3, 4) for t in tune)
    out.fill_(float("nan"))
    plan.image(d_vis, out)
    torch.cuda.synchronize()
    want, _ = oracle.image_batch(ws.ant_xyz, layers, vis.reshape(-1).numpy(), "fft")
    assert_close(split(out, layers), want, what="autotuned")
    plan.close()


@pytest.mark.parametrize("flags", [0, 1])
def test_graph_replay_tracks_new_visibilities(torch, ctx, flags):
    ws = synth.uneven_batch(seed=10, n_times=30)
    layers, total, vis_a = mixed_layers(ws, [20], [0, 100, 200, 300])
    _, _, vis_b = mixed_layers(ws, [25], [0, 100, 200, 300])
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    d_vis = vis_a.reshape(-1).cuda()
    out = torch.full((total,), float("nan"), device="cuda")
    wsum = torch.zeros(len(layers), device="cuda")
    plan.capture(d_vis, out, wsum, flags)
    for vis in (vis_b, vis_a):
        d_vis.copy_(vis.reshape(-1))
        out.fill_(float("nan"))
        plan.replay()
        torch.cuda.synchronize()
        plan.check()
        want, ws_want = oracle.image_batch(ws.ant_xyz, layers, vis.reshape(-1).numpy(), "fft")
        ws_want = np.asarray(ws_want)
        if flags:
            want = [w / s for w, s in zip(want, ws_want)]
        assert_close(split(out, layers), want, what="replay")
        assert np.allclose(wsum.cpu().numpy(), ws_want, rtol=1e-6)
    plan.close()


def test_graph_of_tensor_core_mode(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws = synth.station_512(seed=3, n_times=1)
    layers = [dict(n_px=512, weighting=0, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=c * ws.n_baselines) for c in range(4)]
    layers, total = binding.layer_out_offsets(layers)
    vis = ws.vis("cpu", times=[0])[0, :4, :].contiguous().reshape(-1)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    d_vis = vis.cuda()
    a = torch.empty(total, device="cuda")
    b = torch.full((total,), float("nan"), device="cuda")
    plan.image(d_vis, a, flags=binding.TRANSFORM_BF16X3)
    plan.capture(d_vis, b, None, binding.TRANSFORM_BF16X3)
    b.fill_(float("nan"))
    plan.replay()
    torch.cuda.synchronize()
    # same kernels; only the order of the shared-memory gridding atomics may differ
    assert (a - b).abs().max().item() <= 1e-5 * a.abs().max().item()
    plan.close()


def test_replay_without_capture_is_an_error(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws = synth.single_image(seed=1)
    layers = [dict(n_px=256, weighting=0, freq_hz=float(ws.freqs_hz[0]),
                   delta_u=float(ws.delta_u[0]), vis_offset=0)]
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    with pytest.raises(binding.BlinkError) as ei:
        plan.replay()
    assert ei.value.status == binding.ERR_INVALID
    plan.close()
