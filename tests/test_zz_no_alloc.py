"""blink_image_batch_noalloc: the allocation-free variant for callers that may
not allocate device memory while they run (real-time pipelines that reserve
all GPU memory up front, hosts whose allocator owns the device).

Called through the C ABI on two calls in a row (the static scratch keeps
the previous call's contents).  When its tables fit the static array it runs
the same deterministic kernels as blink_image_batch, so its images must be
the same bits; they must also match the FP64 oracle within the image
tolerance of the parity tests.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2405_13478_gb300 import binding, build

    build.build()
    lib = binding.lib()
    fn = lib.blink_image_batch_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(binding.Layer), ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                   ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    ctx = binding.Context(0)
    yield torch, binding, fn, ctx
    ctx.close()


def noalloc(env, xyz, layers, vis, total, flags=0):
    torch, binding, fn, _ = env
    out = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    ws = torch.zeros(len(layers), dtype=torch.float32, device="cuda")
    msg = ctypes.create_string_buffer(256)
    arr = binding.make_layers(layers)
    st = fn(ctypes.c_void_p(xyz.data_ptr()), xyz.shape[0], arr, len(layers),
            ctypes.c_void_p(vis.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(ws.data_ptr()), flags,
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), msg, 256)
    torch.cuda.synchronize()
    return st, msg.value.decode(), out, ws


def reference(env, xyz, layers, vis, total, flags=0):
    torch, _, _, ctx = env
    out = torch.empty(total, dtype=torch.float32, device="cuda")
    ws = torch.zeros(len(layers), dtype=torch.float32, device="cuda")
    ctx.image_batch(xyz, layers, vis, out, ws, flags)
    torch.cuda.synchronize()
    return out, ws


def check_same(layers, got, want):
    g = got.cpu().numpy()
    w = want.cpu().numpy()
    for L in layers:
        o, n = L["out_offset"], L["n_px"] ** 2
        peak = np.abs(w[o:o + n]).max()
        assert np.isfinite(g[o:o + n]).all()
        assert np.abs(g[o:o + n] - w[o:o + n]).max() <= IMG_TOL * peak


def check_oracle(ws, args, got, flags, picks=(0, -1)):
    """A few layers of a call against the FP64 oracle (1e-5 of the peak)."""
    _, layers, vis, _ = args
    B = ws.n_baselines
    g = got.cpu().numpy()
    v = vis.cpu().numpy()
    for k in picks:
        L = layers[k]
        want, ws_ = oracle.image_batch(ws.ant_xyz, [dict(L, vis_offset=0, out_offset=0)],
                                       v[L["vis_offset"]:L["vis_offset"] + B], "fft")
        w = want[0] / (ws_[0] if flags & 1 else 1.0)
        n2 = L["n_px"] ** 2
        img = g[L["out_offset"]:L["out_offset"] + n2].reshape(w.shape)
        assert np.abs(img - w).max() <= IMG_TOL * np.abs(w).max()


def workload(env, ws, times, chans):
    torch, binding, _, _ = env
    vis = ws.vis("cuda", times=times)[:, chans, :].contiguous().reshape(-1)
    B = ws.n_baselines
    layers = []
    for t in range(len(times)):
        for k, c in enumerate(chans):
            layers.append(dict(n_px=int(ws.n_px[c]), weighting=ws.weighting,
                               freq_hz=float(ws.freqs_hz[c]), delta_u=float(ws.delta_u[c]),
                               vis_offset=(t * len(chans) + k) * B))
    layers, total = binding.layer_out_offsets(layers)
    return torch.as_tensor(ws.ant_xyz).cuda(), layers, vis, total


def test_noalloc_matches_image_batch_two_calls_in_a_row(env):
    # call 1: 96 uniform-weighted 180^2 layers over 32 channels (fused path)
    a_ws = synth.station_batch(seed=21, n_times=3)
    a = workload(env, a_ws, [0, 1, 2], list(range(32)))
    # call 2: 1024^2 natural layers of a 3 km array (row/column path with scratch rows)
    w2 = synth.single_image(seed=22)
    w2.n_px = np.array([1024])
    w2.delta_u = np.array([synth.max_uv(w2.ant_xyz, w2.freqs_hz[0]) / 511])
    b = workload(env, w2, [0], [0])
    # call 3: 512^2 station layers, whose support takes the compact gridding
    c_ws = synth.station_512(seed=23, n_times=2)
    c = workload(env, c_ws, [0, 1], [0, 5, 10, 15])
    for (ws, args), flags in (((a_ws, a), 0), ((w2, b), 1), ((c_ws, c), 0), ((a_ws, a), 1)):
        st, msg, got, gws = noalloc(env, *args, flags)
        assert st == 0, msg
        want, wws = reference(env, *args, flags)
        check_same(args[1], got, want)
        torch = env[0]
        assert torch.equal(got, want)  # the same kernels on the same tables
        assert np.allclose(gws.cpu().numpy(), wws.cpu().numpy(), rtol=1e-7)
        check_oracle(ws, args, got, flags)


def test_noalloc_rejects_requests_beyond_its_limits(env):
    torch, binding, _, _ = env
    ws = synth.station_batch(seed=23, n_times=1)
    xyz = torch.as_tensor(ws.ant_xyz).cuda()
    vis = torch.zeros(ws.n_baselines, dtype=torch.complex64, device="cuda")
    # more distinct channels than the static limit
    many = [dict(n_px=180, weighting=1, freq_hz=1.5e8 + k, delta_u=0.5, vis_offset=0,
                 out_offset=0) for k in range(300)]
    st, msg, _, _ = noalloc(env, xyz, many, vis, 180 * 180)
    assert st == binding.ERR_WORKSPACE and "channels" in msg
    # tables larger than the static array: 4096 antennas -> 8.4 M baselines
    big = torch.zeros((4096, 3), dtype=torch.float64, device="cuda")
    st, msg, _, _ = noalloc(env, big, many[:1], vis, 180 * 180)
    assert st == binding.ERR_WORKSPACE and "BLINK_NOALLOC_SCRATCH_BYTES" in msg
    # one size per call
    mixed = [dict(many[0]), dict(many[0], n_px=128)]
    st, msg, _, _ = noalloc(env, xyz, mixed, vis, 180 * 180)
    assert st == binding.ERR_INVALID and "n_px" in msg
