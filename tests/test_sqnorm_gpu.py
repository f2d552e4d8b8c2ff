"""Per-layer sums of squares of the fused epilogue (blink_epilogue.d_sqnorm),
the per-layer scaled adjoint (blink_plan_degrid_scaled) and the autograd
least-squares loss built from the two, on every kernel path.

Bars:
- the reduction alone: each sum against the FP64 sum of the GPU's own stored
  output.  The kernels add at most 2 N2 <= 64 squares in FP32 before FP64,
  so the relative error is below 64 u (u = 2^-24), written as 5e-6;
- the whole path: against the FP64 oracle's images minus the reference.
  With |g - o| <= e = 1e-5 max|o| per pixel (the image bar),
  |sum g^2 - sum o^2| <= e (2 sum |o| + n e), plus the reduction's 5e-6;
- the scaled adjoint: layer l of the result is scale[l] times the unscaled
  one, within one FP32 rounding of the product (1e-6 of the layer's peak);
- results are the same bits from call to call and through a CUDA graph
  (except on the shared-atomic fused path, which adds in arrival order).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
RED = 5e-6


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
    return [flat[L["out_offset"]:L["out_offset"] + L["n_px"] ** 2] for L in layers]


def mixed_case(seed):
    """Full-support layers of every path family: fused sizes, 512^2 and
    1024^2 with row buckets (3 km array), in one plan."""
    ws = synth.single_image(seed=seed)
    nb = ws.n_baselines
    f = float(ws.freqs_hz[0])
    layers = []
    for k, (n, w) in enumerate([(128, 0), (180, 1), (256, 0), (512, 1), (1024, 0), (1024, 1)]):
        du = synth.max_uv(ws.ant_xyz, f) / (n / 2 - 1)
        layers.append(dict(n_px=n, weighting=w, freq_hz=f * (1 - 0.01 * k), delta_u=du,
                           vis_offset=k * nb))
    vis = synth.noise((len(layers) * nb,), 1.0, seed, "cpu")
    return ws, layers, vis


def compact_case(seed, n_px=512):
    """Station layers whose support fits the compact gridding."""
    ws = synth.station_gains(seed=seed, n_times=1)
    nb = ws.n_baselines
    layers = [dict(n_px=n_px, weighting=w, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=k * nb) for k, (c, w) in enumerate([(0, 0), (3, 1), (7, 0)])]
    vis = synth.noise((len(layers) * nb,), 1.0, seed, "cpu")
    return ws, layers, vis


def force(plan, path):
    from paper_2405_13478_gb300 import binding
    if path is None:
        return
    for g in range(len(plan.tuning())):
        try:
            plan.set_tuning(g, path)
        except binding.BlinkError:
            pass  # the group cannot take this path; it keeps its default


def check_case(torch, ctx, ws, layers, vis, path, with_ref):
    from paper_2405_13478_gb300 import binding
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    force(plan, path)
    want, _ = oracle.image_batch(ws.ant_xyz, layers, vis.numpy())
    ref = None
    if with_ref:  # half of the dirty image plus noise: the residual keeps structure
        rng = np.random.default_rng(3)
        ref = np.concatenate([0.5 * w.reshape(-1) for w in want]).astype(np.float32)
        ref += rng.normal(0, 0.01 * np.abs(ref).max(), ref.size).astype(np.float32)
    d_vis = vis.reshape(-1).cuda()
    d_ref = None if ref is None else torch.as_tensor(ref).cuda()
    out = torch.full((total,), float("nan"), device="cuda")
    sq = torch.full((len(layers),), float("nan"), dtype=torch.float64, device="cuda")
    plan.image(d_vis, out, ref=d_ref, sqnorm=sq)
    plan.check()
    got_img, got_sq = out.cpu().numpy(), sq.cpu().numpy()
    # the same bits again, and through a graph.  Layers that a forced path
    # grids with shared-memory atomics (path 2; paths 3 and 4 on sizes whose
    # channels have no row buckets because the fused kernel always fits them)
    # add in arrival order and may differ in the last bits.
    out2 = torch.empty_like(out)
    sq2 = torch.empty_like(sq)
    plan.image(d_vis, out2, ref=d_ref, sqnorm=sq2)
    sq3 = torch.zeros_like(sq)
    plan.capture(d_vis, torch.empty_like(out), ref=d_ref, sqnorm=sq3)
    sq3.zero_()
    plan.replay()
    plan.check()
    for k, L in enumerate(layers):
        o0, n2 = L["out_offset"], L["n_px"] ** 2
        x, y = out[o0:o0 + n2], out2[o0:o0 + n2]
        if path is None or L["n_px"] >= 512:
            assert torch.equal(x, y), f"layer {k}: images differ between calls"
            assert sq[k] == sq2[k] and sq[k] == sq3[k], f"layer {k}: sums differ between calls"
        else:
            assert float((x - y).abs().max()) <= 1e-5 * float(x.abs().max())
            assert abs(float(sq[k] - sq2[k])) <= 1e-5 * float(sq[k])
            assert abs(float(sq[k] - sq3[k])) <= 1e-5 * float(sq[k])
    plan.close()
    refs = split(ref, layers) if ref is not None else [0.0] * len(layers)
    for k, (g, o, r) in enumerate(zip(split(got_img, layers), want, refs)):
        g64 = g.astype(np.float64)
        own = float(np.sum(g64 * g64))
        assert abs(got_sq[k] - own) <= RED * own, f"layer {k}: reduction {got_sq[k]!r} vs {own!r}"
        o = o.reshape(-1) - (r.astype(np.float64) if ref is not None else 0.0)
        e = TOL * np.abs(want[k]).max() + (TOL * np.abs(r).max() if ref is not None else 0.0)
        assert np.abs(g64 - o).max() <= e, f"layer {k}: image"
        ex = float(np.sum(o * o))
        bound = e * (2 * np.abs(o).sum() + o.size * e) + RED * ex
        assert abs(got_sq[k] - ex) <= bound, f"layer {k}: {got_sq[k]!r} vs oracle {ex!r} (bound {bound:.3e})"


@pytest.mark.parametrize("path", [None, 2, 3, 4])
@pytest.mark.parametrize("with_ref", [False, True])
def test_sqnorm_every_path(torch, ctx, path, with_ref):
    ws, layers, vis = mixed_case(17)
    check_case(torch, ctx, ws, layers, vis, path, with_ref)


@pytest.mark.parametrize("path", [None, 3])
def test_sqnorm_compact_gridding(torch, ctx, path):
    ws, layers, vis = compact_case(4)
    check_case(torch, ctx, ws, layers, vis, path, True)


def test_sqnorm_refuses_tensor_modes(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws, layers, vis = compact_case(5)
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    out = torch.empty(total, device="cuda")
    sq = torch.empty(len(layers), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.BlinkError) as ei:
        plan.image(vis.reshape(-1).cuda(), out, flags=binding.TRANSFORM_BF16X3, sqnorm=sq)
    assert ei.value.status == binding.ERR_UNSUPPORTED
    plan.close()


def test_degrid_scaled_is_per_layer_scale(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws, layers, vis = mixed_case(23)
    layers, total = binding.layer_out_offsets(layers)
    nb = ws.n_baselines
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    rng = np.random.default_rng(9)
    dimg = torch.as_tensor(rng.normal(size=total).astype(np.float32)).cuda()
    scale = torch.as_tensor(np.array([1.0, -2.5, 0.0, 3e-3, 7.0, -1.0], np.float32)).cuda()
    d1 = torch.zeros(len(layers) * nb, dtype=torch.complex64, device="cuda")
    d2 = torch.zeros_like(d1)
    plan.degrid(dimg, d1)
    plan.degrid(dimg, d2, layer_scale=scale)
    torch.cuda.synchronize()
    a = d1.cpu().numpy().reshape(len(layers), nb)
    b = d2.cpu().numpy().reshape(len(layers), nb)
    s = scale.cpu().numpy()
    for k in range(len(layers)):
        want = s[k].astype(np.float64) * a[k].astype(np.complex128)
        assert np.abs(b[k] - want).max() <= 1e-6 * max(np.abs(want).max(), 1e-30), f"layer {k}"
    plan.close()


@pytest.mark.parametrize("n_px", [180, 1024])
def test_autograd_sqnorm_loss(torch, ctx, n_px):
    """sum_l c_l |image_l - ref_l|^2 from image_sqnorm and from dirty_images
    + torch: the same loss and the same visibility gradient."""
    from paper_2405_13478_gb300 import autograd, binding
    ws = synth.station_gains(seed=12, n_times=1)
    B = ws.n_baselines
    layers = [dict(n_px=n_px, weighting=w, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5, vis_offset=k * B)
              for k, (c, w) in enumerate([(1, 0), (6, 1), (3, 0)])]
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    v0 = ws.vis("cuda", times=[0])[:, [1, 6, 3], :].reshape(-1).contiguous()
    t = (0.5 * autograd.dirty_images(v0, plan, total)).detach()
    c = torch.tensor([1.0, 0.25, -0.5], dtype=torch.float64, device="cuda")
    a = v0.clone().requires_grad_(True)
    img = autograd.dirty_images(a, plan, total)
    r = (img - t).double()
    per = torch.stack([(r[L["out_offset"]:L["out_offset"] + n_px * n_px] ** 2).sum() for L in layers])
    la = (c * per).sum()
    la.backward()
    b = v0.clone().requires_grad_(True)
    sq = autograd.image_sqnorm(b, plan, total, ref=t)
    lb = (c * sq).sum()
    lb.backward()
    torch.cuda.synchronize()
    assert torch.allclose(sq.detach(), per.detach(), rtol=1e-5, atol=0)
    assert abs(float(la.detach()) - float(lb.detach())) <= 1e-5 * float(per.detach().abs().sum())
    ga, gb = a.grad, b.grad
    assert float((ga - gb).abs().max()) <= 1e-5 * float(ga.abs().max())
    plan.close()


@pytest.mark.parametrize("case,path,flags", [("mixed", None, 0), ("mixed", 3, 1), ("mixed", 4, 0),
                                             ("compact1024", None, 0), ("compact1024", 3, 0),
                                             ("compact512", None, 0x20)])
def test_kept_adjoint_is_the_adjoint_of_the_stored_images(torch, ctx, case, path, flags):
    """blink_plan_degrid_adjoint from the columns kept by the forward (fused
    into the 1024^2 column pass, or from the stored images elsewhere and in
    the tensor-core modes) gives the bits of blink_plan_degrid_scaled on the
    stored images."""
    from paper_2405_13478_gb300 import binding
    if case == "mixed":
        ws, layers, vis = mixed_case(29)
    else:
        ws, layers, vis = compact_case(6, int(case[len("compact"):]))
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    force(plan, path)
    rng = np.random.default_rng(2)
    d_vis = vis.reshape(-1).cuda()
    ref = torch.as_tensor(rng.normal(0, 1.0, total).astype(np.float32)).cuda()
    out = torch.empty(total, device="cuda")
    adj = torch.full((plan.adjoint_bytes() // 4,), float("nan"), device="cuda")
    plan.image(d_vis, out, flags=flags, ref=ref, adjoint=adj)
    plan.check()
    scale = torch.as_tensor(rng.normal(size=len(layers)).astype(np.float32)).cuda()
    nb = ws.n_baselines
    d1 = torch.zeros(len(layers) * nb, dtype=torch.complex64, device="cuda")
    d2 = torch.zeros_like(d1)
    nflag = flags & binding.NORMALIZE
    plan.degrid(out, d1, nflag, layer_scale=scale)
    plan.degrid_adjoint(adj, d2, nflag, layer_scale=scale)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(d1)).all()
    assert torch.equal(d1, d2)
    plan.close()


@pytest.mark.parametrize("case", ["mixed", "compact1024"])
def test_no_image_output_with_kept_adjoint(torch, ctx, case):
    """With the adjoint columns kept, the image array may be omitted: the
    sums of squares and the kept columns are the bits of a call that stores
    the images (1024^2 fused; other sizes through a temporary array)."""
    from paper_2405_13478_gb300 import binding
    ws, layers, vis = mixed_case(31) if case == "mixed" else compact_case(8, 1024)
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    d_vis = vis.reshape(-1).cuda()
    ref = torch.as_tensor(np.random.default_rng(4).normal(0, 1.0, total).astype(np.float32)).cuda()
    out = torch.empty(total, device="cuda")
    n_adj = plan.adjoint_bytes() // 4
    a1, a2 = torch.empty(n_adj, device="cuda"), torch.empty(n_adj, device="cuda")
    s1 = torch.empty(len(layers), dtype=torch.float64, device="cuda")
    s2 = torch.empty_like(s1)
    plan.image(d_vis, out, ref=ref, sqnorm=s1, adjoint=a1)
    plan.image(d_vis, None, ref=ref, sqnorm=s2, adjoint=a2)
    plan.check()
    assert torch.equal(s1, s2)
    d1 = torch.zeros(len(layers) * ws.n_baselines, dtype=torch.complex64, device="cuda")
    d2 = torch.zeros_like(d1)
    plan.degrid_adjoint(a1, d1)
    plan.degrid_adjoint(a2, d2)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
    # the same through a CUDA graph (the plan's own image array, where one is
    # needed, is allocated by the capture's first run, outside the graph)
    a3, s3 = torch.empty(n_adj, device="cuda"), torch.empty_like(s1)
    plan.capture(d_vis, None, ref=ref, sqnorm=s3, adjoint=a3)
    a3.zero_()
    s3.zero_()
    plan.replay()
    plan.check()
    d3 = torch.zeros_like(d1)
    plan.degrid_adjoint(a3, d3)
    torch.cuda.synchronize()
    assert torch.equal(s1, s3) and torch.equal(d1, d3)
    with pytest.raises(binding.BlinkError):
        plan.image(d_vis, None, ref=ref, sqnorm=s2)  # no images and nothing kept
    plan.close()
