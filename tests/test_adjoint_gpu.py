"""GPU adjoint (blink_degrid, gain gradients, autograd) against the FP64 oracle.

Tolerance: the gradient is an FP32 forward 2-D transform of the image
gradient followed by a gather, so its error is bounded like the forward
image's: max |gpu - oracle| <= 1e-5 * max |oracle| per layer (the oracle's
own adjoint is pinned by FP64 finite differences in test_oracle_adjoint).
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


def layer_cells(xyz, L):
    u, v = oracle.uv(xyz, L["freq_hz"])
    return oracle.cells(u, v, L["delta_u"], L["n_px"])


def run_degrid(torch, ctx, xyz, layers, resid_list, nb, flags=0):
    from paper_2405_13478_gb300 import binding
    layers, total = binding.layer_out_offsets(layers)
    r = torch.cat([torch.as_tensor(x.reshape(-1), dtype=torch.float32) for x in resid_list]).cuda()
    dvis = torch.full((len(layers) * nb,), complex(float("nan"), 0), dtype=torch.complex64,
                      device="cuda")
    lay = [dict(L, vis_offset=k * nb) for k, L in enumerate(layers)]
    ctx.degrid(torch.as_tensor(xyz).cuda(), lay, r, dvis, flags)
    torch.cuda.synchronize()
    return dvis.cpu().numpy().reshape(len(layers), nb)


@pytest.mark.parametrize("n_px", [16, 20, 128, 180, 256, 512, 1024])
@pytest.mark.parametrize("weighting", [0, 1])
def test_degrid_matches_oracle(torch, ctx, n_px, weighting):
    ws = synth.single_image(seed=n_px + 7)
    du = synth.max_uv(ws.ant_xyz, ws.freqs_hz[0]) / (n_px / 2 - 1)
    if n_px <= 20:
        du *= 3.0  # also exercise dropped baselines
    L = dict(n_px=n_px, weighting=weighting, freq_hz=float(ws.freqs_hz[0]), delta_u=du,
             vis_offset=0)
    rng = np.random.default_rng(n_px)
    resid = rng.normal(size=(n_px, n_px))
    got = run_degrid(torch, ctx, ws.ant_xyz, [L], [resid], ws.n_baselines)[0]
    ku, kv = layer_cells(ws.ant_xyz, L)
    want = oracle.degrid(ku, kv, resid.astype(np.float32).astype(np.float64), weighting, "fft")
    assert np.isfinite(got).all()
    assert np.abs(got - want).max() <= TOL * np.abs(want).max()
    assert not got[ku == oracle.DROPPED].any()


def test_degrid_station_layers_and_normalize(torch, ctx):
    ws = synth.station_gains(seed=3, n_times=1)
    layers = [dict(n_px=1024, weighting=0, freq_hz=float(f), delta_u=0.5, vis_offset=0)
              for f in ws.freqs_hz[[0, 7]]]
    layers += [dict(n_px=180, weighting=1, freq_hz=float(ws.freqs_hz[3]), delta_u=0.5,
                    vis_offset=0)]
    rng = np.random.default_rng(5)
    res = [rng.normal(size=(L["n_px"], L["n_px"])) for L in layers]
    got = run_degrid(torch, ctx, ws.ant_xyz, layers, res, ws.n_baselines)
    got_n = run_degrid(torch, ctx, ws.ant_xyz, layers, res, ws.n_baselines, flags=1)
    for k, L in enumerate(layers):
        ku, kv = layer_cells(ws.ant_xyz, L)
        want = oracle.degrid(ku, kv, res[k].astype(np.float32).astype(np.float64),
                             L["weighting"], "fft")
        assert np.abs(got[k] - want).max() <= TOL * np.abs(want).max()
        _, _, wsum = oracle.grid(ku, kv, np.zeros(ku.size, np.complex64), L["n_px"],
                                 L["weighting"])
        assert np.abs(got_n[k] * wsum - got[k]).max() <= 1e-6 * np.abs(got[k]).max()


def test_adjoint_identity_on_gpu(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws = synth.station_batch(seed=4, n_times=1)
    B = ws.n_baselines
    layers = [dict(n_px=180, weighting=w, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=k * B) for k, (c, w) in enumerate(((0, 1), (31, 0)))]
    layers, total = binding.layer_out_offsets(layers)
    vis = synth.noise((2 * B,), 1.0, 9, "cpu").cuda()
    img = torch.empty(total, device="cuda")
    ctx.image_batch(torch.as_tensor(ws.ant_xyz).cuda(), layers, vis, img)
    r = torch.randn(total, generator=torch.Generator().manual_seed(3)).cuda()
    dvis = torch.empty(2 * B, dtype=torch.complex64, device="cuda")
    ctx.degrid(torch.as_tensor(ws.ant_xyz).cuda(), layers, r, dvis)
    torch.cuda.synchronize()
    lhs = float((r.double() * img.double()).sum())
    rhs = float((vis.to(torch.complex128) * dvis.to(torch.complex128).conj()).real.sum())
    scale = float((r.double().abs() * img.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_autograd_gains_station_gains_slice(torch, ctx):
    """station-gains form: V = g_i conj(g_j) M, loss = sum (image(V) - image(M))^2;
    gradients w.r.t. V and g from torch.autograd (library kernels) against
    the CPU reference gradient of the oracle."""
    from paper_2405_13478_gb300 import autograd, binding
    ws = synth.station_gains(seed=11, n_times=1)
    B, n_ant = ws.n_baselines, ws.n_ant
    chans = [0, 5]
    model = torch.as_tensor(synth.model_vis(ws.ant_xyz, ws.freqs_hz[chans], ws.sky)
                            .astype(np.complex64)).reshape(-1)
    layers = [dict(n_px=1024, weighting=0, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=k * B) for k, c in enumerate(chans)]
    layers, total = binding.layer_out_offsets(layers)
    d_xyz = torch.as_tensor(ws.ant_xyz).cuda()
    plan = ctx.plan(d_xyz, layers)
    g = torch.as_tensor(ws.gains.astype(np.complex64)).cuda().requires_grad_(True)
    m = model.cuda()
    target = autograd.dirty_images(m, plan, total).detach()
    vis = autograd.apply_gains(g, m, ctx, n_ant, layers)
    vis.retain_grad()
    img = autograd.dirty_images(vis, plan, total)
    loss = ((img - target) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    # CPU reference: oracle images, residual, adjoint and chain rule (FP64)
    mnp = model.numpy()
    gnp = ws.gains.astype(np.complex64).astype(np.complex128)
    i, j = np.triu_indices(n_ant, 1)
    gam_g = np.zeros(n_ant, np.complex128)
    for k, L in enumerate(layers):
        mk = mnp[k * B:(k + 1) * B].astype(np.complex128)
        vk = (gnp[i] * np.conj(gnp[j]) * mk)
        ku, kv = layer_cells(ws.ant_xyz, L)
        gi, _, _ = oracle.grid_c128(ku, kv, vk, 1024, 0)
        gt, _, _ = oracle.grid_c128(ku, kv, mk, 1024, 0)
        ii, _ = oracle.image_fft(gi)
        it, _ = oracle.image_fft(gt)
        gam_v = oracle.degrid(ku, kv, 2 * (ii - it), 0, "fft")
        got_v = vis.grad.cpu().numpy()[k * B:(k + 1) * B]
        assert np.abs(got_v - gam_v).max() <= 1e-4 * np.abs(gam_v).max()
        oracle.gain_grad(n_ant, gam_v, gnp, mk, gam_g)
    got_g = g.grad.cpu().numpy()
    assert np.abs(got_g - gam_g).max() <= 1e-4 * np.abs(gam_g).max()
    plan.close()


@pytest.mark.parametrize("n_ant", [17, 256, 300, 1024])
def test_gain_gradient_kernels_match_oracle_chain_rule(torch, ctx, n_ant):
    """blink_gain_grad alone: random visibility gradients, models and gains
    over several layers at scattered offsets, against the oracle's chain rule
    (FP64, summed over layers); two calls give the same bits."""
    B = n_ant * (n_ant - 1) // 2
    n_layers = 5
    rng = np.random.default_rng(n_ant)
    offs = [k * B + 7 * k for k in range(n_layers)]          # gaps between layers
    size = offs[-1] + B
    cplx = lambda n: (rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)
    dvis, model, gains = cplx(size), cplx(size), cplx(n_ant)
    layers = [dict(n_px=256, weighting=0, freq_hz=1.5e8, delta_u=0.5, vis_offset=o) for o in offs]
    want = np.zeros(n_ant, np.complex128)
    for o in offs:
        oracle.gain_grad(n_ant, dvis[o:o + B], gains, model[o:o + B], want)
    d_dv, d_m, d_g = (torch.as_tensor(x).cuda() for x in (dvis, model, gains))
    got = torch.empty(n_ant, dtype=torch.complex64, device="cuda")
    again = torch.empty_like(got)
    ctx.gain_grad(n_ant, layers, d_dv, d_m, d_g, got)
    ctx.gain_grad(n_ant, layers, d_dv, d_m, d_g, again)
    torch.cuda.synchronize()
    assert torch.equal(got, again)
    g = got.cpu().numpy()
    assert np.abs(g - want).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("n_px", [180, 256])
def test_degrid_unaligned_image_gradient(torch, ctx, n_px):
    """The image gradient at an odd float offset (the column pass then reads
    its strips element by element instead of in 16-byte pieces)."""
    from paper_2405_13478_gb300 import binding
    ws = synth.single_image(seed=n_px + 31)
    du = synth.max_uv(ws.ant_xyz, ws.freqs_hz[0]) / (n_px / 2 - 1)
    L = dict(n_px=n_px, weighting=0, freq_hz=float(ws.freqs_hz[0]), delta_u=du, vis_offset=0,
             out_offset=1)
    resid = np.random.default_rng(n_px).normal(size=(n_px, n_px))
    r = torch.zeros(n_px * n_px + 1, dtype=torch.float32)
    r[1:] = torch.as_tensor(resid.reshape(-1), dtype=torch.float32)
    dvis = torch.empty(ws.n_baselines, dtype=torch.complex64, device="cuda")
    ctx.degrid(torch.as_tensor(ws.ant_xyz).cuda(), [L], r.cuda(), dvis)
    torch.cuda.synchronize()
    ku, kv = layer_cells(ws.ant_xyz, L)
    want = oracle.degrid(ku, kv, resid.astype(np.float32).astype(np.float64), 0, "fft")
    got = dvis.cpu().numpy()
    assert np.abs(got - want).max() <= TOL * np.abs(want).max()


@pytest.mark.parametrize("n_px", [512, 1024])
def test_autograd_images_with_reference(torch, ctx, n_px):
    """dirty_images(vis, plan, n, ref=t) is image - t, subtracted by the fused
    epilogue at the store; the loss sum r^2 and its gradient with respect to
    the visibilities agree with the plain images minus t in torch."""
    from paper_2405_13478_gb300 import autograd, binding
    ws = synth.station_gains(seed=12, n_times=1)
    B = ws.n_baselines
    layers = [dict(n_px=n_px, weighting=w, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5, vis_offset=k * B)
              for k, (c, w) in enumerate([(1, 0), (6, 1)])]
    layers, total = binding.layer_out_offsets(layers)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    v0 = ws.vis("cuda", times=[0])[:, [1, 6], :].reshape(-1).contiguous()
    t = (0.5 * autograd.dirty_images(v0, plan, total)).detach()
    a = v0.clone().requires_grad_(True)
    img = autograd.dirty_images(a, plan, total)
    la = ((img - t) ** 2).sum()
    la.backward()
    b = v0.clone().requires_grad_(True)
    r = autograd.dirty_images(b, plan, total, ref=t)
    lb = (r * r).sum()
    lb.backward()
    torch.cuda.synchronize()
    peak = float(img.detach().abs().max())
    assert float((r.detach() - (img.detach() - t)).abs().max()) <= 1e-6 * peak
    assert abs(float(la.detach()) - float(lb.detach())) <= 1e-5 * float(la.detach())
    ga, gb = a.grad, b.grad
    assert float((ga - gb).abs().max()) <= 1e-5 * float(ga.abs().max())
    plan.close()
