"""Failure detection without a GPU fault: the tensor-core kernels' barrier
waits are bounded; when one runs out the kernel records BLINK_ERR_TIMEOUT in
the plan's status word, drains its own copies and MMAs, frees its tensor
memory and returns.  The test lowers the wait limit so the first waits give
up at once, reads the status, then checks that the same context and plan
produce correct images again."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


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


def test_bounded_wait_timeout_is_reported_and_the_context_recovers(torch, ctx):
    from paper_2405_13478_gb300 import binding
    ws = synth.station_512(seed=7, n_times=1)
    B = ws.n_baselines
    layers = [dict(n_px=512, weighting=0, freq_hz=float(ws.freqs_hz[c]), delta_u=0.5,
                   vis_offset=k * B) for k, c in enumerate((0, 8, 15))]
    layers, total = binding.layer_out_offsets(layers)
    vis = ws.vis("cpu", times=[0])[0, [0, 8, 15], :].contiguous().reshape(-1)
    plan = ctx.plan(torch.as_tensor(ws.ant_xyz).cuda(), layers)
    d_vis = vis.cuda()
    out = torch.full((total,), float("nan"), device="cuda")
    ctx.set_wait_limit(0)
    try:
        plan.image(d_vis, out, flags=binding.TRANSFORM_BF16X3)
        with pytest.raises(binding.BlinkError) as ei:
            plan.check()
        assert ei.value.status == binding.ERR_TIMEOUT
        assert torch.isnan(out).any()            # timed-out tiles were not written
    finally:
        ctx.set_wait_limit(-1)
    plan.check()                                 # the status word was cleared
    out.fill_(float("nan"))
    plan.image(d_vis, out, flags=binding.TRANSFORM_BF16X3)
    plan.check()
    torch.cuda.synchronize()
    want, _ = oracle.image_batch(ws.ant_xyz, layers, vis.numpy(), "fft")
    o = out.cpu().numpy()
    for L, w in zip(layers, want):
        g = o[L["out_offset"]:L["out_offset"] + 512 * 512].reshape(512, 512)
        assert np.isfinite(g).all()
        assert np.abs(g - w).max() <= 1e-5 * np.abs(w).max()
    plan.close()
