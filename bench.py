#!/usr/bin/env python
"""Throughput of the BLINK dirty-image path on GB300.

Workload (the configuration the headline metric is quoted on): a 256-antenna
station (32640 baselines) in a 38 m disk, 1000 time steps x 32 channels over
150-180 MHz, 180 x 180 all-sky images, uniform weighting, 20 point sources +
sigma = 1 noise -- 32000 dirty images per step.

One step = one pass of the whole path over the batch through the C ABI:
uv, cells and weight tables (plan build, one host sync), then the gridding +
FFT kernels, then the plan release.  Inputs are device resident when the timed region
starts; `e2e` repeats the measurement with host buffers and the host<->device
copies inside the timed region.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dirty images/s and Gvis/s gridded on 1 GB300, % roofline, error vs FP64 oracle"
UNIT = "images/s"
KERNEL = "k_image_sched<180, false>"
CSRC = os.path.join(ROOT, "paper_2405_13478_gb300", "csrc")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the plan-reuse and fused-epilogue timings of the default workload")
    p.add_argument("--n-times", type=int, default=None, help="time steps per rank")
    p.add_argument("--workload", default="station", choices=["single", "station", "uneven", "station512", "gains"],
                   help="station (default): the headline station batch; the others measure the "
                        "single-image latency, uneven batch, tensor-core modes and adjoint")
    return p.parse_args()


def dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- replicas
# The path shards by layers: every rank images its own batch (its own time
# steps), there is no data-path collective, and the only cross-rank traffic is
# the barrier and the max-over-ranks of the timed interval (weak scaling).
STATION_WORKLOAD = ("station: 256 antennas in a 38 m disk, 32640 baselines, 1000 time steps x "
                    "32 channels (150-180 MHz), 180^2 all-sky images, uniform weighting, "
                    "20 sources + sigma=1 noise")


def init_replicas(backend: str):
    """(rank, world, local_rank, process group module or None).  The group is
    created only when WORLD_SIZE > 1 (torchrun sets RANK/WORLD_SIZE/MASTER_*)."""
    rank, world, local = dist()
    if world == 1:
        return rank, world, local, None
    import torch
    import torch.distributed as tdist

    if backend == "nccl":
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        tdist.init_process_group(backend)
    return rank, world, local, tdist


def max_over_ranks(value: float, pg, device) -> float:
    """The slowest rank's value (the whole job ends when it does)."""
    if pg is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, steps: int, ms: float) -> float:
    """Units per second over all ranks for `steps` steps of `ms` (max over ranks)."""
    return world * units_per_rank * steps / (ms / 1e3)


def rank_workload(rank: int, n_times: int):
    """Rank `rank`'s own station batch: same shape on every rank, independent
    data (seeded by the rank)."""
    import synth

    return synth.station_batch(seed=rank, n_times=n_times)


# Sources the dominant kernel (the fused 180^2 image kernel, its launcher and
# argument struct) is compiled from, plus the schedule builder whose tables it
# reads: the committed DRAM-traffic figure is valid only while these are
# unchanged.  The large-image, tensor-core and adjoint kernels live in other
# files and do not void it.
KERNEL_SOURCES = ("blink_common.cuh", "blink_fft.cuh", "blink_kernels.cuh", "blink_pairs.cuh",
                  "blink_image_small.cuh", "blink_tables.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_record():
    """The committed ncu summary of the dominant kernel (DRAM bytes and FP32
    instruction counts per layer), or None if it was taken from other kernel
    sources than the current ones."""
    path = os.path.join(ROOT, "profiles", "k_image_sched_180_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("csrc_sha") != kernel_source_hash():
        return None
    return d


def ncu_traffic():
    """DRAM bytes per layer of the dominant kernel from the committed ncu
    summary, or None if there is none for the current kernel sources."""
    d = ncu_record()
    return None if d is None else float(d["dram_bytes_per_layer"])


def fft_flops(n: int) -> float:
    """Flops of one complex n-point FFT by the usual 5 n log2 n convention."""
    import math
    return 5.0 * n * math.log2(n)


def image_flops(n_px: int, rows: int, entries: int) -> float:
    """Algorithmic FP32 flops of one dirty image on the half-plane path:
    `entries` complex additions of gridding (2 flops each), pass 1 on the
    `rows` support rows, pass 2 as n_px/2 paired transforms (each gives two
    real image columns)."""
    return 2.0 * entries + (rows + n_px // 2) * fft_flops(n_px)


def support_rows(ant_xyz, freqs_hz, delta_u, n_px):
    """Support rows R of each channel (largest |k_v| + 1 over the baselines,
    capped at n_px/2) -- bookkeeping for the flop count only."""
    import numpy as np
    i, j = np.triu_indices(len(ant_xyz), k=1)
    dy = ant_xyz[j, 1] - ant_xyz[i, 1]
    out = []
    for f in np.atleast_1d(freqs_hz):
        k = np.rint(np.abs(dy) * f / 299792458.0 / delta_u).max()
        out.append(int(min(k, n_px // 2 - 1)) + 1)
    return out


def alu_peak():
    """Measured FP32 and FP64 FMA rates of this GPU (TFLOP/s)."""
    from paper_2405_13478_gb300 import binding
    import torch
    dev = torch.cuda.current_device()
    return binding.fma_peak_tflops(dev, 32), binding.fma_peak_tflops(dev, 64)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def _lines(self):
        try:
            with open(self.path) as f:
                return f.read().splitlines()
        except OSError:
            return []

    def start(self):
        """Starts sampling every 50 ms and returns once the sampler writes, so
        the samples taken after this call fall in the timed region."""
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        self.skip = 0
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while not self._lines() and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.skip = len(self._lines())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = self._lines()
        os.unlink(self.path)
        # samples written during the region; the last one before it if none
        inside = lines[self.skip:]
        fallback = not inside
        if fallback:
            inside = lines[max(0, self.skip - 1):self.skip]
        rows = []
        for ln in inside:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None,
               "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
               "samples": len(rows)}
        if fallback:
            out["sampled_just_before_region"] = True
        return out


def cpu_baseline(ws, seconds: float = 10.0):
    """The FP64 oracle, as it stands, on all host cores over a bounded sample
    of the same workload (20 time steps x 32 channels, repeated for ~10 s)."""
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    n_t = 20
    vis = ws.vis("cpu", times=range(n_t)).reshape(-1).numpy()
    layers = ws.layers(times=range(n_t))
    oracle.image_batch(ws.ant_xyz, layers[:cores], vis, "fft", n_threads=cores)  # warm
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.image_batch(ws.ant_xyz, layers, vis, "fft", n_threads=cores)
        done += len(layers)
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_t} time steps x 32 channels of the same workload ({len(layers)} "
                      f"images of 180^2, uniform), repeated {done // len(layers)}x in {el:.1f} s; "
                      "FP64 C oracle, FFT route, OpenMP over images"}


def sampled_error(ctx, ws, d_xyz, vis, images, layers, n=8):
    """Max |gpu - oracle| / max |oracle| over a few layers of the batch."""
    import numpy as np
    import torch

    import oracle

    rng = np.random.default_rng(1)
    pick = sorted(set(rng.integers(0, len(layers), n).tolist()))
    B = ws.n_baselines
    sub = [dict(layers[k], vis_offset=i * B) for i, k in enumerate(pick)]
    v = torch.stack([vis[layers[k]["vis_offset"]:layers[k]["vis_offset"] + B] for k in pick])
    want, _ = oracle.image_batch(ws.ant_xyz, sub, v.cpu().reshape(-1).numpy(), "fft")
    worst = 0.0
    for k, w in zip(pick, want):
        o = layers[k]["out_offset"]
        g = images[o:o + 180 * 180].cpu().numpy().reshape(180, 180)
        worst = max(worst, float(np.abs(g - w).max() / np.abs(w).max()))
    return worst


def epilogue_variants(torch, binding, ctx, ws, d_xyz, larr, vis, images, wsum, layers, steps,
                      warmup):
    """The same batch through one reused plan: the plain transform, and the
    fused epilogue (per-channel antenna gains applied at gridding, a
    reference image subtracted at the store) as a difference-imaging search
    would run it.  Returns (dict, error of the epilogue vs the oracle)."""
    import numpy as np

    import oracle

    C, B = ws.n_chan, ws.n_baselines
    stream = torch.cuda.current_stream()
    plan = binding.Plan(ctx, d_xyz, larr)
    rng = np.random.default_rng(3)
    g = (np.abs(rng.normal(1.0, 0.1, (C, ws.n_ant)))
         * np.exp(1j * rng.uniform(-np.pi, np.pi, (C, ws.n_ant)))).astype(np.complex64)
    d_g = torch.as_tensor(g.reshape(-1)).cuda()
    ref = torch.empty_like(images)
    plan.image(vis, ref)                                  # reference = dirty images of the batch
    ref.mul_(0.5)

    def timed(fn):
        for _ in range(warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    L = len(layers)
    ms_plain = timed(lambda: plan.image(vis, images, wsum))
    ms_gains = timed(lambda: plan.image(vis, images, wsum, gains=d_g, gain_stride=ws.n_ant,
                                        gain_period=C))
    ms_ref = timed(lambda: plan.image(vis, images, wsum, ref=ref))
    ms_epi = timed(lambda: plan.image(vis, images, wsum, gains=d_g, gain_stride=ws.n_ant,
                                      gain_period=C, ref=ref))
    # sampled error of the epilogue against the oracle
    pick = [0, L // 2 + 7, L - 1]
    sub = [dict(layers[k], vis_offset=i * B) for i, k in enumerate(pick)]
    v = torch.stack([vis[layers[k]["vis_offset"]:layers[k]["vis_offset"] + B] for k in pick])
    n2 = 180 * 180
    r = torch.stack([ref[layers[k]["out_offset"]:layers[k]["out_offset"] + n2] for k in pick])
    rows = np.stack([g[k % C] for k in pick]).astype(np.complex128)
    want, _ = oracle.image_batch(ws.ant_xyz, sub, v.cpu().reshape(-1).numpy(), "fft",
                                 gains=rows.reshape(-1), gain_stride=ws.n_ant,
                                 ref=r.cpu().double().reshape(-1).numpy())
    worst = 0.0
    for k, w, rr in zip(pick, want, r.cpu().numpy()):
        o = layers[k]["out_offset"]
        got = images[o:o + n2].cpu().numpy().reshape(180, 180)
        worst = max(worst, float(np.abs(got - w).max() / (np.abs(w).max() + np.abs(rr).max())))
    plan.close()
    del ref
    bytes_plain = B * 8 + n2 * 4
    bytes_epi = bytes_plain + n2 * 4                      # + reference read
    return {"plan_reused": {"images_per_s": L / (ms_plain / 1e3), "ms_per_step": ms_plain,
                            "hbm_gbs": L * bytes_plain / (ms_plain / 1e3) / 1e9},
            "epilogue_gains": {"images_per_s": L / (ms_gains / 1e3), "ms_per_step": ms_gains},
            "epilogue_ref": {"images_per_s": L / (ms_ref / 1e3), "ms_per_step": ms_ref,
                             "hbm_gbs": L * bytes_epi / (ms_ref / 1e3) / 1e9},
            "epilogue_gains_ref": {"images_per_s": L / (ms_epi / 1e3), "ms_per_step": ms_epi,
                                   "hbm_gbs": L * bytes_epi / (ms_epi / 1e3) / 1e9,
                                   "algorithmic_bytes_per_image": bytes_epi,
                                   "err_vs_oracle": worst,
                                   "what": "per-channel antenna gains (32 rows, period 32) "
                                           "applied at gridding + reference image subtracted "
                                           "at the store"}}


def link_ceiling(torch, h_vis, h_img, chunk=128 << 20):
    """What the host link alone allows for the e2e step: plain pinned-memory
    cudaMemcpyAsync copies of the same bytes (the visibilities host -> device
    and the images device -> host, in 128 MB pieces like the library's
    pipeline), each direction alone and both at once on two streams."""
    src = torch.view_as_real(h_vis).reshape(-1).view(torch.uint8)
    dst = h_img.reshape(-1).view(torch.uint8)
    d_in = torch.empty(chunk, dtype=torch.uint8, device="cuda")
    d_out = torch.zeros(chunk, dtype=torch.uint8, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def h2d():
        with torch.cuda.stream(s_in):
            for o in range(0, src.numel(), chunk):
                m = min(chunk, src.numel() - o)
                d_in[:m].copy_(src[o:o + m], non_blocking=True)

    def d2h():
        with torch.cuda.stream(s_out):
            for o in range(0, dst.numel(), chunk):
                m = min(chunk, dst.numel() - o)
                dst[o:o + m].copy_(d_out[:m], non_blocking=True)

    def timed(*fns):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in fns:
            f()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0)

    timed(h2d, d2h)  # warm
    ms_in = min(timed(h2d) for _ in range(3))
    ms_out = min(timed(d2h) for _ in range(3))
    ms_both = min(timed(h2d, d2h) for _ in range(3))
    del d_in, d_out
    return {"link_gbs_h2d": src.numel() / ms_in / 1e6, "link_gbs_d2h": dst.numel() / ms_out / 1e6,
            "link_ms_both": ms_both, "link_ms_ideal": max(ms_in, ms_out),
            "link_method": "plain pinned cudaMemcpyAsync of the same bytes in 128 MB pieces, H2D and "
                           "D2H on two streams at once (best of 3); frac_of_link = that time / e2e time; "
                           "frac_of_link_ideal = the slower direction alone / e2e time (a full-duplex "
                           "link at the measured one-way rates)"}


def run_reference(args):
    import synth

    rank, world, _ = dist()
    if rank != 0:
        return
    ws = synth.station_batch(seed=0, n_times=20)
    import oracle

    cores = os.cpu_count() or 1
    vis = ws.vis("cpu").reshape(-1).numpy()
    layers = ws.layers()
    for _ in range(args.warmup):
        oracle.image_batch(ws.ant_xyz, layers, vis, "fft", n_threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.image_batch(ws.ant_xyz, layers, vis, "fft", n_threads=cores)
    el = time.perf_counter() - t0
    value = args.steps * len(layers) / el
    sample = (f"each step: 20 time steps x 32 channels ({len(layers)} images of 180^2, "
              "uniform) of the workload; FP64 C oracle, FFT route, OpenMP over images")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": STATION_WORKLOAD, "layers_per_gpu": 32000, "n_px": 180,
                   "baselines": ws.n_baselines,
                   "parallelism": f"replicas x{world} (rank 0 times the oracle)",
                   "sample_layers_per_step": len(layers)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_2405_13478_gb300 import binding, build

    rank, world, local = dist()
    torch.cuda.set_device(local)
    rank, world, local, pg = init_replicas("nccl")
    if rank == 0:
        build.build()
    if pg:
        pg.barrier()
    lib = binding.lib()  # noqa: F841  (fails loudly when the library is missing)

    # Each rank images its own 1000 x 32 batch (weak scaling, no data-path collective).
    ws = rank_workload(rank, args.n_times or 1000)
    layers = ws.layers()
    L = len(layers)
    B = ws.n_baselines
    N = 180
    layers, total = binding.layer_out_offsets(layers)
    larr = binding.layer_array([d["n_px"] for d in layers], [d["weighting"] for d in layers],
                               [d["freq_hz"] for d in layers], [d["delta_u"] for d in layers],
                               [d["vis_offset"] for d in layers], [d["out_offset"] for d in layers])
    vis = ws.vis("cuda").reshape(-1)                     # complex64, 8.36 GB at 1000 steps
    images = torch.empty(total, dtype=torch.float32, device="cuda")
    wsum = torch.empty(L, dtype=torch.float32, device="cuda")
    d_xyz = torch.as_tensor(ws.ant_xyz).cuda()
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        plan = binding.Plan(ctx, d_xyz, larr)     # uv, cells, weight tables (one host sync)
        if ev:
            ev[0].record(stream)
        plan.image(vis, images, wsum)              # gridding + transform
        if ev:
            ev[1].record(stream)
        plan.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for k in range(args.steps):
        step(kev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), pg, "cuda")
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    value = whole_job_rate(L, world, args.steps, ms)
    err = sampled_error(ctx, ws, d_xyz, vis, images, layers) if rank == 0 else None
    variants = None
    if rank == 0 and not args.no_variants:
        variants = epilogue_variants(torch, binding, ctx, ws, d_xyz, larr, vis, images, wsum,
                                     layers, args.steps, args.warmup)

    # e2e: the host-buffer entry point (pinned host memory), copies inside the
    # timed region, overlapped with the kernels by the library's pipeline
    h_vis = torch.empty(vis.shape, dtype=vis.dtype, pin_memory=True)
    h_vis.copy_(vis)
    h_img = torch.empty(images.shape, dtype=images.dtype, pin_memory=True)
    h_ws = torch.empty(wsum.shape, dtype=wsum.dtype, pin_memory=True)
    torch.cuda.synchronize()
    del vis
    if pg:
        pg.barrier()
    ctx.image_batch_host(ws.ant_xyz, larr, h_vis, h_img, h_ws)   # warm-up (staging pool)
    torch.cuda.synchronize()
    calls_ms = []
    for _ in range(args.e2e_steps):
        t_call = time.perf_counter()
        ctx.image_batch_host(ws.ant_xyz, larr, h_vis, h_img, h_ws)
        calls_ms.append(1e3 * (time.perf_counter() - t_call))
        print(f"e2e call: {calls_ms[-1]:.1f} ms", file=sys.stderr, flush=True)
    # the median call: the host of a shared GPU machine occasionally stalls one call
    e2e_ms = max_over_ranks(statistics.median(calls_ms), pg, "cuda")
    e2e_value = whole_job_rate(L, world, 1, e2e_ms)
    h2d_bytes = int(h_vis.numel() * 8)
    d2h_bytes = int(images.numel() * 4 + wsum.numel() * 4)
    link = link_ceiling(torch, h_vis, h_img) if rank == 0 else None
    del h_vis

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(synth.station_batch(seed=0, n_times=20))

    if rank == 0:
        peak, peak_kind = measured_peaks()
        bytes_per_layer = B * 8 + N * N * 4          # vis in + image out (algorithmic)
        kms = statistics.mean(kern_ms)
        achieved = L * bytes_per_layer / (kms / 1e3) / 1e9
        rec = ncu_record()
        tr = None if rec is None else float(rec["dram_bytes_per_layer"])
        # FP32 arithmetic of the same kernel against the measured FMA peak
        rows = support_rows(ws.ant_xyz, ws.freqs_hz, float(ws.delta_u[0]), N)
        flops_layer = statistics.mean(image_flops(N, r, 2 * B) for r in rows)
        try:
            p32, p64 = alu_peak()
        except Exception:
            p32 = p64 = None
        alu = {"unit": "TFLOP/s", "flops_per_image": flops_layer,
               "convention": "5 n log2 n per complex n-point FFT on the support rows and the n/2 paired "
                             "columns, plus 2 flops per gridded entry",
               "achieved": L * flops_layer / (kms / 1e3) / 1e12, "peak": p32,
               "peak_kind": "measured (blink_probe_fma_peak, FP32 FMA)", "fp64_peak": p64}
        alu["frac"] = alu["achieved"] / p32 if p32 else None
        if rec is not None and rec.get("fp32_flops_per_layer"):
            alu["executed_fp32_flops_per_image"] = rec["fp32_flops_per_layer"]
            alu["executed_achieved"] = L * rec["fp32_flops_per_layer"] / (kms / 1e3) / 1e12
            alu["executed_frac"] = alu["executed_achieved"] / p32 if p32 else None
        variants = variants or {}
        if not args.no_variants:
            del images, wsum
            torch.cuda.empty_cache()
            variants["workloads"] = secondary_workloads(torch, binding, ctx, min(args.steps, 20),
                                                        args.warmup)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": STATION_WORKLOAD,
                       "layers_per_gpu": L, "n_px": N, "baselines": B,
                       "l2": "inputs larger than L2 (8.36 GB of visibilities per GPU)",
                       "parallelism": f"replicas x{world} (independent layers, no collective)"},
            "gvis_per_s": value * B / 1e9,
            "err_vs_oracle": err,
            "variants": variants,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": (tr * L) if tr is not None else None,
                         "kernel": KERNEL, "kernel_ms": kms,
                         "algorithmic_bytes_per_launch": L * bytes_per_layer,
                         "alu": alu},
            "cpu_baseline": cpu,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "method": f"median of {args.e2e_steps} timed calls of blink_image_batch_host "
                              "(pinned host buffers) after one warm-up call",
                    "calls_ms": [round(c, 2) for c in calls_ms],
                    "h2d_bytes_per_step": h2d_bytes,
                    "d2h_bytes_per_step": d2h_bytes},
            "gpu_launches": 7 * args.steps,  # 6 table kernels + 1 fused image kernel per step
        }
        if link:
            out["e2e"].update(link)
            out["e2e"]["frac_of_link"] = link["link_ms_both"] / e2e_ms
            out["e2e"]["frac_of_link_ideal"] = link["link_ms_ideal"] / e2e_ms
        print(json.dumps(out), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()


# --------------------------------------------------------------------------
# Secondary workloads: the single-image latency, the uneven mixed-size batch,
# the tensor-core transform modes and the differentiable path.  Each measure_*
# returns a dict; the default run reports them (at reduced time steps) under
# "variants" of its line, and `--workload NAME` prints a full-size line of its
# own with the same schema.  Single GPU (rank 0 only).
def _setup_single():
    import torch

    from paper_2405_13478_gb300 import binding, build

    rank, world, local = dist()
    if rank != 0:
        return None
    torch.cuda.set_device(local)
    build.build()
    return torch, binding, binding.Context(local)


def _time_steps(torch, step, steps, warmup):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, clocks.stop()


def _line(args, metric_value, ms, config, clk, extra):
    out = {"metric": METRIC, "value": metric_value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, "clocks": clk}
    out.update(extra)
    print(json.dumps(out), flush=True)


def _sample_error(torch, ws, layers, vis_flat, out, picks):
    import numpy as np

    import oracle

    B = ws.n_baselines
    sub = [dict(layers[k], vis_offset=i * B) for i, k in enumerate(picks)]
    v = torch.stack([vis_flat[layers[k]["vis_offset"]:layers[k]["vis_offset"] + B] for k in picks])
    want, _ = oracle.image_batch(ws.ant_xyz, sub, v.cpu().reshape(-1).numpy(), "fft")
    worst = 0.0
    for k, w in zip(picks, want):
        o, n = layers[k]["out_offset"], layers[k]["n_px"]
        g = out[o:o + n * n].cpu().numpy().reshape(n, n)
        worst = max(worst, float(np.abs(g - w).max() / np.abs(w).max()))
    return worst


def _hbm_roofline(nbytes, ms, kernel, per_unit=None):
    peak, kind = measured_peaks()
    gbs = nbytes / (ms / 1e3) / 1e9
    out = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
           "peak_kind": kind, "traffic": None, "kernel": kernel, "algorithmic_bytes_per_launch": nbytes}
    if per_unit:
        out["algorithmic_bytes_per_image"] = per_unit
    return out


def _layer_array(binding, layers):
    return binding.layer_array([d["n_px"] for d in layers], [d["weighting"] for d in layers],
                               [d["freq_hz"] for d in layers], [d["delta_u"] for d in layers],
                               [d["vis_offset"] for d in layers], [d["out_offset"] for d in layers])


def measure_single(torch, binding, ctx, steps, warmup):
    """One 256^2 image of a 128-antenna 3 km array: latency of a whole call."""
    import synth

    ws = synth.single_image(seed=0)
    layers, total = binding.layer_out_offsets(ws.layers())
    vis = ws.vis("cuda").reshape(-1)
    out = torch.empty(total, device="cuda")
    d_xyz = torch.as_tensor(ws.ant_xyz).cuda()
    ms, clk = _time_steps(torch, lambda: ctx.image_batch(d_xyz, layers, vis, out), steps, warmup)
    plan = ctx.plan(d_xyz, layers)
    ms_k, _ = _time_steps(torch, lambda: plan.image(vis, out), steps, warmup)
    err = _sample_error(torch, ws, layers, vis, out, [0])
    plan.close()
    return {"workload": "single 256^2 image, 128 antennas in a 3 km disk, 8128 baselines, 160 MHz, "
                        "natural weighting (latency of one blink_image_batch call; no roofline claim)",
            "images_per_s": 1e3 / ms, "ms_per_step": ms, "latency_us": ms * 1e3,
            "latency_plan_cached_us": ms_k * 1e3, "err_vs_oracle": err, "clocks": clk,
            "l2": "inputs fit in L2 (latency of a single call)"}


def measure_uneven(torch, binding, ctx, n_t, steps, warmup):
    """Uneven batch: 768 channels x n_t steps, 128^2..1024^2 by channel group."""
    import synth

    ws = synth.uneven_batch(seed=0, n_times=n_t)
    layers, total = binding.layer_out_offsets(ws.layers())
    larr = _layer_array(binding, layers)
    free, _ = torch.cuda.mem_get_info()
    if total * 4 + ws.n_layers * ws.n_baselines * 8 > 0.85 * free:
        raise SystemExit(f"uneven with {n_t} time steps does not fit in device memory; pass --n-times")
    vis = ws.vis("cuda").reshape(-1)
    out = torch.empty(total, device="cuda")
    d_xyz = torch.as_tensor(ws.ant_xyz).cuda()
    ms, clk = _time_steps(torch, lambda: ctx.image_batch(d_xyz, larr, vis, out), steps, warmup)
    t_s = min(20, n_t - 1)  # the pulse reaches the top channel at step 20
    picks = [t_s * 768 + c for c in (0, 100, 200, 300, 767)]
    err = _sample_error(torch, ws, layers, vis, out, picks)
    L = len(layers)
    # the same batch through a reused plan: default kernels, autotuned kernels,
    # and the autotuned launches replayed as one CUDA graph
    plan = ctx.plan(d_xyz, larr)
    ms_plan, _ = _time_steps(torch, lambda: plan.image(vis, out), steps, warmup)
    plan.autotune(vis, out)
    ms_tuned, _ = _time_steps(torch, lambda: plan.image(vis, out), steps, warmup)
    plan.capture(vis, out)
    ms_graph, _ = _time_steps(torch, lambda: plan.replay(), steps, warmup)
    err_graph = _sample_error(torch, ws, layers, vis, out, picks)
    tuning = plan.tuning()
    plan.close()
    nbytes = L * ws.n_baselines * 8 + total * 4
    peak, _ = measured_peaks()
    del vis, out
    return {"workload": f"uneven batch: 128 antennas in a 3 km disk, 768 channels x {n_t} steps, "
                        "images 128/256/512/1024 by channel group, dispersed pulse + noise",
            "layers": L, "image_floats": total, "images_per_s": L / (ms / 1e3), "ms_per_step": ms,
            "err_vs_oracle": err, "clocks": clk,
            "l2": f"inputs larger than L2 ({total * 4 / 1e9:.1f} GB of images per step)",
            "roofline": _hbm_roofline(nbytes, ms, "whole step, plan build included (all sizes)"),
            "planned": {"images_per_s": L / (ms_plan / 1e3), "ms_per_step": ms_plan,
                        "hbm_frac": nbytes / (ms_plan / 1e3) / 1e9 / peak},
            "autotuned": {"images_per_s": L / (ms_tuned / 1e3), "ms_per_step": ms_tuned,
                          "hbm_frac": nbytes / (ms_tuned / 1e3) / 1e9 / peak},
            "autotuned_graph": {"images_per_s": L / (ms_graph / 1e3), "ms_per_step": ms_graph,
                                "err_vs_oracle": err_graph,
                                "hbm_frac": nbytes / (ms_graph / 1e3) / 1e9 / peak},
            "tuning": [{"n_px": n, "path": ["default", "scheduled fused", "atomic fused",
                                            "persistent queue", "waves"][p_], "scratch_bytes": w}
                       for n, p_, w in tuning]}


def measure_station512(torch, binding, ctx, n_t, steps, warmup):
    """Station 512^2 batch: FP32 FFT against the tensor-core modes."""
    import synth

    ws = synth.station_512(seed=0, n_times=n_t)
    layers, total = binding.layer_out_offsets(ws.layers())
    larr = _layer_array(binding, layers)
    vis = ws.vis("cuda").reshape(-1)
    out = torch.empty(total, device="cuda")
    d_xyz = torch.as_tensor(ws.ant_xyz).cuda()
    L = len(layers)
    per_image = ws.n_baselines * 8 + 512 * 512 * 4
    peak, _ = measured_peaks()
    modes = {"fft_fp32": 0x00, "bf16": 0x10, "bf16x3": 0x20, "fp16": 0x30, "fp16x3": 0x40}
    res, clk0 = {}, None
    for name, flag in modes.items():
        def step(flag=flag):
            plan = binding.Plan(ctx, d_xyz, larr)
            plan.image(vis, out, None, flag)
            plan.close()
        ms, clk = _time_steps(torch, step, steps, warmup)
        clk0 = clk0 or clk
        err = _sample_error(torch, ws, layers, vis, out, [0, L // 2, L - 1])
        res[name] = {"images_per_s": L / (ms / 1e3), "ms_per_step": ms, "err_vs_oracle": err,
                     "hbm_frac": L * per_image / (ms / 1e3) / 1e9 / peak}
    # tensor work of the split mode: 3 products of pass 2 (512 x 512 x 2 Rp,
    # Rp = 48) and of pass 1 (2 x 512 columns x 2 Kc, Kc = 96, per 64-row half
    # of a 128-row tile)
    flops = 3 * (2 * 512 * 512 * 96 + 2 * 64 * 1024 * 192) * L
    tf = flops / (res["bf16x3"]["ms_per_step"] / 1e3) / 1e12
    try:
        peak_tf = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        kind = "measured"
    except Exception:
        peak_tf, kind = 1900.0, "fallback"
    del vis, out
    return {"workload": f"station: 256 antennas, 32640 baselines, {n_t} steps x 16 channels, 512^2 "
                        "images, natural weighting, 50 sources 1e-3..10 Jy + noise",
            "layers": L, "images_per_s": res["fft_fp32"]["images_per_s"],
            "ms_per_step": res["fft_fp32"]["ms_per_step"], "err_vs_oracle": res["fft_fp32"]["err_vs_oracle"],
            "clocks": clk0, "l2": f"inputs larger than L2 ({total * 4 / 1e9:.1f} GB of images per step)",
            "modes": res,
            "roofline": _hbm_roofline(L * per_image, res["fft_fp32"]["ms_per_step"],
                                      "whole FP32 FFT step, plan build included", per_image),
            "tensor_bf16x3": {"achieved": tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf,
                              "peak_kind": kind, "algorithmic_flops_per_step": flops,
                              "note": "the split-precision GEMMs at 512^2 are below the ridge point "
                                      "(about 115 flop/byte): HBM is their bound"}}


def measure_gains(torch, binding, ctx, n_t, steps, warmup):
    """Differentiable 1024^2 imaging with antenna gains: forward + backward."""
    import numpy as np

    import synth
    from paper_2405_13478_gb300 import autograd

    ws = synth.station_gains(seed=0, n_times=n_t)
    B, n_ant = ws.n_baselines, ws.n_ant
    model_c = torch.as_tensor(synth.model_vis(ws.ant_xyz, ws.freqs_hz, ws.sky).astype(np.complex64)).cuda()
    model = model_c.unsqueeze(0).expand(n_t, -1, -1).contiguous().reshape(-1)
    layers, total = binding.layer_out_offsets(ws.layers())
    d_xyz = torch.as_tensor(ws.ant_xyz).cuda()
    plan = ctx.plan(d_xyz, layers)
    target = autograd.dirty_images(model, plan, total).detach()
    g0 = torch.as_tensor(ws.gains.astype(np.complex64)).cuda()
    box = {}

    def step():
        g = g0.clone().requires_grad_(True)
        vis = autograd.apply_gains(g, model, ctx, n_ant, layers)
        # per-layer |image - model image|^2 from the imaging kernels (the
        # library's reference-subtraction epilogue sums the squares as it
        # stores the residual); the backward hands the stored residual and a
        # per-layer factor to the adjoint, so no image-sized torch op runs
        loss = autograd.image_sqnorm(vis, plan, total, ref=target).sum()
        loss.backward()
        box["vis"] = vis
        return g.grad

    ms, clk = _time_steps(torch, step, steps, warmup)
    L = len(layers)
    img = autograd.dirty_images(box["vis"].detach(), plan, total)  # the forward images, for the error check
    err = _sample_error(torch, ws, layers, box["vis"].detach(), img.detach(), [0, L - 1])
    n2 = 1024 * 1024
    # what the step has to move: the model visibilities and the model image in
    # (the visibilities, the residual image, its gradient and the visibility
    # gradient are intermediates: the residual is summed and column-transformed
    # where it is formed); an unfused step also writes and re-reads the image
    # and its gradient and the visibility gradient
    per_image = 8 * B + 4 * n2
    unfused = 8 * B + 4 * n2 + 4 * n2 + 8 * B   # vis in, image out, dL/dI in, dL/dV out
    plan.close()
    return {"workload": f"station: 256 antennas, {n_t} steps x 8 channels, 1024^2 images, gains on a "
                        "20-source model, loss = sum (image - model image)^2, forward + backward",
            "layers": L, "images_per_s": L / (ms / 1e3), "ms_per_step": ms, "clocks": clk,
            "err_vs_oracle": err, "err_what": "forward images vs the oracle (gradients: GPU tests)",
            "l2": f"inputs larger than L2 ({2 * total * 4 / 1e9:.2f} GB of images and image gradients)",
            "roofline": dict(_hbm_roofline(L * per_image, ms, "whole forward + backward step", per_image),
                             unfused_bytes_per_image=unfused,
                             frac_of_unfused_bytes=L * unfused / (ms / 1e3) / 1e9 / measured_peaks()[0])}


def _standalone(args, fn, n_default, **kw):
    env = _setup_single()
    if env is None:
        return
    torch, binding, ctx = env
    if n_default is None:
        d = fn(torch, binding, ctx, args.steps, args.warmup)
    else:
        d = fn(torch, binding, ctx, args.n_times or n_default, args.steps, args.warmup)
    ctx.close()
    value, ms, clk = d.pop("images_per_s"), d.pop("ms_per_step"), d.pop("clocks")
    cfg = {"workload": d.pop("workload")}
    for k in ("layers", "image_floats", "l2"):
        if k in d:
            cfg[k] = d.pop(k)
    _line(args, value, ms, cfg, clk, d)


def run_single(args):
    _standalone(args, measure_single, None)


def run_uneven(args):
    _standalone(args, measure_uneven, 100)


def run_station512(args):
    _standalone(args, measure_station512, 2000)


def run_gains(args):
    _standalone(args, measure_gains, 100)


def secondary_workloads(torch, binding, ctx, steps, warmup):
    """The four secondary workloads at reduced time steps (device memory and
    run time of the default bench); full sizes: --workload NAME."""
    out = {}
    for name, fn, n_t in (("single", measure_single, None), ("uneven", measure_uneven, 10),
                          ("station512", measure_station512, 200), ("gains", measure_gains, 20)):
        try:
            d = fn(torch, binding, ctx, steps, warmup) if n_t is None else fn(torch, binding, ctx, n_t, steps, warmup)
            if n_t is not None:
                d["reduced"] = f"{n_t} time steps (full size: bench.py --workload {name})"
            out[name] = d
        except Exception as e:  # report, never hide, a failed variant
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "station":
        run_ours(args)
    else:
        {"single": run_single, "uneven": run_uneven, "station512": run_station512, "gains": run_gains}[args.workload](args)


if __name__ == "__main__":
    main()
