"""The multi-GPU form of the path is replicas: every rank images its own
layers, with no data-path collective; the bench only takes a barrier and the
max over ranks of the timed interval.  These tests run that host logic as two
gloo ranks on the CPU (no GPU involved)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench

    r, w, local, pg = bench.init_replicas("gloo")
    assert (r, w, local) == (rank, world, rank) and pg is not None
    pg.barrier()
    # each rank's own timed interval; the job's is the slowest
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, pg, "cpu")
    ws = bench.rank_workload(rank, n_times=2)
    vis = ws.vis("cpu", times=[0])[0, :2].numpy()
    res = {"rank": rank, "ms": ms, "layers": ws.n_layers, "ant0": ws.ant_xyz[0].tolist(),
           "vis_sum": float(np.abs(vis).sum()),
           "rate": bench.whole_job_rate(ws.n_layers, w, 20, ms)}
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    pg.barrier()
    pg.destroy_process_group()


def test_two_gloo_ranks_share_nothing_but_the_timing(tmp_path):
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    assert r[0]["ms"] == r[1]["ms"] == 15.0                 # max over ranks, on every rank
    assert r[0]["layers"] == r[1]["layers"] == 2 * 32      # same shape per rank (weak scaling)
    assert r[0]["ant0"] != r[1]["ant0"]                    # independent data per rank
    assert r[0]["vis_sum"] != r[1]["vis_sum"]
    # whole-job rate: both ranks' units over the slowest rank's time
    assert r[0]["rate"] == pytest.approx(2 * 64 * 20 / 0.015)


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.init_replicas("gloo") == (0, 1, 0, None)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    """The reference arm times the oracle on the host cores and prints one line
    with the same metric, unit and workload as the GPU arm."""
    sys.path.insert(0, ROOT)
    import bench

    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.STATION_WORKLOAD and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
