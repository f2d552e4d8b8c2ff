"""The baseline <-> antenna-pair map the CUDA kernels use (blink_pairs.cuh),
compiled for the host and checked exhaustively against the lexicographic
enumeration of the pairs (i < j): every baseline of arrays of 2..700 and 4096
antennas, and the row boundaries of arrays up to 65535 antennas."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2405_13478_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_baseline_pair_is_exact():
    d = tempfile.mkdtemp(prefix="pairs_")
    try:
        exe = os.path.join(d, "pair_index_check")
        subprocess.run(["g++", "-O2", "-std=c++17", f"-I{CSRC}",
                        os.path.join(HERE, "pair_index_check.cpp"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    finally:
        shutil.rmtree(d, ignore_errors=True)
