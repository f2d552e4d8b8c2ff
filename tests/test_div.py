"""The arithmetic of the cell assignment (blink_div.cuh), compiled for the
host: (1) the FP64 quotient by a reused divisor from its correctly rounded
reciprocal (two residual corrections after Markstein 1990), bit for bit
against IEEE division on 24 M quotients (wide exponent ranges, the baseline
/ wavelength / cell-size ranges of Sec. 5.2.1, exact and near-halfway
quotients); (2) the cell index of one axis (FP32 estimate, exact FP64 path
near cell edges) against its definition k = round(RN(RN(d / lambda) /
delta_u)) on 20 M offsets, most within 1e-12 to 1e-1 cells of a cell edge or
of the grid border, where a wrong rounding would move a visibility to the
neighbouring cell."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2405_13478_gb300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_division_and_cell_index_match_their_definitions():
    d = tempfile.mkdtemp(prefix="div_")
    try:
        exe = os.path.join(d, "div_check")
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", f"-I{CSRC}",
                        os.path.join(HERE, "div_check.cpp"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    finally:
        shutil.rmtree(d, ignore_errors=True)
