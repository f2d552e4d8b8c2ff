"""The in-register DFT codelets of the CUDA transform (blink_fft.cuh: radix
2/3/4/5 butterflies, Cooley-Tukey and prime-factor splits), compiled for the
host and checked against the direct DFT sum (Sec. 5.2.2 defines the transform
as the inverse DFT of the grid) for every codelet length the size plans use,
in both directions."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2405_13478_gb300", "csrc")


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.mark.skipif(_nvcc() is None, reason="needs nvcc to compile the codelet header")
def test_codelets_match_the_direct_dft():
    d = tempfile.mkdtemp(prefix="codelets_")
    try:
        exe = os.path.join(d, "fft_codelet_check")
        subprocess.run([_nvcc(), "-O2", "-std=c++17", "--expt-relaxed-constexpr", f"-I{CSRC}",
                        os.path.join(HERE, "fft_codelet_check.cu"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    finally:
        shutil.rmtree(d, ignore_errors=True)
