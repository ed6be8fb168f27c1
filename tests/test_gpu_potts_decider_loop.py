"""The 8-Potts decider-loop replica (tests/gpu_potts_decider_loop.cu) builds and runs on
one warp per block and prints the cycles per site of the slot decider's loop alone: the
chain-latency bound of the 8-Potts sweeps that bench.py reports."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_potts_decider_loop_replica():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "potts_decider_loop")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "gpu_potts_decider_loop.cu")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    m = re.search(r"potts decider loop: ([0-9.]+) cycles/site", out)
    assert m, out
    print(out.strip())
    assert 5.0 < float(m.group(1)) < 400.0, out
