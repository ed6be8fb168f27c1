"""The decider-loop replica (tests/gpu_decider_loop.cu) builds and runs: it gives the
cycles per attempt of the Ising decider's loop alone on one warp, the C_crit of the
chain-latency bound that bench.py reports."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_decider_loop_replica():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "decider_loop")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "gpu_decider_loop.cu")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    vals = {int(m.group(1)): float(m.group(2)) for m in re.finditer(r"mode (\d+) \(.*?\): ([0-9.]+)", out)}
    assert set(vals) == set(range(13)), out
    assert all(2.0 < v < 500.0 for v in vals.values()), out
    # the accept chain alone is the shortest, the full loop among the longest; the
    # byte-parallel loop is no slower than the per-site one
    assert vals[5] < vals[3] < vals[0]
    assert vals[10] <= vals[0] * 1.02
