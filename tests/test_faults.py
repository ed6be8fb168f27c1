"""Failure paths tested on the host, with no GPU fault (no device waits exist to time out):
a missing or foreign checkpoint file (host-only), a truncated checkpoint, a device
allocation that fails at every allocation point of context creation (the
MUCA_TEST_FAIL_ALLOC hook: MUCA_ERR_OOM and no device memory left behind), and the
per-iteration metric lines of MUCA_METRICS_LOG."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


def test_checkpoint_missing_or_foreign_is_io_error(muca, tmp_path):
    """muca_load checks the file before any device work."""
    m = muca
    with pytest.raises(m.MucaError) as ei:
        m.Muca.load(str(tmp_path / "nothing.ckpt"))
    assert ei.value.code == m._muca.MUCA_ERR_IO
    bad = tmp_path / "foreign.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(200))
    with pytest.raises(m.MucaError) as ei:
        m.Muca.load(str(bad))
    assert ei.value.code == m._muca.MUCA_ERR_IO
    short = tmp_path / "short.ckpt"
    short.write_bytes(b"MUCACKP1")   # the header cut after its magic
    with pytest.raises(m.MucaError) as ei:
        m.Muca.load(str(short))
    assert ei.value.code == m._muca.MUCA_ERR_IO


@pytest.mark.gpu
def test_truncated_checkpoint_is_io_error(muca, tmp_path):
    m = muca
    path = str(tmp_path / "run.ckpt")
    with m.Muca(m.MUCA_ISING, 16, 2, 64, 7) as g:
        g.iterate(5)
        g.update_weights()
        g.save(path)
    size = os.path.getsize(path)
    for cut in (size - 1, size // 2, 300):
        with open(path, "rb") as fh:
            data = fh.read()[:cut]
        tpath = str(tmp_path / ("cut%d.ckpt" % cut))
        with open(tpath, "wb") as fh:
            fh.write(data)
        with pytest.raises(m.MucaError) as ei:
            m.Muca.load(tpath)
        assert ei.value.code == m._muca.MUCA_ERR_IO, cut
    # the intact file still loads
    h = m.Muca.load(path)
    assert h.iteration == 1
    h.close()


def _ckpt_offsets(m, path, model, L, p, n_bins, n_thr):
    """Byte offsets of the lattice and of E in a checkpoint file (format version 3:
    the header, then the lattice as row words x p chains, E, M, the two count words
    per chain, then the per-bin arrays: ln W, P, production ln W, the n_thr
    thresholds, H and the three production sums)."""
    lat_words = L * ((L + 31) // 32 if model == m.MUCA_ISING else (L + 3) // 4)
    body = 4 * lat_words * p + 4 * p + 4 * p + 16 * p + 8 * n_bins * 3 + 4 * n_thr + 8 * n_bins + 24 * n_bins
    header = os.path.getsize(path) - body
    assert 0 < header < 512, header
    return header, header + 4 * lat_words * p


@pytest.mark.gpu
@pytest.mark.parametrize("model,L,q", [(0, 16, 2), (1, 12, 8)])
def test_inconsistent_checkpoint_is_io_error(muca, tmp_path, model, L, q):
    """A checkpoint whose spins lie outside the model, or whose energies are not those
    of its spins, is refused with MUCA_ERR_IO before any sweep can walk a chain off the
    weight table."""
    m = muca
    p = 37
    path = str(tmp_path / "ok.ckpt")
    with m.Muca(model, L, q, p, 5) as g:
        g.iterate(3)
        g.update_weights()
        g.save(path)
        n_bins, n_thr = g.n_bins, g.get_thresholds().size
    lat0, e0 = _ckpt_offsets(m, path, model, L, p, n_bins, n_thr)
    data = bytearray(open(path, "rb").read())
    cases = {}
    bad = bytearray(data)
    bad[e0 + 4 * 3] ^= 0x04            # chain 3's E off by a multiple of the level spacing
    cases["energy"] = bad
    bad = bytearray(data)
    if model == m.MUCA_POTTS:
        bad[lat0 + 4 * 5] = 9           # a Potts spin of chain 5 outside 0..q-1
    else:
        # a bit past site L - 1 in the last word of row 0 of chain 5 (L = 16 < 32)
        bad[lat0 + 4 * 5 + 3] |= 0x80
    cases["spin"] = bad
    for name, blob in cases.items():
        bpath = str(tmp_path / (name + ".ckpt"))
        open(bpath, "wb").write(bytes(blob))
        with pytest.raises(m.MucaError) as ei:
            m.Muca.load(bpath)
        assert ei.value.code == m._muca.MUCA_ERR_IO, name
    h = m.Muca.load(path)
    h.close()


_OOM_CHILD = r"""
import ctypes, sys
sys.path.insert(0, %r)
import paper_1212_3975_gb300 as m
cudart = ctypes.CDLL("libcudart.so.13")
free, total = ctypes.c_size_t(), ctypes.c_size_t()
def free_mem():
    cudart.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total))
    return free.value
cudart.cudaFree(None)
f0 = free_mem()
h = ctypes.c_void_p()
rc = m.lib().muca_init(ctypes.byref(h), 0, 32, 2, 64, 1, None, None)
f1 = free_mem()
print(rc, f0 - f1)
"""


@pytest.mark.gpu
@pytest.mark.parametrize("k", [1, 2, 8, 15, 16])
def test_allocation_failure_cleans_up(muca, k):
    """The k-th of the 16 allocations of context creation (15 device buffers, then the
    pinned statistics buffer) fails: MUCA_ERR_OOM, nothing leaked."""
    env = dict(os.environ, MUCA_TEST_FAIL_ALLOC=str(k))
    out = subprocess.run([sys.executable, "-c", _OOM_CHILD % ROOT], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    rc, leaked = (int(x) for x in out.stdout.split())
    assert rc == muca._muca.MUCA_ERR_OOM
    assert leaked == 0


@pytest.mark.gpu
def test_allocation_hook_beyond_the_last_allocation(muca):
    """With the hook set past the last allocation, creation succeeds."""
    env = dict(os.environ, MUCA_TEST_FAIL_ALLOC="17")
    out = subprocess.run([sys.executable, "-c", _OOM_CHILD % ROOT], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert int(out.stdout.split()[0]) == 0


_METRICS_CHILD = r"""
import sys
sys.path.insert(0, %r)
import paper_1212_3975_gb300 as m
g = m.Muca(m.MUCA_ISING, 8, 2, 16, 3)
for _ in range(3):
    g.iterate(50)
    g.update_weights()
g.close()
"""


@pytest.mark.gpu
def test_metrics_log_lines(muca, tmp_path):
    log = str(tmp_path / "metrics.jsonl")
    env = dict(os.environ, MUCA_METRICS_LOG=log)
    out = subprocess.run([sys.executable, "-c", _METRICS_CHILD % ROOT], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    lines = [json.loads(x) for x in open(log)]
    assert [x["iteration"] for x in lines] == [1, 2, 3]
    for x in lines:
        assert x["total"] == 16 * 50 * 64 and 0 <= x["lo"] <= x["hi"] <= 64
        assert x["attempts_per_ns"] > 0 and x["covered"] in (0, 1)
