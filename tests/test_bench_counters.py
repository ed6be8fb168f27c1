"""The ncu counters bench.py builds its issue fractions on were measured on the current
sweep kernel sources (each carries the hash of ws_bodies.cuh, sweep_ws.cu and
sweep_kernels.cu it was measured on; a stale counter is reported as null).  A change to
those sources needs a new capture: this test says so on the CPU, before a GPU run."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_counters_match_kernel_sources():
    import bench
    current = bench.sweep_source_sha16()
    stale = [k for k in bench.COUNTERS if not bench.counters(k)["matches_source"]]
    assert not stale, "re-capture %s with ncu: the sweep sources are now %s" % (stale, current)


def test_profiles_cite_the_same_sources():
    import bench
    current = bench.sweep_source_sha16()
    for name in ("ising_ws_sweep_L64_p1024.md", "ising_ws_compact_L64_p9728.md", "ising_ws_t16_L64_p14592.md",
                 "potts_ws_sweep_L32_p4096.md"):
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            assert current in fh.read(), name
