"""CPU oracle of the parallel multicanonical method (arXiv:1212.3975).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is independent of the
CUDA library: neither imports, links or calls the other.

Modules:
  muca_oracle.c  Philox4x32-10, Hamiltonians (Eqs. 3-4), infinite-temperature start,
                 typewriter MUCA sweeps with integer thresholds, per-chain histograms
                 and (E, M) records (Secs. 2-3, 5).
  weights.py     bins, accessible energies, thresholds from ln W (Eq. 1), the simple and
                 accumulated recursions, boundary correction, convergence (Secs. 2-3).
  reweight.py    Eq. 2 time-series reweighting in series and binned form, C_V (Sec. 5).
  muca.py        the whole procedure in the paper's order.

Parity status: every function is pinned by tests/test_oracle_*.py against exact
enumeration, an independent transfer matrix, Kaufman's finite-lattice partition
function, an independent Philox implementation, and invariants; Potts beyond the small
exactly enumerable lattices is pinned only by the invariants and the small-lattice
exactness (see the design notes).
"""
from . import sampler, weights, reweight  # noqa: F401
from .muca import MucaOracle  # noqa: F401
from .sampler import ISING, POTTS  # noqa: F401
