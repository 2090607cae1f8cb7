"""THE ORACLE -- test infrastructure, not product code.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  It shares no code with the CUDA path:
the only thing both sides read is the problem data from ``workloads``.

Contents (each function cites the passage of arXiv:1804.05028 it restates):

* ``ed_oracle.c`` (compiled by :func:`build`): brute-force representatives by
  applying every group element (Eqs. 3-4), the sector basis (Alg. 3's loop,
  single process), and columns of the symmetry-adapted Hamiltonian (Eq. 5 with
  the conjugation of Eq. 2).
* :mod:`oracle.core`: the same objects assembled into a sparse matrix, the
  character-projection dimension formula, the literal Eq. 2 projection in the
  full 2^N space, the unsymmetrised Hamiltonian, the sublattice tables of
  Eqs. 8-10 from their definitions, and a plain fp64 Lanczos.

Parity pins for all of the above live in ``tests/test_oracle_pins.py``.
"""
from .core import *  # noqa: F401,F403
from .core import build  # noqa: F401
