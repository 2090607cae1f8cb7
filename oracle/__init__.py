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

Parity pins for all of the above live in ``tests/test_oracle_pins.py``; each function
is pinned to something other than itself:

* ``apply_sym``, ``sublattice_tables``, ``representatives``: the integers the paper
  prints for its two- and three-sublattice worked examples (``tests/golden/``), and
  the orbit minimum and stabiliser order found by repeated shifts (brute force).
* ``basis``: the character-projection count (closed form), strict order, and the
  16 momentum sectors of the 16-site chain summing to C(16, 8).
* ``columns`` / ``hamiltonian`` / ``rows``: the literal Eq. 2 projection in the 2^N
  space (real and complex sectors, anisotropy); planted mistakes (character instead
  of its conjugate, missing or inverted norm ratio, exchange sign, S^z S^z sign and
  factor, a dropped term) each fail it; rows equal matrix rows.
* ``projected_hamiltonian`` / ``full_hamiltonian``: the 4-site ring (E0 = -2J), the
  XX chain against free fermions (E0 = -J / sin(pi/N)), the union of momentum spectra
  equal to the unsymmetrised spectrum, C4v sector spectra inside it.
* ``dimension_formula``: the enumerated bases above, and the sum over sectors.
* ``lanczos``: dense diagonalisation, and the unsymmetrised 16-site chain.
* spin-flip sectors: dimensions adding up to the unflipped sector and the literal
  projection with the flip.
"""
from .core import *  # noqa: F401,F403
from .core import build  # noqa: F401
