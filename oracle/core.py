"""Oracle implementation (test infrastructure only; see the package docstring)."""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp
from scipy.linalg import eigh_tridiagonal

__all__ = [
    "build", "lib", "OracleProblem", "representatives", "basis", "columns",
    "hamiltonian", "apply", "rows", "dimension_formula", "projected_hamiltonian",
    "full_hamiltonian", "lanczos", "sublattice_tables", "apply_sym", "max_threads",
    "StoredMatrix", "stored_matrix",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ed_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ed_oracle.c with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Prob(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("n_sym", ctypes.c_int32),
                ("phase_denom", ctypes.c_int32), ("n_bonds", ctypes.c_int32),
                ("n_classes", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("perm", ctypes.c_void_p), ("phase_num", ctypes.c_void_p),
                ("bonds", ctypes.c_void_p), ("bond_class", ctypes.c_void_p),
                ("J", ctypes.c_void_p), ("Jz", ctypes.c_void_p), ("flip", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER(_Prob)
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            L.or_apply_sym.argtypes = [P, ctypes.c_int, vp, i64, vp]
            L.or_representatives.argtypes = [P, vp, i64, vp, vp, vp, vp]
            L.or_basis.argtypes = [P, ctypes.c_int, vp, vp, i64]
            L.or_basis.restype = i64
            L.or_columns.argtypes = [P, vp, i64, vp, vp, vp, vp, vp]
            L.or_max_threads.restype = ctypes.c_int
            L.or_rows_slots.argtypes = [P, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp]
            L.or_csr_spmv.argtypes = [i64, vp, vp, vp, vp, vp, vp, i64]
            L.or_csr_spmv_complex.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, i64]
            _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().or_max_threads())


class OracleProblem:
    """Holds a workloads.Problem's arrays in C layout for the oracle library."""

    def __init__(self, p):
        self.p = p
        self._perm = np.ascontiguousarray(p.perm, dtype=np.int32)
        self._pnum = np.ascontiguousarray(p.phase_num, dtype=np.int32)
        self._bonds = np.ascontiguousarray(p.bonds, dtype=np.int32)
        self._bcls = np.ascontiguousarray(p.bond_class, dtype=np.int32)
        self._J = np.ascontiguousarray(p.J, dtype=np.float64)
        self._Jz = np.ascontiguousarray(p.Jz, dtype=np.float64)
        fl = getattr(p, "flip", None)
        self._flip = None if fl is None else np.ascontiguousarray(fl, dtype=np.uint8)
        self.s = _Prob(p.n_sites, p.n_sym, p.phase_denom, p.n_bonds, p.n_classes, 0,
                       self._perm.ctypes.data, self._pnum.ctypes.data,
                       self._bonds.ctypes.data, self._bcls.ctypes.data,
                       self._J.ctypes.data, self._Jz.ctypes.data,
                       None if self._flip is None else self._flip.ctypes.data)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _op(p):
    return p if isinstance(p, OracleProblem) else OracleProblem(p)


def apply_sym(p, g: int, states) -> np.ndarray:
    """g|s> for each s, one site at a time: (g s)[perm[g][p]] = s[p]."""
    op = _op(p)
    s = np.ascontiguousarray(states, dtype=np.uint64)
    out = np.empty_like(s)
    lib().or_apply_sym(op.ref, int(g), s.ctypes.data, s.size, out.ctypes.data)
    return out


def representatives(p, states):
    """Eqs. 3-4 by applying every symmetry: (rep, first minimising g, |Stab(rep)|, kept).

    ``kept`` is whether the representative survives the Eq. 2 projection (the
    sum of chi over its stabiliser is non-zero).
    """
    op = _op(p)
    s = np.ascontiguousarray(states, dtype=np.uint64)
    n = s.size
    rep = np.empty(n, np.uint64)
    g = np.empty(n, np.int32)
    st = np.empty(n, np.int32)
    kp = np.empty(n, np.int32)
    lib().or_representatives(op.ref, s.ctypes.data, n, rep.ctypes.data, g.ctypes.data,
                             st.ctypes.data, kp.ctypes.data)
    return rep, g, st, kp.astype(bool)


def basis(p):
    """Sorted representatives of the sector that survive the projection, and |Stab|.

    Alg. 3's loop on one process: every configuration with n_up up spins, in
    increasing int, kept when it is its own representative.
    """
    op = _op(p)
    L = lib()
    D = int(L.or_basis(op.ref, p.n_up if not isinstance(p, OracleProblem) else p.p.n_up,
                       None, None, 0))
    out = np.empty(D, np.uint64)
    stab = np.empty(D, np.int32)
    n_up = p.n_up if not isinstance(p, OracleProblem) else p.p.n_up
    D2 = int(L.or_basis(op.ref, n_up, out.ctypes.data, stab.ctypes.data, D))
    assert D2 == D
    return out, stab


def columns(p, states):
    """Diagonal and off-diagonal terms <j|H|i> of the columns i given by ``states``.

    Returns (diag[n], list of (rep_j array, complex value array)) per column.
    """
    op = _op(p)
    s = np.ascontiguousarray(states, dtype=np.uint64)
    n, nb = s.size, op.p.n_bonds
    diag = np.zeros(n)
    nt = np.zeros(n, np.int32)
    reps = np.zeros(n * nb, np.uint64)
    re = np.zeros(n * nb)
    im = np.zeros(n * nb)
    lib().or_columns(op.ref, s.ctypes.data, n, diag.ctypes.data, nt.ctypes.data,
                     reps.ctypes.data, re.ctypes.data, im.ctypes.data)
    reps = reps.reshape(n, nb)
    val = (re + 1j * im).reshape(n, nb)
    return diag, nt, reps, val


def hamiltonian(p, basis_states=None):
    """Sparse symmetry-adapted Hamiltonian H[j, i] = <j|H|i> on the oracle basis.

    The index of a representative is its position in the sorted basis (found by
    ``np.searchsorted`` on the whole array, Sec. IV's ``Basis`` without a prefix
    map).  Returns (H as scipy CSR, basis states, |Stab|).
    """
    op = _op(p)
    if basis_states is None:
        bs, stab = basis(op.p)
    else:
        bs, stab = basis_states
    D = bs.size
    diag, nt, reps, val = columns(op, bs)
    rows, cols, vals = [np.arange(D)], [np.arange(D)], [diag.astype(complex)]
    for i in range(D):
        k = nt[i]
        if k == 0:
            continue
        j = np.searchsorted(bs, reps[i, :k])
        if np.any(j >= D) or np.any(bs[np.minimum(j, D - 1)] != reps[i, :k]):
            raise AssertionError("kept representative missing from the basis")
        rows.append(j)
        cols.append(np.full(k, i))
        vals.append(val[i, :k])
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(D, D)).tocsr()
    H.sum_duplicates()
    if op.p.is_real():
        H = H.real.tocsr()
    return H, bs, stab


class StoredMatrix:
    """The symmetry-adapted Hamiltonian stored row by row (CSR), fp64.

    Row i holds H[i][j] = conj(<j|H|i>) (Hermitian H: the conjugate of column i), in
    bond order, duplicates not merged; the diagonal is kept apart.  Column indices are
    uint32 (D < 2^32).  The rows are kept as consecutive row blocks, each its own CSR
    (so that building never holds two copies of the entries).  ``matvec`` is the
    stored-matrix product of Sec. IV.
    """

    def __init__(self, D, blocks, diag, cplx):
        self.D, self.blocks, self.diag, self.cplx = D, blocks, diag, cplx

    @property
    def nnz(self) -> int:
        """Stored off-diagonal entries (one per surviving exchange term)."""
        return int(sum(b[2][-1] for b in self.blocks))

    def matvec(self, x):
        L = lib()
        dt = np.complex128 if self.cplx else np.float64
        x = np.ascontiguousarray(x, dtype=dt)
        y = np.empty(self.D, dt)
        es = y.itemsize
        for r0, r1, rowptr, col, vre, vim in self.blocks:
            yp = y.ctypes.data + r0 * es
            dp = self.diag.ctypes.data + r0 * 8
            if not self.cplx:
                L.or_csr_spmv(r1 - r0, rowptr.ctypes.data, col.ctypes.data, vre.ctypes.data,
                              dp, x.ctypes.data, yp, r0)
            else:
                L.or_csr_spmv_complex(r1 - r0, rowptr.ctypes.data, col.ctypes.data,
                                      vre.ctypes.data, vim.ctypes.data, dp, x.ctypes.data, yp, r0)
        return y


def stored_matrix(p, basis_states=None, chunk_rows: int = 1 << 20, progress=None) -> StoredMatrix:
    """Build the whole Hamiltonian of a sector as a :class:`StoredMatrix`.

    Every exchange term's representative comes from applying every group element
    (Eq. 4); its index is its position in the sorted oracle basis (binary search over
    the whole array); a representative absent from the basis is one the projection
    removes.  Rows are produced in blocks of ``chunk_rows`` (n_bonds slots per row,
    then compacted), so the peak extra memory is one block of slots.
    """
    op = _op(p)
    if basis_states is None:
        bs, stab = basis(op.p)
    else:
        bs, stab = basis_states
    bs = np.ascontiguousarray(bs, dtype=np.uint64)
    stab = np.ascontiguousarray(stab, dtype=np.int32)
    D, nb = bs.size, op.p.n_bonds
    if D >= 1 << 32:
        raise ValueError("dimension too large for uint32 column indices")
    cplx = not op.p.is_real()
    rows = min(chunk_rows, max(D, 1))
    s_col = np.zeros(rows * nb, np.uint32)
    s_re = np.zeros(rows * nb)
    s_im = np.zeros(rows * nb) if cplx else None
    s_nt = np.zeros(rows, np.int32)
    diag = np.zeros(D)
    blocks = []
    L = lib()
    for r0 in range(0, D, rows):
        r1 = min(D, r0 + rows)
        L.or_rows_slots(op.ref, bs.ctypes.data, stab.ctypes.data, D, r0, r1,
                        diag[r0:r1].ctypes.data, s_nt.ctypes.data, s_col.ctypes.data,
                        s_re.ctypes.data, None if s_im is None else s_im.ctypes.data)
        n = r1 - r0
        nt = s_nt[:n]
        keep = (np.arange(nb, dtype=np.int32)[None, :] < nt[:, None]).ravel()
        rowptr = np.zeros(n + 1, np.int64)
        rowptr[1:] = np.cumsum(nt, dtype=np.int64)
        blocks.append((r0, r1, rowptr, s_col[:n * nb][keep].copy(), s_re[:n * nb][keep].copy(),
                       s_im[:n * nb][keep].copy() if cplx else None))
        if progress:
            progress(r1, D)
    return StoredMatrix(D, blocks, diag, cplx)


def apply(p, x, H=None):
    """y = H x on the oracle basis (x indexed like the sorted oracle basis)."""
    if H is None:
        H, _, _ = hamiltonian(p)
    return H @ x


def rows(p, states, x_of):
    """y_i = (H x)_i for the representatives ``states`` (row sampling).

    Row i of the Hermitian H is the conjugate of column i, so
    y_i = diag_i x(s_i) + sum_k conj(<j_k|H|i>) x(s_{j_k}).  ``x_of`` maps an
    array of representatives to their coefficients (state-keyed vectors).
    """
    diag, nt, reps, val = columns(p, states)
    xi = x_of(np.asarray(states, dtype=np.uint64))
    y = diag * xi
    y = y.astype(complex) if np.iscomplexobj(val) and not _op(p).p.is_real() else y
    out = np.empty(len(states), dtype=complex)
    for r in range(len(states)):
        k = nt[r]
        acc = diag[r] * xi[r]
        if k:
            acc = acc + np.sum(np.conj(val[r, :k]) * x_of(reps[r, :k]))
        out[r] = acc
    return out.real if _op(p).p.is_real() else out


def _cycle_lengths(perm_row):
    seen = np.zeros(len(perm_row), bool)
    out = []
    for p in range(len(perm_row)):
        if not seen[p]:
            L, q = 0, p
            while not seen[q]:
                seen[q] = True
                q = perm_row[q]
                L += 1
            out.append(L)
    return out


def dimension_formula(p) -> int:
    """D_rho = (1/|G|) sum_g chi(g)^* F(g) (projection onto a 1-D irrep).

    F(g), the number of configurations with n_up up spins left unchanged by g,
    is the coefficient of x^n_up in prod over cycles c of g of (1 + x^|c|).  For
    an element that also reverses every spin, a fixed configuration alternates
    along every cycle, so F = 2^(number of cycles) when all cycles have even
    length (and then n_up = N/2 automatically), else 0.  Exact integer arithmetic
    on the phases; a closed form independent of any representative search.
    """
    N, n_up = p.n_sites, p.n_up
    flip = getattr(p, "flip", None)
    acc = 0j
    for g in range(p.n_sym):
        cyc = _cycle_lengths(p.perm[g])
        if flip is not None and flip[g]:
            F = (2 ** len(cyc)) if (all(L % 2 == 0 for L in cyc) and 2 * n_up == N) else 0
        else:
            poly = np.zeros(N + 1, dtype=object)
            poly[0] = 1
            for L in cyc:
                new = poly.copy()
                new[L:] = new[L:] + poly[:N + 1 - L]
                poly = new
            F = int(poly[n_up]) if 0 <= n_up <= N else 0
        ang = -2 * math.pi * int(p.phase_num[g]) / p.phase_denom
        acc += F * complex(math.cos(ang), math.sin(ang))
    val = acc / p.n_sym
    D = int(round(val.real))
    if abs(val.real - D) > 1e-6 or abs(val.imag) > 1e-6:
        raise AssertionError(f"projection count not an integer: {val}")
    return D


def _sector_states(N, n_up):
    s = np.arange(1 << N, dtype=np.uint64)
    pc = np.zeros(s.size, np.int64)
    for b in range(N):
        pc += ((s >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return s[pc == n_up]


def full_hamiltonian(p):
    """Unsymmetrised H (Eq. 21 with classes) on all configurations of the sector.

    Built straight from the bonds: S^z S^z diagonal, (S^+S^- + h.c.)/2 exchanging
    antiparallel spins.  Returns (CSR matrix, configurations).
    """
    N = p.n_sites
    states = _sector_states(N, p.n_up)
    idx = {int(s): i for i, s in enumerate(states)}
    r, c, v = [], [], []
    for i, s in enumerate(states.tolist()):
        d = 0.0
        for (a, b), cls in zip(p.bonds.tolist(), p.bond_class.tolist()):
            sa, sb = (s >> (N - 1 - a)) & 1, (s >> (N - 1 - b)) & 1
            if sa == sb:
                d += 0.25 * p.J[cls] * p.Jz[cls]
            else:
                d -= 0.25 * p.J[cls] * p.Jz[cls]
                t = s ^ (1 << (N - 1 - a)) ^ (1 << (N - 1 - b))
                r.append(idx[t]); c.append(i); v.append(0.5 * p.J[cls])
        r.append(i); c.append(i); v.append(d)
    H = sp.coo_matrix((v, (r, c)), shape=(len(states),) * 2).tocsr()
    H.sum_duplicates()
    return H, states


def projected_hamiltonian(p):
    """<j|H|i> from the literal Eq. 2 vectors in the configuration space.

    |s_rho> = (1/N_s) sum_g chi(g)^* g|s> is built as a dense vector for every
    representative of the oracle basis, normalised numerically (no closed form
    for N_s is used), and H is sandwiched between them.  Also returns the
    largest norm of a projected vector of a representative that the basis drops
    (it must vanish).  For N <= 12.
    """
    Hf, states = full_hamiltonian(p)
    idx = {int(s): i for i, s in enumerate(states)}
    bs, _ = basis(p)
    rep, g0, st, kp = representatives(p, states)
    chi = np.exp(2j * np.pi * p.phase_num / p.phase_denom)
    allrep = np.unique(rep)
    vecs = {}
    dropped = 0.0
    for r in allrep.tolist():
        v = np.zeros(len(states), complex)
        for g in range(p.n_sym):
            t = int(apply_sym(p, g, np.array([r], np.uint64))[0])
            v[idx[t]] += np.conj(chi[g])
        nrm = np.linalg.norm(v)
        if r in set(bs.tolist()):
            vecs[r] = v / nrm
        else:
            dropped = max(dropped, nrm)
    V = np.stack([vecs[int(s)] for s in bs], axis=1)
    Hp = V.conj().T @ (Hf @ V)
    return Hp, bs, dropped


def lanczos(matvec, v0, max_steps=200, tol=1e-13, min_steps=2):
    """Plain fp64 Lanczos with full re-orthogonalisation (two Gram-Schmidt sweeps).

    Returns (E0, alphas, betas, steps).  Stops when the lowest Ritz value moves
    by less than ``tol`` * max(1, |E0|) or on breakdown (beta < 1e-14 |alpha|).
    The tridiagonal eigenvalues come from scipy's ``eigh_tridiagonal``.
    """
    v = np.asarray(v0, dtype=complex if np.iscomplexobj(v0) else float)
    v = v / np.linalg.norm(v)
    V = [v]
    alphas, betas = [], []
    e_old = None
    for k in range(max_steps):
        w = matvec(V[-1])
        a = np.vdot(V[-1], w).real
        alphas.append(a)
        w = w - a * V[-1] - (betas[-1] * V[-2] if betas else 0)
        for _ in range(2):
            for u in V:
                w = w - np.vdot(u, w) * u
        b = np.linalg.norm(w)
        ev = eigh_tridiagonal(np.array(alphas), np.array(betas), eigvals_only=True)
        e0 = ev[0]
        if e_old is not None and k + 1 >= min_steps and abs(e0 - e_old) < tol * max(1, abs(e0)):
            return e0, np.array(alphas), np.array(betas), k + 1
        e_old = e0
        if b < 1e-14 * max(1.0, abs(a)) or len(alphas) >= len(v):
            return e0, np.array(alphas), np.array(betas), k + 1
        betas.append(b)
        V.append(w / b)
    return e_old, np.array(alphas), np.array(betas), max_steps


def sublattice_tables(p, n_sublat: int, X: int, sub: int):
    """Rep_X and Sym_X of a substate, from their definitions (Eqs. 8-10).

    G_X is every g that carries the labels of sublattice X onto those of
    sublattice 0 (the most significant block).  ``sub`` is the substate of
    sublattice X read as an n-bit integer (its first label most significant);
    g sub is read on sublattice 0 the same way.  Returns (Rep_X, sorted Sym_X).
    """
    N = p.n_sites
    n = N // n_sublat
    if getattr(p, "flip", None) is not None:
        raise NotImplementedError("sublattice tables of the worked examples: no spin flip")
    blk = lambda Y: set(range(Y * n, (Y + 1) * n))
    vals = {}
    for g in range(p.n_sym):
        if {int(p.perm[g, q]) for q in blk(X)} != blk(0):
            continue
        out = 0
        for k in range(n):
            if (sub >> (n - 1 - k)) & 1:
                tgt = int(p.perm[g, X * n + k])
                out |= 1 << (n - 1 - tgt)
        vals[g] = out
    rep = min(vals.values())
    return rep, sorted(g for g, v in vals.items() if v == rep)
