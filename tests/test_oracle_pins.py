"""Pins of the oracle against things other than itself (CPU only).

Each test fixes part of the oracle to something the paper or the mathematics
decides: the paper's two worked examples (integers printed in Sec. III), the
character-projection count of a sector (group theory, independent of any
representative search), the literal Eq. 2 vectors in configuration space,
spectra of the unsymmetrised Hamiltonian, and closed forms (4-site ring, XX chain
by free fermions).  The last group plants typical mistakes in a copy of the
oracle's matrix elements and checks that a pin catches each of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def _bits(s):
    return int("".join("1" if c == "u" else "0" for c in s), 2)


# ---------------------------------------------------------------- worked examples
def test_worked_example_two_sublattices():
    g = GOLD["two_sublattices"]
    p = w.chain(6, n_sublat=2, n_up=3)
    s = _bits(g["state"])
    assert s == g["state_int"]
    assert (s >> 3) == g["substate_A"] and (s & 7) == g["substate_B"]
    rep_a, _ = oracle.sublattice_tables(p, 2, 0, g["substate_A"])
    rep_b, sym_b = oracle.sublattice_tables(p, 2, 1, g["substate_B"])
    assert rep_a == g["Rep_A"] and rep_b == g["Rep_B"]
    assert [f"T{k}" for k in sym_b] == g["Sym_B"]
    # G_A / G_B: elements carrying sublattice A (resp. B) onto A
    blk = lambda X: set(range(3 * X, 3 * X + 3))
    GA = [f"T{k}" for k in range(6) if set(p.perm[k, :3].tolist()) == blk(0)]
    GB = [f"T{k}" for k in range(6) if set(p.perm[k, 3:].tolist()) == blk(0)]
    assert GA == g["G_A"] and GB == g["G_B"]
    assert int(oracle.apply_sym(p, 1, [s])[0]) == g["representative_int"] == _bits(g["representative"])
    rep, gmin, stab, kept = oracle.representatives(p, [s])
    assert int(rep[0]) == g["representative_int"] and f"T{gmin[0]}" == g["g"]


def test_worked_example_three_sublattices():
    g = GOLD["three_sublattices"]
    p = w.chain(6, n_sublat=3, n_up=3)
    s = _bits(g["state"])
    assert s == g["state_int"]
    for X, name in enumerate("ABC"):
        sub = (s >> (2 * (2 - X))) & 3
        assert sub == g["substates"][name]
        rep, sym = oracle.sublattice_tables(p, 3, X, sub)
        assert rep == g["Rep"][name]
        assert [f"T{k}" for k in sym] == g["Sym"][name]
    for name, val in g["candidates"].items():
        assert int(oracle.apply_sym(p, int(name[1:]), [s])[0]) == val
    rep, gmin, _, _ = oracle.representatives(p, [s])
    assert int(rep[0]) == g["representative_int"] == _bits(g["representative"])
    assert f"T{gmin[0]}" == g["g"]


def test_representative_is_orbit_minimum_bruteforce():
    # the orbit computed by a separate route: repeated application of the generator T1
    p = w.chain(10, n_up=4)
    states = oracle.core._sector_states(10, 4)
    rep, g, stab, kept = oracle.representatives(p, states)
    for s, r, t in zip(states.tolist(), rep.tolist(), stab.tolist()):
        orbit, x = [], s
        for _ in range(10):
            orbit.append(x)
            x = ((x >> 1) | ((x & 1) << 9))          # move every spin one site along
        assert r == min(orbit)
        assert t == sum(1 for o in orbit if o == r)


# ---------------------------------------------------------------- dimensions
@pytest.mark.parametrize("mk", [
    lambda: [w.chain(16, n_sublat=2, k=k, n_up=8) for k in range(16)],
    lambda: [w.chain(12, n_sublat=3, k=k, n_up=5) for k in range(12)],
    lambda: [w.square_torus(4, momentum=m, point_irrep=ir, n_sublat=4, J2=0.5, n_up=7)
             for m in [(0, 0), (1, 0), (1, 1), (2, 2), (0, 2)]
             for ir in range(w.n_point_irreps((4, 0), (0, 4), m))],
])
def test_dimension_matches_projection_count(mk):
    for p in mk():
        b, stab = oracle.basis(p)
        assert b.size == oracle.dimension_formula(p), p.name
        assert np.all(np.diff(b.astype(np.float64)) > 0)


def test_abelian_sector_dims_add_up():
    tot = sum(oracle.basis(w.chain(16, 2, k=k, n_up=8))[0].size for k in range(16))
    assert tot == math.comb(16, 8)


# ---------------------------------------------------------------- Eq. 2 literally
@pytest.mark.parametrize("p", [
    w.chain(10, 2, k=0, n_up=5), w.chain(10, 2, k=3, n_up=5), w.chain(10, 1, k=5, n_up=4),
    w.chain(12, 2, k=4, n_up=6, Jz=0.3),
    w.square_torus(3, momentum=(0, 0), point_irrep=1, n_sublat=1, J2=0.4, n_up=4),
    w.square_torus(3, momentum=(1, 0), point_irrep=1, n_sublat=1, J2=0.4, n_up=4),
    w.square_torus(3, momentum=(1, 2), point_irrep=0, n_sublat=1, J2=0.4, n_up=5),
])
def test_matrix_elements_equal_literal_projection(p):
    H, bs, stab = oracle.hamiltonian(p)
    Hp, bs2, dropped = oracle.projected_hamiltonian(p)
    assert np.array_equal(bs, bs2)
    assert dropped < 1e-12                    # dropped representatives have vanishing norm
    assert np.abs(H.toarray() - Hp).max() < 1e-13


# ---------------------------------------------------------------- spectra
def test_union_of_momentum_spectra_is_full_spectrum():
    N = 12
    Hf, _ = w and oracle.full_hamiltonian(w.chain(N, 1, n_up=6))
    full = np.linalg.eigvalsh(Hf.toarray())
    ev = []
    for k in range(N):
        H, _, _ = oracle.hamiltonian(w.chain(N, 2, k=k, n_up=6))
        Hd = H.toarray()
        assert np.abs(Hd - Hd.conj().T).max() < 1e-14
        ev.extend(np.linalg.eigvalsh(Hd))
    assert len(ev) == len(full)
    assert np.abs(np.sort(ev) - full).max() < 1e-11


def test_c4v_sector_spectra_inside_full_spectrum():
    base = dict(n_sublat=1, J2=0.45, n_up=4)
    Hf, _ = oracle.full_hamiltonian(w.square_torus(3, **base))
    full = np.linalg.eigvalsh(Hf.toarray())
    for m in w.momenta((3, 0), (0, 3)):
        for ir in range(w.n_point_irreps((3, 0), (0, 3), m)):
            H, _, _ = oracle.hamiltonian(w.square_torus(3, momentum=m, point_irrep=ir, **base))
            for e in np.linalg.eigvalsh(H.toarray()):
                assert np.min(np.abs(full - e)) < 1e-11


def test_four_site_ring_ground_state():
    H, _, _ = oracle.hamiltonian(w.chain(4, 1, n_up=2))
    assert abs(np.linalg.eigvalsh(H.toarray())[0] - (-2.0)) < 1e-14


@pytest.mark.parametrize("N", [8, 12, 16])
def test_xx_chain_free_fermion_ground_state(N):
    # Jz = 0: Jordan-Wigner fermions at half filling, E0 = -J / sin(pi / N) for N % 4 == 0
    e0 = min(np.linalg.eigvalsh(oracle.hamiltonian(w.chain(N, 2, k=k, n_up=N // 2, Jz=0.0))[0].toarray())[0]
             for k in range(N))
    assert abs(e0 + 1.0 / math.sin(math.pi / N)) < 1e-12


def test_chain16_ground_state_against_unsymmetrised_lanczos():
    Hf, _ = oracle.full_hamiltonian(w.chain(16, 1, n_up=8))
    e_full = spla.eigsh(Hf, k=1, which="SA", tol=1e-14)[0][0]
    e_sec = min(np.linalg.eigvalsh(oracle.hamiltonian(w.chain(16, 2, k=k, n_up=8))[0].toarray())[0]
                for k in (0, 8))
    assert abs(e_full - e_sec) < 1e-11


def test_lanczos_matches_dense():
    H, bs, _ = oracle.hamiltonian(w.config_chain16())
    v0 = w.state_uniform(bs, 1805)
    e, a, b, k = oracle.lanczos(lambda v: H @ v, v0)
    assert abs(e - np.linalg.eigvalsh(H.toarray())[0]) < 1e-11


def test_rows_equal_matrix_rows():
    p = w.chain(12, 2, k=5, n_up=6)
    H, bs, _ = oracle.hamiltonian(p)
    x = w.state_uniform(bs, 7) + 1j * w.state_uniform(bs, 8)
    xf = lambda s: w.state_uniform(s, 7) + 1j * w.state_uniform(s, 8)
    y = oracle.rows(p, bs[::5], xf)
    assert np.abs(y - (H @ x)[::5]).max() < 1e-13


# ---------------------------------------------------------------- planted mistakes
def _mutant_matrix(p, mutate, mutate_diag=None, drop_last=False):
    bs, stab = oracle.basis(p)
    diag, nt, reps, val = oracle.columns(p, bs)
    D = bs.size
    M = np.zeros((D, D), complex)
    M[np.arange(D), np.arange(D)] = diag if mutate_diag is None else mutate_diag(diag)
    for i in range(D):
        for k in range(nt[i] - (1 if drop_last and nt[i] else 0)):
            j = int(np.searchsorted(bs, reps[i, k]))
            M[j, i] += mutate(val[i, k], stab[i], stab[j])
    return M


def _differs_from_projection(M_of):
    for p in [w.chain(10, 2, k=3, n_up=5), w.chain(10, 2, k=0, n_up=5)]:
        Hp, _, _ = oracle.projected_hamiltonian(p)
        if np.abs(M_of(p) - Hp).max() > 1e-8:
            return True
    return False


def test_unmutated_columns_equal_projection():
    """The columns as the oracle emits them reproduce the literal Eq. 2 projection (the
    baseline against which the planted mistakes below are detected)."""
    assert not _differs_from_projection(lambda p: _mutant_matrix(p, lambda v, ti, tj: v))


@pytest.mark.parametrize("name,mutate_diag,drop_last", [
    ("S^z S^z sign", lambda d: -d, False),
    ("S^z S^z as J/2 instead of J/4", lambda d: 2 * d, False),
    ("one exchange term dropped per column", None, True),
])
def test_planted_diagonal_and_dropped_terms_are_caught(name, mutate_diag, drop_last):
    assert _differs_from_projection(
        lambda p: _mutant_matrix(p, lambda v, ti, tj: v, mutate_diag, drop_last)), name


@pytest.mark.parametrize("name,mutate", [
    ("chi instead of chi*", lambda v, ti, tj: np.conj(v)),
    ("no norm ratio", lambda v, ti, tj: v / math.sqrt(tj / ti)),
    ("inverted norm ratio", lambda v, ti, tj: v * ti / tj),
    ("sign of exchange", lambda v, ti, tj: -v),
])
def test_planted_mistakes_are_caught(name, mutate):
    caught = False
    for p in [w.chain(10, 2, k=3, n_up=5), w.chain(10, 2, k=0, n_up=5)]:
        M = _mutant_matrix(p, mutate)
        Hp, _, _ = oracle.projected_hamiltonian(p)
        if np.abs(M - Hp).max() > 1e-8:
            caught = True
    assert caught, name


# ---------------------------------------------------------------- spin flip (Z2)
@pytest.mark.parametrize("base", [w.chain(12, 2, k=0, n_up=6), w.chain(12, 2, k=5, n_up=6),
                                  w.chain(10, 1, k=3, n_up=5),
                                  w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5,
                                                 n_sublat=4, n_up=8)])
def test_spin_flip_sectors(base):
    """Even and odd flip sectors: dimensions add up to the unflipped sector's, the
    projection count (flip elements fix alternating configurations only) matches the
    enumeration, and the two spectra together are the unflipped spectrum."""
    ev_all, dims = [], []
    for parity in (0, 1):
        p = w.with_spin_flip(base, parity)
        b, _ = oracle.basis(p)
        assert b.size == oracle.dimension_formula(p)
        dims.append(b.size)
        if b.size:
            H, _, _ = oracle.hamiltonian(p)
            Hd = H.toarray()
            assert np.abs(Hd - Hd.conj().T).max() < 1e-14
            ev_all.extend(np.linalg.eigvalsh(Hd))
    H0, b0, _ = oracle.hamiltonian(base)
    assert sum(dims) == b0.size
    assert np.abs(np.sort(ev_all) - np.linalg.eigvalsh(H0.toarray())).max() < 1e-11


def test_spin_flip_literal_projection():
    for parity in (0, 1):
        p = w.with_spin_flip(w.chain(10, 2, k=3, n_up=5), parity)
        H, bs, _ = oracle.hamiltonian(p)
        Hp, bs2, dropped = oracle.projected_hamiltonian(p)
        assert np.array_equal(bs, bs2) and dropped < 1e-12
        assert np.abs(H.toarray() - Hp).max() < 1e-13


# ---------------------------------------------------------------- stored matrix
def _dense_from_matvec(S, D, cplx):
    eye = np.eye(D, dtype=complex if cplx else float)
    return np.stack([S.matvec(eye[:, i]) for i in range(D)], axis=1)


@pytest.mark.parametrize("p", [w.chain(10, 2, k=3, n_up=5), w.chain(10, 2, k=0, n_up=5),
                               w.chain(12, 3, k=4, n_up=5),
                               w.with_spin_flip(w.chain(10, 1, k=3, n_up=5), 1)],
                         ids=lambda p: p.name)
def test_stored_matrix_equals_literal_projection(p):
    """The stored-matrix rows (conjugated columns, targets found by binary search in the
    basis, |Stab_j| read from the basis) reproduce <i|H|j> of the literal Eq. 2 vectors,
    in real and complex sectors; block boundaries (chunk_rows) do not matter."""
    Hp, bs, _ = oracle.projected_hamiltonian(p)
    for chunk in (7, 1 << 20):
        S = oracle.stored_matrix(p, chunk_rows=chunk)
        M = _dense_from_matvec(S, bs.size, not p.is_real())
        assert np.abs(M - Hp).max() < 1e-12


def test_stored_matrix_transposed_is_caught():
    """A planted mistake -- storing columns where rows belong (no conjugation) -- fails
    the projection pin in a complex sector."""
    p = w.chain(10, 2, k=3, n_up=5)
    Hp, bs, _ = oracle.projected_hamiltonian(p)
    M = _dense_from_matvec(oracle.stored_matrix(p), bs.size, True)
    assert np.abs(M.T - Hp).max() > 1e-6


def test_stored_matrix_ground_state_and_term_count():
    """On the 16-site chain: E0 of the stored matrix equals the unsymmetrised ground
    state (minimum over the k = 0 sector), and one stored entry per surviving exchange
    term (the oracle's column count)."""
    p = w.config_chain16()
    bs, stab = oracle.basis(p)
    S = oracle.stored_matrix(p, (bs, stab), chunk_rows=100)
    _, nt, _, _ = oracle.columns(p, bs)
    assert S.nnz == int(nt.sum())
    Hf, _ = oracle.full_hamiltonian(p)
    e_full = spla.eigsh(Hf, k=1, which="SA")[0][0]
    e, _, _, _ = oracle.lanczos(S.matvec, w.state_uniform(bs, 1805))
    assert abs(e - e_full) < 1e-10


@pytest.mark.parametrize("p", [
    w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8),
    w.square_torus(4, momentum=(1, 0), point_irrep=1, J2=0.5, n_sublat=2, n_up=8),
], ids=lambda p: p.name)
def test_stored_matrix_by_coupling_class(p):
    """H is linear in the exchange of each class (Eq. 21): the stored matrices built with
    one class's exchange alone (the other set to zero, which stores no entry for its
    bonds) add up, weighted by J_c, to the literal Eq. 2 projection of the whole H.  Their
    entry counts add up to the whole matrix's."""
    Hp, bs, _ = oracle.projected_hamiltonian(p)
    parts = []
    for c in range(p.n_classes):
        J = [0.0] * p.n_classes
        J[c] = 1.0
        S = oracle.stored_matrix(p.with_couplings(J, p.Jz))
        parts.append((S, _dense_from_matvec(S, bs.size, not p.is_real())))
    M = sum(p.J[c] * parts[c][1] for c in range(p.n_classes))
    assert np.abs(M - Hp).max() < 1e-12
    assert sum(S.nnz for S, _ in parts) == oracle.stored_matrix(p).nnz


def test_square36_golden_energies_concave_in_J2():
    """The committed oracle energies of the 6x6 sector (tests/golden): E0(J2) is the
    minimum over states of <psi|H_1 + J2 H_2|psi>, a minimum of affine functions of J2,
    so it is concave: every second difference over the scan J2 = 0.40 .. 0.60 is <= 0
    (up to the energies' 1e-13 convergence).  The class-split matrices hold together
    exactly the entries of the whole matrix at J2 = 0.5."""
    import json
    import os
    gdir = os.path.join(os.path.dirname(__file__), "golden")
    g5 = json.load(open(os.path.join(gdir, "square36_e0.json")))
    gs = json.load(open(os.path.join(gdir, "square36_scan_e0.json")))
    assert gs["dim"] == g5["dim"] == 31566122
    assert sum(gs["offdiag_terms_per_class"]) == g5["offdiag_terms"]
    pts = sorted([(e["J2"], e["E0"]) for e in gs["scan"]] + [(0.5, g5["E0"])])
    assert [round(j, 2) for j, _ in pts] == [0.40, 0.45, 0.50, 0.55, 0.60]
    e = np.array([v for _, v in pts])
    assert np.all(e[:-2] - 2 * e[1:-1] + e[2:] <= 1e-12 * np.abs(e[1:-1]))


def test_square36_stored_matrix_product_against_matrix_free_rows():
    """The committed oracle product on the 6x6 sector (tests/golden/square36_hv.json, from
    the stored matrix, CSR rows built with targets found by binary search in the basis)
    against the oracle's other path, matrix-free rows with the representative and the
    index of every term found anew (Eqs. 3-5), on the file's 1024 sampled rows: the same
    values to 1e-12 of max|y|.  The sampled states are representatives of the sector, the
    file's block sums add up to its total, and |<x, y>| <= ||x|| ||y|| with
    ||x||^2 <= D / 3 (a plausibility bound: x is uniform on [-1, 1))."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "square36_hv.json")))
    p = w.config_square36(0.5)
    states = np.array(g["sample_states"], dtype=np.uint64)
    rep, _, _, kept = oracle.representatives(p, states)
    assert np.array_equal(rep, states) and np.all(kept)
    assert np.all(np.diff(states.astype(np.float64)) > 0)   # sorted rows, sorted basis
    y = oracle.rows(p, states, lambda q: w.state_uniform(q, 1804))
    ref = np.array(g["sample_y"])
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(sum(g["block_sums"]) - g["y_sum"]) <= 1e-9 * sum(g["abs_block_sums"])
    assert abs(g["x_dot_y"]) <= np.sqrt(g["dim"] / 3 * 1.01 * g["y_norm2"])
