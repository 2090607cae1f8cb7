"""The problem descriptors themselves: groups closed, characters homomorphisms,
bonds invariant, sublattice splits stable (Sec. III B), sizes as stated."""
import numpy as np
import pytest

import workloads as w


def _check_group(p):
    G = p.perm
    idx = {tuple(r): i for i, r in enumerate(G.tolist())}
    assert len(idx) == len(G)
    assert tuple(range(p.n_sites)) in idx
    for a in range(len(G)):
        for b in range(len(G)):
            c = idx[tuple(G[a][G[b]].tolist())]
            assert (p.phase_num[a] + p.phase_num[b] - p.phase_num[c]) % p.phase_denom == 0
    bonds = {(min(a, b), max(a, b), int(c)) for (a, b), c in zip(p.bonds.tolist(), p.bond_class)}
    assert len(bonds) == p.n_bonds
    for g in G:
        img = {(min(g[a], g[b]), max(g[a], g[b]), int(c)) for (a, b), c in zip(p.bonds.tolist(), p.bond_class)}
        assert img == bonds
    n = p.n_sites // p.n_sublat
    for g in G:
        for X in range(p.n_sublat):
            assert len({int(g[X * n + k]) // n for k in range(n)}) == 1


@pytest.mark.parametrize("p", [
    w.config_chain16(), w.config_chain16(4), w.config_square36(), w.config_square36(n_sublat=2),
    w.config_tilted40(), w.chain(6, 2), w.chain(6, 3),
    w.square_torus(4, momentum=(1, 0), point_irrep=1, J2=0.5, n_sublat=4),
])
def test_descriptor_consistent(p):
    _check_group(p)


def test_sizes():
    assert w.config_square36().n_sym == 288 and w.config_square36().n_bonds == 144
    assert w.config_tilted40().n_sym == 160 and w.config_tilted40().n_bonds == 80
    assert w.config_chain16().n_sym == 16
    assert len(w.config_square25_sectors()) == 572


def test_four_sublattice_split_of_5x5_is_rejected():
    with pytest.raises(ValueError):
        w.square_torus(5, n_sublat=4)


def test_state_keyed_vectors_are_deterministic():
    s = np.arange(1000, dtype=np.uint64) * np.uint64(977)
    a, b = w.state_uniform(s, 3), w.state_uniform(s, 3)
    assert np.array_equal(a, b) and a.min() >= -1 and a.max() < 1
    assert abs(a.mean()) < 0.1 and not np.array_equal(a, w.state_uniform(s, 4))
    g = w.state_gaussian(s, 3)
    assert abs(g.mean()) < 0.15 and abs(g.std() - 1) < 0.1
    # SplitMix64 reference value (Vigna's splitmix64.c with state 0 -> first output)
    assert int(w.splitmix64(np.array([0x9E3779B97F4A7C15], np.uint64))[0]) == 0xE220A8397B1DCDAF
