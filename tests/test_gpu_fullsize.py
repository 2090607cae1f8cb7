"""Full-size sectors: the 6x6 J1-J2 torus (36 translations x C4v, Gamma-A1, Sz=0) and
the 40-site tilted cluster (40 translations x C4, Gamma-A, Sz=0).

The oracle cannot enumerate C(36,18) or C(40,20) configurations in seconds, so the
GPU basis is checked through properties that fix it completely: its size equals the
character-projection count, it is strictly increasing, every sampled entry is a
surviving representative with the right stabiliser order (oracle brute force), and
sampled arbitrary configurations get the oracle's representative, stabiliser order
and a consistent index.  H x is compared row by row with the oracle's matrix-free
rows on state-keyed input vectors.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as w

GOLDEN_SQ36 = os.path.join(os.path.dirname(__file__), "golden", "square36_e0.json")

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _popcount(a):
    a = a.copy()
    c = np.zeros(a.size, np.int64)
    while np.any(a):
        c += (a & np.uint64(1)).astype(np.int64)
        a >>= np.uint64(1)
    return c


def _random_configs(N, n_up, n, seed):
    rng = np.random.default_rng(seed)
    out = np.zeros(n, np.uint64)
    for i in range(n):
        bits = rng.choice(N, n_up, replace=False)
        out[i] = np.bitwise_or.reduce(np.uint64(1) << bits.astype(np.uint64))
    return out


def _check_sector(p, n_basis_samples, n_config_samples, n_rows):
    import paper_1804_05028_gb300 as ed
    B = ed.build_basis_from(p)
    D = B.dim
    assert D == oracle.dimension_formula(p)
    s, t = B.export()
    for a in range(0, D, 1 << 26):           # strictly increasing, in chunks
        seg = s[a:min(D, a + (1 << 26) + 1)]
        assert np.all(seg[1:] > seg[:-1])
    rng = np.random.default_rng(1804)
    pick = np.sort(rng.choice(D, n_basis_samples, replace=False))
    assert np.all(_popcount(s[pick]) == p.n_up)
    rep, g, stab, kept = oracle.representatives(p, s[pick])
    assert np.array_equal(rep, s[pick]) and np.all(kept)
    assert np.array_equal(stab, t[pick].astype(np.int32))
    # arbitrary configurations through find_rep
    cfg = _random_configs(p.n_sites, p.n_up, n_config_samples, 1805)
    orep, og, ostab, okept = oracle.representatives(p, cfg)
    for method in (0, 1):
        rt, gt, pt, st, it = B.find_rep(torch.from_numpy(cfg.view(np.int64)).cuda().view(torch.uint64),
                                        method=method)
        rt = rt.cpu().view(torch.int64).numpy().view(np.uint64)
        pt, st, it = pt.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy()
        assert np.array_equal(rt, orep) and np.array_equal(st, ostab)
        assert np.array_equal(it >= 0, okept)
        assert np.array_equal(s[it[it >= 0]], orep[it >= 0])
        assert np.array_equal(pt[okept], p.phase_num[og[okept]])
    # H x on sampled rows, fp64 and fp32
    x = w.state_uniform(s, 1804)
    y = B.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    # the host-buffer entry point runs the product in row chunks with the copies of y
    # overlapped; rows are independent, so it agrees with the single launch to rounding
    # (the product groups 32 consecutive rows per warp and sums each row's terms in that
    # group's order, so a chunk boundary inside a group may change the last bit)
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.empty_like(xp).pin_memory()
    B.apply_H_host(xp, yp)
    assert np.abs(yp.numpy() - y).max() <= 1e-14 * np.abs(y).max()
    rows = np.sort(rng.choice(D, n_rows, replace=False))
    y_ref = oracle.rows(p, s[rows], lambda q: w.state_uniform(q, 1804))
    scale = np.abs(y_ref).max()
    assert np.abs(y[rows] - y_ref).max() <= 1e-12 * scale
    x32 = x.astype(np.float32)
    y32 = B.apply_H(torch.from_numpy(x32).cuda()).cpu().numpy()
    y_ref32 = oracle.rows(p, s[rows], lambda q: w.state_uniform(q, 1804).astype(np.float32).astype(np.float64))
    assert np.abs(y32[rows] - y_ref32).max() <= 2e-6 * scale
    info = B.info()
    B.close()
    return info


def test_square36_j1j2_gamma_a1():
    _check_sector(w.config_square36(), 3000, 20000, 20000)


def test_tilted40_gamma_a():
    """The 40-site sector's product on 1e5 seeded rows (its stored matrix would not fit
    in host memory)."""
    _check_sector(w.config_tilted40(), 2000, 10000, 100000)


def test_square36_spin_flip_even_odd():
    """The 6x6 Gamma-A1 S^z = 0 sector split by the spin flip: dimensions add up, both
    halves pass the sampled checks, and the lower ground state of the two equals the
    unflipped sector's."""
    import paper_1804_05028_gb300 as ed
    base = w.config_square36()
    e, dims = [], []
    for parity in (0, 1):
        p = w.with_spin_flip(base, parity)
        _check_sector(p, 1000, 5000, 100)
        B = ed.build_basis_from(p)
        dims.append(B.dim)
        e.append(B.lanczos()["E0"])
        B.close()
    B0 = ed.build_basis_from(base)
    assert sum(dims) == B0.dim
    e0 = B0.lanczos()["E0"]
    assert abs(min(e) - e0) < 1e-10 * abs(e0)


@pytest.mark.parametrize("p", [
    w.square_torus(6, momentum=(0, 0), point_irrep=0, n_sublat=4, J1=1.0, J2=0.5, n_up=5),
    w.square_torus(6, momentum=(1, 2), point_irrep=0, n_sublat=4, J1=1.0, J2=0.5, n_up=5),
    w.tilted_square_40(momentum=(0, 0), point_irrep=0, n_sublat=4, J1=1.0, J2=0.0, n_up=4),
], ids=lambda p: f"{p.name}_up{p.n_up}")
def test_full_lattices_at_low_filling_every_row(p):
    """The tables of the 6x6 torus (288 elements) and of the 40-site cluster depend on the
    lattice and the group, not on n_up; at low filling the sectors are small enough to
    check every row against the oracle, through the same kernel and tables (level 2 in
    global memory) that the half-filled sectors use."""
    import paper_1804_05028_gb300 as ed
    B = ed.build_basis_from(p)
    D = B.dim
    assert D == oracle.dimension_formula(p) and D > 0
    s, t = B.export()
    assert np.all(s[1:] > s[:-1]) and np.all(_popcount(s) == p.n_up)
    rep, g, stab, kept = oracle.representatives(p, s)
    assert np.array_equal(rep, s) and np.all(kept) and np.array_equal(stab, t.astype(np.int32))
    cplx = not p.is_real()
    x = w.state_uniform(s, 1804)
    xf = (lambda q: w.state_uniform(q, 1804))
    if cplx:
        x = x + 1j * w.state_uniform(s, 1805)
        xf = (lambda q: w.state_uniform(q, 1804) + 1j * w.state_uniform(q, 1805))
    y_ref = oracle.rows(p, s, xf)
    scale = np.abs(y_ref).max()
    dt = torch.complex128 if cplx else torch.float64
    y = B.apply_H(torch.from_numpy(x).to(dt).cuda()).cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-12 * scale
    x32 = x.astype(np.complex64 if cplx else np.float32)
    y32 = B.apply_H(torch.from_numpy(x32).cuda()).cpu().numpy()
    xf32 = (lambda q: xf(q).astype(x32.dtype).astype(np.complex128 if cplx else np.float64))
    y_ref32 = oracle.rows(p, s, xf32)
    assert np.abs(y32 - y_ref32).max() <= 2e-6 * scale
    B.close()


def test_square36_e0_against_oracle():
    """The 6x6 J1-J2 Gamma-A1 sector's ground-state energy against the oracle's
    (tests/golden/square36_e0.json, written by tests/golden/make_square36_e0.py from
    oracle/ alone: brute-force basis over all 2^36 configurations, the stored
    symmetry-adapted matrix, fp64 Lanczos with full reorthogonalisation).

    fp64: E0 within 1e-10 relative, and the first Lanczos coefficients from the same
    state-keyed start vector within 1e-11 (alpha_0 = <v0|H|v0> sums the whole product);
    mixed precision (fp32 vectors, fp64 scalars): E0 within the metric's 1e-9."""
    import paper_1804_05028_gb300 as ed
    g = json.load(open(GOLDEN_SQ36))
    B = ed.build_basis_from(w.config_square36(0.5))
    assert B.dim == g["dim"]
    assert B.count_terms()[1] == g["offdiag_terms"]
    r64 = B.lanczos(dtype=torch.float64, seed=1805)
    assert r64["converged"]
    assert abs(r64["E0"] - g["E0"]) <= 1e-10 * abs(g["E0"]), (r64["E0"], g["E0"])
    na = min(5, len(g["alpha"]))
    assert np.allclose(r64["alpha"][:na], g["alpha"][:na], rtol=0, atol=1e-11 * abs(g["E0"]))
    assert np.allclose(r64["beta"][:na - 1], g["beta"][:na - 1], rtol=0, atol=1e-11 * abs(g["E0"]))
    r32 = B.lanczos(dtype=torch.float32, seed=1805)
    assert abs(r32["E0"] - g["E0"]) <= 1e-9 * abs(g["E0"]), (r32["E0"], g["E0"])
    B.close()


def test_square36_product_against_oracle_stored_matrix():
    """H x on the whole 6x6 J1-J2 sector against the oracle's stored-matrix product
    (tests/golden/square36_hv.json, written by tests/golden/make_square36_hv.py from
    oracle/ alone), x the state-keyed vector with seed 1804, fp64: <x, y>, ||y||^2 and the
    sums of y over 256 row blocks (every row, in aggregate) within 1e-12 of the scale of
    the quantity (the sum of |y| over the block), and y at 1024 sampled rows within
    1e-12 max|y|."""
    import paper_1804_05028_gb300 as ed
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "square36_hv.json")))
    B = ed.build_basis_from(w.config_square36(0.5))
    assert B.dim == g["dim"] and B.count_terms()[1] == g["offdiag_terms"]
    s, _ = B.export()
    x = w.state_uniform(s, 1804)
    y = B.apply_H(torch.from_numpy(x).cuda()).cpu().numpy()
    B.close()
    ymax = np.abs(y).max()
    scale_dot = float(np.abs(x) @ np.abs(y))
    assert abs(float(x @ y) - g["x_dot_y"]) <= 1e-12 * scale_dot
    assert abs(float(y @ y) - g["y_norm2"]) <= 1e-12 * float(y @ y)
    blk = g["block_rows"]
    for k, a in enumerate(range(0, g["dim"], blk)):
        seg = y[a:a + blk]
        assert abs(float(seg.sum()) - g["block_sums"][k]) <= 1e-12 * g["abs_block_sums"][k], k
    rows = np.array(g["sample_rows"])
    assert np.abs(y[rows] - np.array(g["sample_y"])).max() <= 1e-12 * ymax


def test_square36_fp32_product_against_oracle_stored_matrix():
    """The fp32 product (the mixed form's) on the same vector, rounded to fp32 first,
    against the oracle's fp64 stored-matrix product.  Rounding x to fp32 moves each entry
    by at most u |x_j| (u = 2^-24) and the product rounds y_i once, so every row is within
    2u sum_j |H_ij| |x_j| + u |y_i| <= 1e-6 max|y| here, and every block sum within 1e-6
    of the block's sum of |y|."""
    import paper_1804_05028_gb300 as ed
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "square36_hv.json")))
    B = ed.build_basis_from(w.config_square36(0.5))
    s, _ = B.export()
    x = w.state_uniform(s, 1804)
    y = B.apply_H(torch.from_numpy(x).float().cuda()).cpu().numpy().astype(np.float64)
    B.close()
    ymax = np.abs(y).max()
    blk = g["block_rows"]
    for k, a in enumerate(range(0, g["dim"], blk)):
        assert abs(float(y[a:a + blk].sum()) - g["block_sums"][k]) <= 1e-6 * g["abs_block_sums"][k], k
    rows = np.array(g["sample_rows"])
    assert np.abs(y[rows] - np.array(g["sample_y"])).max() <= 1e-6 * ymax
