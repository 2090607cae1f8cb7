"""Parity of the CUDA path (through the C ABI) with the oracle, element by element.

Integer work (representatives, stabiliser orders, basis, indices, characters) must be
bit-exact.  Floating point: fp64 H x within 1e-12 of max|y| (each row sums at most a
few hundred terms of size <= max|J| |x|, so rounding stays near 1e-15 relative; 1e-12
leaves three orders of margin), fp32 within 2e-6 (float eps 6e-8 times the same sums),
E0 within 1e-10 relative in fp64.

Mixed precision (fp32 vectors, fp64 scalars): every Lanczos vector is stored rounded to
fp32 (unit roundoff u = 2^-24 ~ 6e-8), so the computed tridiagonal matrix is that of an
operator perturbed by rounding errors of relative size u per vector; the lowest Ritz
value then carries an error of order u ||H||, which is not averaged away on sectors of a
few hundred states (observed up to 6.5e-8 relative here).  Small sectors are held to
TOL_F32_E0 = 4 u (||H|| ~ |E0| on these sectors); the metric's 1e-9 bar is checked on
the full 6x6 sector against the oracle's E0 (tests/test_gpu_fullsize.py), where the
rounding errors of 3e7 components average out.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


TOL_F32_E0 = 4 * 2.0 ** -24


def _ed():
    import paper_1804_05028_gb300 as ed
    return ed


def gpu_basis(p, **kw):
    return _ed().build_basis_from(p, **kw)


def _sector_states(N, n_up=None):
    s = np.arange(1 << N, dtype=np.uint64)
    if n_up is None:
        return s
    pc = np.zeros(s.size, np.int64)
    for b in range(N):
        pc += ((s >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return s[pc == n_up]


SMALL = [
    w.chain(6, 2, n_up=3), w.chain(6, 3, n_up=3),
    w.chain(12, 1, k=0, n_up=6), w.chain(12, 2, k=5, n_up=6), w.chain(12, 3, k=4, n_up=5),
    w.chain(12, 4, k=6, n_up=6), w.chain(12, 6, k=1, n_up=4),
    w.chain(16, 2, k=0, n_up=8), w.chain(16, 4, k=3, n_up=8), w.chain(16, 8, k=8, n_up=7),
    w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8),
    w.square_torus(4, momentum=(0, 0), point_irrep=3, J2=0.5, n_sublat=2, n_up=8),
    w.square_torus(4, momentum=(2, 2), point_irrep=1, J2=0.5, n_sublat=4, n_up=7),
    w.square_torus(4, momentum=(1, 0), point_irrep=1, J2=0.5, n_sublat=4, n_up=8),
    w.square_torus(4, momentum=(1, 1), point_irrep=0, J2=0.5, n_sublat=1, n_up=6),
    w.square_torus(3, momentum=(1, 2), point_irrep=0, J2=0.4, n_sublat=1, n_up=4),
    # spin flip (Z2) at S^z = 0
    w.with_spin_flip(w.chain(12, 2, k=0, n_up=6), 0),
    w.with_spin_flip(w.chain(12, 1, k=5, n_up=6), 1),
    w.with_spin_flip(w.chain(16, 4, k=3, n_up=8), 1),
    w.with_spin_flip(w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8), 0),
    w.with_spin_flip(w.square_torus(4, momentum=(2, 2), point_irrep=1, J2=0.5, n_sublat=2, n_up=8), 1),
]


def _id(p):
    return f"{p.name}_up{p.n_up}"


# ------------------------------------------------------------------ worked examples
def test_worked_examples_on_gpu():
    for nsub, rep_int, g_name in [(2, 14, 1), (3, 7, 2)]:
        p = w.chain(6, nsub, n_up=3)
        B = gpu_basis(p)
        s = torch.tensor([50], dtype=torch.uint64, device="cuda")
        rep, sym, ph, stab, idx = B.find_rep(s)
        assert int(rep.cpu()[0]) == rep_int and int(sym.cpu()[0]) == g_name
        assert int(stab.cpu()[0]) == 1
        rep2, _, _, stab2, _ = B.find_rep(s, method=1)
        assert int(rep2.cpu()[0]) == rep_int and int(stab2.cpu()[0]) == 1


# ------------------------------------------------------------------ find_rep, exhaustive
def _two_level_ok(p):
    n = p.n_sites // p.n_sublat
    return 2 <= p.n_sublat <= 4 and n <= 11


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("p", SMALL, ids=_id)
def test_find_rep_exhaustive(p, method):
    if method == 1 and not _two_level_ok(p):
        pytest.skip("two-level search needs 2..4 sublattices of <= 11 sites")
    B = gpu_basis(p)
    states = _sector_states(p.n_sites)
    rep, sym, ph, stab, idx = B.find_rep(torch.from_numpy(states.view(np.int64)).view(torch.uint64).cuda(),
                                         method=method)
    rep = rep.cpu().view(torch.int64).numpy().view(np.uint64)
    sym, ph, stab, idx = sym.cpu().numpy(), ph.cpu().numpy(), stab.cpu().numpy(), idx.cpu().numpy()
    orep, og, ostab, okept = oracle.representatives(p, states)
    assert np.array_equal(rep, orep)
    assert np.array_equal(stab, ostab)
    if method == 0:
        # the minimising element is unique up to the stabiliser: check g s == rep
        for g in np.unique(sym):
            sel = sym == g
            assert np.array_equal(oracle.apply_sym(p, int(g), states[sel]), orep[sel])
        assert np.array_equal(ph, p.phase_num[sym])
    else:
        assert np.all(sym == -1)
    ob, _ = oracle.basis(p)
    pos = np.searchsorted(ob, orep)
    in_basis = (pos < ob.size) & (ob[np.minimum(pos, max(ob.size - 1, 0))] == orep) if ob.size else np.zeros(states.size, bool)
    assert np.array_equal(idx >= 0, in_basis)
    assert np.array_equal(idx[in_basis], pos[in_basis])
    # every minimiser of a surviving representative has the same character: compare it
    assert np.array_equal(ph[in_basis], p.phase_num[og[in_basis]])


# ------------------------------------------------------------------ basis, bit-exact
EXTRA = [
    w.chain(20, 4, k=0, n_up=10), w.chain(20, 5, k=7, n_up=9), w.chain(18, 3, k=9, n_up=9),
    w.chain(16, 2, k=0, n_up=0), w.chain(16, 2, k=3, n_up=0), w.chain(16, 2, k=0, n_up=1),
    w.chain(16, 2, k=0, n_up=16), w.chain(8, 8, k=4, n_up=4),
] + [w.chain(16, 2, k=k, n_up=8) for k in range(16)]


@pytest.mark.parametrize("p", SMALL + EXTRA, ids=_id)
def test_basis_bit_exact(p):
    B = gpu_basis(p)
    s, t = B.export()
    ob, ostab = oracle.basis(p)
    assert B.dim == ob.size == oracle.dimension_formula(p)
    assert np.array_equal(s, ob)
    assert np.array_equal(t.astype(np.int32), ostab)


# ------------------------------------------------------------------ H x
def _x_for(states, cplx, seed=1804):
    x = w.state_uniform(states, seed)
    if cplx:
        x = x + 1j * w.state_uniform(states, seed + 1)
    return x


@pytest.mark.parametrize("p", SMALL + EXTRA[:3], ids=_id)
def test_apply_H_fp64(p):
    B = gpu_basis(p)
    if B.dim == 0:
        return
    H, bs, _ = oracle.hamiltonian(p)
    cplx = not p.is_real()
    x = _x_for(bs, cplx)
    y_ref = H @ x
    dt = torch.complex128 if cplx else torch.float64
    y = B.apply_H(torch.from_numpy(x).to(dt).cuda()).cpu().numpy()
    scale = max(np.abs(y_ref).max(), 1.0)
    assert np.abs(y - y_ref).max() <= 1e-12 * scale
    # a second call gives identical bits (fixed summation order, no atomics)
    y2 = B.apply_H(torch.from_numpy(x).to(dt).cuda()).cpu().numpy()
    assert np.array_equal(y, y2)


@pytest.mark.parametrize("p", [SMALL[7], SMALL[10], SMALL[12], SMALL[3]], ids=_id)
def test_apply_H_fp32(p):
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    cplx = not p.is_real()
    x = _x_for(bs, cplx)
    # the oracle result for the fp32-rounded input, compared at float accuracy
    xr = x.astype(np.complex64 if cplx else np.float32)
    y_ref = H @ xr.astype(np.complex128 if cplx else np.float64)
    dt = torch.complex64 if cplx else torch.float32
    y = B.apply_H(torch.from_numpy(xr).to(dt).cuda()).cpu().numpy()
    assert np.abs(y - y_ref).max() <= 2e-6 * max(np.abs(y_ref).max(), 1.0)


def test_apply_H_rows_and_host():
    p = w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8)
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    x = _x_for(bs, False)
    y_ref = H @ x
    xt = torch.from_numpy(x).cuda()
    D = B.dim
    parts = [B.apply_H_rows(xt, a, b).cpu().numpy() for a, b in [(0, 3), (3, D // 2), (D // 2, D)]]
    assert np.abs(np.concatenate(parts) - y_ref).max() < 1e-12 * np.abs(y_ref).max()
    y_h = B.apply_H_host(x)
    assert np.abs(y_h - y_ref).max() < 1e-12 * np.abs(y_ref).max()
    yp = torch.empty(D, dtype=torch.float64).pin_memory()
    B.apply_H_host(torch.from_numpy(x).pin_memory(), yp)
    assert np.abs(yp.numpy() - y_ref).max() < 1e-12 * np.abs(y_ref).max()


def test_couplings_and_anisotropy():
    p = w.chain(12, 2, k=3, n_up=6)
    B = gpu_basis(p)
    for J, Jz in [((0.7,), (0.0,)), ((-1.3,), (2.5,))]:
        q = p.with_couplings(J, Jz)
        H, bs, _ = oracle.hamiltonian(q)
        x = _x_for(bs, True)
        y = B.apply_H(torch.from_numpy(x).cuda(), J=J, Jz=Jz).cpu().numpy()
        assert np.abs(y - H @ x).max() < 1e-12 * np.abs(H @ x).max()


@pytest.mark.parametrize("p", [
    w.chain(20, 4, k=0, n_up=10),      # two-level kernel, 4 blocks of 5 sites
    w.chain(20, 2, k=3, n_up=9),       # two-level kernel, complex characters
    w.chain(20, 5, k=0, n_up=10),      # 5 blocks: the generic kernel (Alg. 2 as printed)
], ids=_id)
def test_apply_H_many_blocks_ragged_tail(p):
    """About 9,000 rows: many 512-row thread blocks and a partial last one, the whole
    product and row ranges that cut blocks, in fp64 and fp32."""
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    D = B.dim
    assert D == bs.size and D > 8 * 512 and D % 512
    cplx = not p.is_real()
    x = _x_for(bs, cplx)
    y_ref = H @ x
    scale = np.abs(y_ref).max()
    dt, dt32 = (torch.complex128, torch.complex64) if cplx else (torch.float64, torch.float32)
    xt = torch.from_numpy(x).to(dt).cuda()
    assert np.abs(B.apply_H(xt).cpu().numpy() - y_ref).max() <= 1e-12 * scale
    cuts = [0, 1, 511, 513, D // 3, D - 7, D]
    parts = [B.apply_H_rows(xt, a, b).cpu().numpy() for a, b in zip(cuts[:-1], cuts[1:])]
    assert np.abs(np.concatenate(parts) - y_ref).max() <= 1e-12 * scale
    x32 = x.astype(np.complex64 if cplx else np.float32)
    y32 = B.apply_H(torch.from_numpy(x32).cuda()).cpu().numpy()
    y_ref32 = H @ x32.astype(np.complex128 if cplx else np.float64)
    assert np.abs(y32 - y_ref32).max() <= 2e-6 * scale


# ------------------------------------------------------------------ Lanczos
@pytest.mark.parametrize("p", [
    w.config_chain16(),
    w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8),
    w.chain(16, 2, k=5, n_up=8),
    w.with_spin_flip(w.config_chain16(), 0),
    w.with_spin_flip(w.config_chain16(), 1),
], ids=_id)
def test_lanczos_E0(p):
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    e_ref = np.linalg.eigvalsh(H.toarray())[0]
    r = B.lanczos()
    assert r["converged"]
    assert abs(r["E0"] - e_ref) <= 1e-10 * abs(e_ref)
    # mixed precision (fp32 vectors, fp64 scalars and reorthogonalisation)
    rf = B.lanczos(dtype=torch.float32 if p.is_real() else torch.complex64)
    assert abs(rf["E0"] - e_ref) <= TOL_F32_E0 * abs(e_ref)


@pytest.mark.parametrize("p", [
    w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8),
    w.chain(16, 2, k=5, n_up=8),
], ids=_id)
def test_lanczos_reorthogonalisation_modes(p):
    """Every reorthogonalisation mode gives the dense E0 (fp64 1e-10, mixed TOL_F32_E0);
    with the full store the ground state comes from the stored Krylov basis and its
    Rayleigh quotient matches E0 to fp64 rounding in fp64 and to TOL_F32_E0 in fp32."""
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    ev, vec = np.linalg.eigh(H.toarray())
    e_ref = ev[0]
    cplx = not p.is_real()
    for dt, tol in ((torch.complex128 if cplx else torch.float64, 1e-10),
                    (torch.complex64 if cplx else torch.float32, TOL_F32_E0)):
        rs = {}
        for mode in ("none", "local", "full"):
            psi = torch.empty(B.dim, dtype=dt, device="cuda")
            r = B.lanczos(dtype=dt, reorth=mode, psi=psi)
            assert r["converged"], mode
            assert abs(r["E0"] - e_ref) <= tol * abs(e_ref), (mode, dt, r["E0"] - e_ref)
            if mode != "none":   # without reorthogonalisation only the energy is claimed
                v = psi.cpu().numpy().astype(np.complex128)
                ov = abs(np.vdot(vec[:, 0], v))
                assert abs(ov - 1.0) < (1e-8 if tol == 1e-10 else 1e-5), (mode, dt, ov)
            rs[mode] = r
        assert rs["none"]["ms_reorth"] == 0.0 and rs["full"]["ms_reorth"] > 0.0
        rq_tol = 1e-12 if tol == 1e-10 else TOL_F32_E0
        assert abs(rs["full"]["rq"] - e_ref) <= rq_tol * abs(e_ref), (dt, rs["full"]["rq"] - e_ref)


def test_lanczos_full_store_limits():
    """The full mode takes at most (slots - 1) steps and refuses a store of one vector or a
    fixed step count the store cannot hold."""
    ed = _ed()
    B = gpu_basis(w.config_chain16())
    kry = torch.empty(11 * B.dim, dtype=torch.float64, device="cuda")
    r = B.lanczos(reorth="full", krylov=kry, max_steps=300, tol=1e-30)
    assert r["steps"] == 10
    with pytest.raises(ed.EdError):
        B.lanczos(reorth="full", krylov=kry[:B.dim])
    with pytest.raises(ed.EdError):
        B.lanczos(reorth="full", krylov=kry, fixed_steps=11)


def test_lanczos_chain16_fixed_100_steps_and_psi():
    p = w.config_chain16()
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    evals, evecs = np.linalg.eigh(H.toarray())
    psi = torch.empty(B.dim, dtype=torch.float64, device="cuda")
    r = B.lanczos(fixed_steps=100, psi=psi)
    assert r["steps"] == 100 or r["converged"]
    assert abs(r["E0"] - evals[0]) < 1e-10 * abs(evals[0])
    assert abs(r["rq"] - evals[0]) < 1e-10 * abs(evals[0])
    v = psi.cpu().numpy()
    assert abs(abs(np.dot(v, evecs[:, 0])) - 1.0) < 1e-8
    # alpha / beta reproduce the oracle's Lanczos on the same start vector for a few steps
    e, a, b, k = oracle.lanczos(lambda u: H @ u, w.state_uniform(bs, 1805), max_steps=5, tol=0)
    assert np.allclose(r["alpha"][:5], a[:5], rtol=0, atol=1e-12)
    assert np.allclose(r["beta"][:4], b[:4], rtol=0, atol=1e-12)


# ------------------------------------------------------------------ edge cases and errors
def test_empty_and_one_state_sectors():
    ed = _ed()
    B0 = gpu_basis(w.chain(16, 2, k=3, n_up=0))
    assert B0.dim == 0
    x = torch.empty(0, dtype=torch.complex128, device="cuda")
    B0.apply_H(x)
    with pytest.raises(ed.EdError) as e:
        B0.lanczos()
    assert e.value.code == 6
    B1 = gpu_basis(w.chain(16, 2, k=0, n_up=0))
    assert B1.dim == 1
    y = B1.apply_H(torch.ones(1, dtype=torch.float64, device="cuda")).item()
    assert abs(y - 16 * 0.25) < 1e-15
    r = B1.lanczos()
    assert abs(r["E0"] - 4.0) < 1e-14 and r["converged"]


def test_descriptor_errors():
    ed = _ed()
    p = w.chain(6, 1, n_up=3)
    # an unstable split: positions 0..5 labelled in order, blocks {0,1,2} / {3,4,5}
    with pytest.raises(ed.EdError) as e:
        ed.build_basis(6, 2, p.bonds, p.bond_class, 1, p.perm, p.phase_num, p.phase_denom, 3)
    assert e.value.code == 2
    with pytest.raises(ed.EdError) as e:
        ed.build_basis(6, 4, p.bonds, p.bond_class, 1, p.perm, p.phase_num, p.phase_denom, 3)
    assert e.value.code == 2
    with pytest.raises(ed.EdError) as e:       # not closed
        ed.build_basis(6, 1, p.bonds, p.bond_class, 1, p.perm[:4], p.phase_num[:4], p.phase_denom, 3)
    assert e.value.code == 1
    bad = p.phase_num.copy(); bad[1] = 1
    with pytest.raises(ed.EdError) as e:       # not a homomorphism
        ed.build_basis(6, 1, p.bonds, p.bond_class, 1, p.perm, bad, 6, 3)
    assert e.value.code == 1
    with pytest.raises(ed.EdError) as e:       # bonds not invariant
        ed.build_basis(6, 1, p.bonds[:5], p.bond_class[:5], 1, p.perm, p.phase_num, p.phase_denom, 3)
    assert e.value.code == 1
    B = gpu_basis(w.chain(6, 2, k=1, n_up=3))
    with pytest.raises(ed.EdError):            # complex sector needs a complex vector
        B.apply_H(torch.zeros(B.dim, dtype=torch.float64, device="cuda"))


def test_sharded_driver_on_one_gpu():
    """The row-sharded driver with the CUDA rows (world size 1: no collective runs)."""
    from paper_1804_05028_gb300.parallel import ShardedOperator, cuda_local_apply, sharded_lanczos
    p = w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8)
    B = gpu_basis(p)
    H, bs, _ = oracle.hamiltonian(p)
    op = ShardedOperator(cuda_local_apply(B), B.dim, 0, 1)
    x = torch.from_numpy(_x_for(bs, False)).cuda()
    assert torch.allclose(op.matvec(x), B.apply_H(x), rtol=0, atol=1e-13)
    e, steps, a, b = sharded_lanczos(op, x.clone())
    e_ref = np.linalg.eigvalsh(H.toarray())[0]
    assert abs(e - e_ref) < 1e-10 * abs(e_ref)
    # fp32 slices: the same driver on the library's fp32 kernels
    e32, _, _, _ = sharded_lanczos(op, x.float().clone())
    assert abs(e32 - e_ref) < TOL_F32_E0 * abs(e_ref)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32, torch.complex128, torch.complex64])
def test_slice_vector_operations(dt):
    """ed_axpy_norm and ed_scale on slices (the rank-local arithmetic of the sharded
    driver) against the same operations in fp64 on the host, on a ragged length."""
    ed = _ed()
    g = torch.Generator(device="cuda").manual_seed(11)
    n = 100003
    mk = lambda: torch.randn(n, dtype=dt, device="cuda", generator=g)
    w, v, vp = mk(), mk(), mk()
    ref = (w.cpu().to(torch.complex128) - 0.37 * v.cpu().to(torch.complex128)
           - 1.25 * vp.cpu().to(torch.complex128))
    scratch = torch.zeros(4096, dtype=torch.float64, device="cuda")
    norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ed.axpy_norm(w, v, vp, 0.37, 1.25, scratch, norm2)
    tol = 1e-14 if dt in (torch.float64, torch.complex128) else 1e-7
    got = w.cpu().to(torch.complex128)
    assert (got - ref).abs().max().item() <= tol * ref.abs().max().item()
    assert abs(norm2.item() - (got.abs() ** 2).sum().item()) <= 1e-12 * norm2.item()
    ed.axpy_norm(w, v, None, 0.5, 0.0, scratch, norm2)   # no previous vector
    ed.scale(w, 0.25)
    ref2 = 0.25 * (got - 0.5 * v.cpu().to(torch.complex128))
    assert (w.cpu().to(torch.complex128) - ref2).abs().max().item() <= 4 * tol * ref2.abs().max().item()
