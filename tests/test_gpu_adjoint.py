"""dE0/dJ through the adjoint product: class-resolved expectations against the oracle,
torch.autograd against central finite differences (h = 1e-4, fp64) and against the
Hellmann-Feynman value from the oracle's dense ground state."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ed():
    import paper_1804_05028_gb300 as ed
    return ed


def _unit(p, c, Jz=None):
    J = [0.0] * p.n_classes
    J[c] = 1.0
    return p.with_couplings(J, Jz)


@pytest.mark.parametrize("p", [
    w.chain(16, 2, k=3, n_up=8, Jz=0.7),
    w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8),
    w.square_torus(4, momentum=(1, 1), point_irrep=0, J2=0.5, n_sublat=1, n_up=6),
    w.square_torus(4, momentum=(1, 0), point_irrep=1, J2=0.5, n_sublat=2, n_up=8),
], ids=lambda p: p.name)
def test_class_expectations_match_oracle(p):
    B = _ed().build_basis_from(p)
    bs, _ = B.export()
    x = w.state_uniform(bs, 11)
    if not p.is_real():
        x = x + 1j * w.state_uniform(bs, 12)
    xt = torch.from_numpy(x).cuda()
    got = B.expect_classes(xt)
    for c in range(p.n_classes):
        Hc, _, _ = oracle.hamiltonian(_unit(p, c, p.Jz))
        ref = np.vdot(x, Hc @ x).real
        assert abs(got[c] - ref) <= 1e-12 * max(1.0, abs(ref))
    # the classes add up to the full product
    J = np.array(p.J)
    full = B.dot(xt, B.apply_H(xt))
    assert abs(np.dot(J, got) - np.real(full)) <= 1e-11 * abs(full)


@pytest.mark.parametrize("J2", [0.40, 0.50, 0.60])
def test_dE0_dJ_autograd_fd_and_hellmann_feynman(J2):
    from paper_1804_05028_gb300.autograd import ground_state_energy
    p = w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=J2, n_sublat=4, n_up=8)
    B = _ed().build_basis_from(p)
    J = torch.tensor([1.0, J2], dtype=torch.float64, requires_grad=True)
    E = ground_state_energy(B, J)
    E.backward()
    g = J.grad.numpy()
    # central finite differences
    h = 1e-4
    fd = []
    for c in range(2):
        e = []
        for sgn in (1, -1):
            Jc = [1.0, J2]
            Jc[c] += sgn * h
            e.append(B.lanczos(J=Jc)["E0"])
        fd.append((e[0] - e[1]) / (2 * h))
    # the h = 1e-4 central stencil has a truncation error of h^2 |d3E/dJ3| / 6, ~1e-7 here
    assert np.allclose(g, fd, rtol=0, atol=1e-6)
    # Hellmann-Feynman from the oracle's dense ground state
    H, bs, _ = oracle.hamiltonian(p)
    ev, vec = np.linalg.eigh(H.toarray())
    psi = vec[:, 0]
    hf = [psi @ (oracle.hamiltonian(_unit(p, c))[0] @ psi) for c in range(2)]
    assert np.allclose(g, hf, rtol=0, atol=1e-9)
    assert abs(E.item() - ev[0]) < 1e-10 * abs(ev[0])


@pytest.mark.parametrize("p", [
    w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8),
    w.square_torus(4, momentum=(1, 0), point_irrep=1, J2=0.5, n_sublat=2, n_up=8),
], ids=lambda p: p.name)
def test_class_expectations_fp32(p):
    """The class-resolved pass on fp32 vectors (the mixed form's adjoint): every class
    against the oracle in fp64 on the same fp32-representable vector.  Each term is a
    product of an fp32 input and an fp32 weight, summed in fp32 per row and class and in
    double across rows.  Recursive fp32 summation of a row's at most 32 terms (one per
    bond), after the rounding of the weight and of each product, is off by at most
    (32 + 3) u sum |terms| (u = 2^-24): the bound is 40 u x^T |H_c| x."""
    B = _ed().build_basis_from(p)
    s, _ = B.export()
    x = w.state_uniform(s, 1806)
    x = (x / np.linalg.norm(x)).astype(np.float32 if B.is_real else np.complex64)
    got = B.expect_classes(torch.from_numpy(x).cuda(), Jz=p.Jz)
    xd = x.astype(np.float64 if B.is_real else np.complex128)
    for c in range(p.n_classes):
        Hc, _, _ = oracle.hamiltonian(_unit(p, c, p.Jz))
        ref = np.vdot(xd, Hc @ xd).real
        bound = 40 * 2.0 ** -24 * np.abs(xd).conj() @ (abs(Hc) @ np.abs(xd))
        assert abs(got[c] - ref) <= bound, (c, got[c], ref, bound)


def test_dE0_dJ_mixed_against_oracle():
    """autograd in the mixed form (fp32 vectors both passes) on the 4x4 J1-J2 sector:
    the gradient against the oracle's dense Hellmann-Feynman value.  The fp32 ground
    state's error enters the gradient to first order: with fp32 storage its residual
    stops near u ||H|| (u = 2^-24), and the gradient error is at most about
    2 ||H_c|| ||residual|| / gap, about 1e-5 here; the test asks 2e-5 and Euler's identity
    sum_c J_c g_c = E0 to the same bound."""
    from paper_1804_05028_gb300.autograd import ground_state_energy
    p = w.square_torus(4, momentum=(0, 0), point_irrep=0, J2=0.5, n_sublat=4, n_up=8)
    B = _ed().build_basis_from(p)
    J = torch.tensor([1.0, 0.5], dtype=torch.float64, requires_grad=True)
    E = ground_state_energy(B, J, dtype=torch.float32)
    E.backward()
    g = J.grad.numpy()
    H, bs, _ = oracle.hamiltonian(p)
    ev, vec = np.linalg.eigh(H.toarray())
    psi = vec[:, 0]
    hf = np.array([psi @ (oracle.hamiltonian(_unit(p, c))[0] @ psi) for c in range(2)])
    assert np.all(np.abs(g - hf) <= 2e-5), (g, hf)
    assert abs(1.0 * g[0] + 0.5 * g[1] - ev[0]) <= 2e-5, (g, ev[0])


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle_e0_square36(J2):
    """The oracle's ground-state energy of the 6x6 sector at J2 (J1 = 1), from the
    committed golden files written by tests/golden/make_square36_e0.py (J2 = 0.5) and
    make_square36_scan.py (0.40, 0.45, 0.55, 0.60)."""
    if abs(J2 - 0.5) < 1e-12:
        return json.load(open(os.path.join(GOLDEN, "square36_e0.json")))["E0"]
    for e in json.load(open(os.path.join(GOLDEN, "square36_scan_e0.json")))["scan"]:
        if abs(e["J2"] - J2) < 1e-12:
            return e["E0"]
    raise KeyError(J2)


@pytest.fixture(scope="module")
def square36():
    B = _ed().build_basis_from(w.config_square36(0.5))
    yield B
    B.close()


@pytest.mark.parametrize("J2", [0.40, 0.45, 0.50, 0.55, 0.60])
def test_dE0_dJ_square36_scan(square36, J2):
    """Full 6x6 J1-J2 Gamma-A1 sector (the basis does not depend on the couplings), J2 in
    {0.40, ..., 0.60}: autograd against central differences in fp64 and Euler's identity
    sum_c J_c dE0/dJ_c = E0 (E0 is homogeneous of degree one in J).

    The central difference with step h has a truncation error h^2 |d3E0/dJ2^3| / 6 that
    grows where E0(J2) bends sharply (towards J2 = 0.6 on this cluster).  That error is
    measured, not assumed: with steps h = 1e-4 and 2h, fd(2h) - fd(h) is three times the
    error of fd(h) to leading order, and the Richardson combination (4 fd(h) - fd(2h)) / 3
    removes it.  The autograd value must agree with the Richardson value to 2e-7 and with
    fd(h) within fd(h)'s own measured truncation error (plus 2e-7).  The forward E0 is
    the oracle's (stored matrix, fp64 Lanczos) within 1e-10."""
    from paper_1804_05028_gb300.autograd import ground_state_energy
    B = square36
    J = torch.tensor([1.0, J2], dtype=torch.float64, requires_grad=True)
    E = ground_state_energy(B, J)
    e_or = _oracle_e0_square36(J2)
    assert abs(E.item() - e_or) <= 1e-10 * abs(e_or), (J2, E.item(), e_or)
    E.backward()
    g = J.grad.numpy()
    h = 1e-4
    e = lambda J1, J2_: B.lanczos(J=[J1, J2_])["E0"]
    fd_h = (e(1.0, J2 + h) - e(1.0, J2 - h)) / (2 * h)
    fd_2h = (e(1.0, J2 + 2 * h) - e(1.0, J2 - 2 * h)) / (4 * h)
    trunc = abs(fd_2h - fd_h) / 3
    rich = (4 * fd_h - fd_2h) / 3
    assert abs(g[1] - rich) < 2e-7, (g[1], rich, fd_h, fd_2h)
    assert abs(g[1] - fd_h) < 2 * trunc + 2e-7, (g[1], fd_h, trunc)
    fd_j1 = (e(1.0 + h, J2) - e(1.0 - h, J2)) / (2 * h)
    assert abs(g[0] - fd_j1) < 2e-6, (g[0], fd_j1)
    assert abs(1.0 * g[0] + J2 * g[1] - E.item()) < 1e-8 * abs(E.item())


def test_dE0_dJ_square36_mixed(square36):
    """The mixed-form gradient on the full 6x6 sector at J2 = 0.5 against the fp64 one
    (bound as in test_dE0_dJ_mixed_against_oracle, relative to |E0|)."""
    from paper_1804_05028_gb300.autograd import ground_state_energy
    g = []
    for dt in (torch.float64, torch.float32):
        J = torch.tensor([1.0, 0.5], dtype=torch.float64, requires_grad=True)
        E = ground_state_energy(square36, J, dtype=dt)
        E.backward()
        g.append(J.grad.numpy().copy())
    assert np.all(np.abs(g[1] - g[0]) <= 2e-5 * 18.2), g
