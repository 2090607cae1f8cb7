"""JSON sector descriptors and the command line (python -m paper_1804_05028_gb300):
descriptors round-trip exactly, `describe` writes them, and `run` computes E0 of a
described sector on the GPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _same(p, q):
    assert p.name == q.name and p.n_sites == q.n_sites and p.n_sublat == q.n_sublat
    assert p.n_classes == q.n_classes and p.n_up == q.n_up and p.phase_denom == q.phase_denom
    assert np.array_equal(p.bonds, q.bonds) and np.array_equal(p.bond_class, q.bond_class)
    assert np.array_equal(p.perm, q.perm) and np.array_equal(p.phase_num, q.phase_num)
    assert tuple(p.J) == tuple(q.J) and tuple(p.Jz) == tuple(q.Jz)
    assert (p.flip is None) == (q.flip is None)
    if p.flip is not None:
        assert np.array_equal(p.flip, q.flip)


@pytest.mark.parametrize("p", [
    w.config_chain16(), w.config_square36(), w.chain(12, 3, k=4, n_up=5, Jz=0.3),
    w.with_spin_flip(w.chain(12, 2, k=0, n_up=6), 1),
    w.square_torus(4, momentum=(1, 0), point_irrep=1, J2=0.5, n_sublat=4, n_up=8),
], ids=lambda p: p.name)
def test_descriptor_round_trip(p):
    q = w.from_dict(json.loads(json.dumps(w.to_dict(p))))
    _same(p, q)
    assert q.is_real() == p.is_real() and q.n_sym == p.n_sym


def _cli(*args):
    return subprocess.run([sys.executable, "-m", "paper_1804_05028_gb300", *args],
                          capture_output=True, text=True, timeout=600, cwd=ROOT)


def test_describe_writes_the_built_in_sector(tmp_path):
    f = tmp_path / "s.json"
    r = _cli("describe", "square36", "--n-up", "17", "-o", str(f))
    assert r.returncode == 0, r.stderr
    q = w.from_dict(json.loads(f.read_text()))
    _same(w.config_square36().with_n_up(17), q)
    assert _cli("describe", "no_such_sector").returncode == 2


def test_run_without_a_gpu_reports_an_error(tmp_path):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present (the GPU test runs the sector)")
    f = tmp_path / "c.json"
    f.write_text(json.dumps(w.to_dict(w.config_chain16())))
    r = _cli("run", str(f))
    assert r.returncode == 1 and r.stderr.startswith("error:")


@pytest.mark.gpu
def test_run_chain16_ground_state(tmp_path):
    import oracle
    f = tmp_path / "c.json"
    assert _cli("describe", "chain16", "-o", str(f)).returncode == 0
    H, bs, _ = oracle.hamiltonian(w.config_chain16())
    e_ref = np.linalg.eigvalsh(H.toarray())[0]
    for dt, tol in (("f64", 1e-10), ("f32", 1e-6)):
        r = _cli("run", str(f), "--dtype", dt)
        assert r.returncode == 0, r.stderr
        d = json.loads(r.stdout.strip().splitlines()[-1])
        assert d["dim"] == bs.size and d["converged"]
        assert abs(d["E0"] - e_ref) <= tol * abs(e_ref)
    # full reorthogonalisation and a fixed step count
    r = _cli("run", str(f), "--dtype", "f32", "--reorth", "full", "--fixed-steps", "40")
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["steps"] == 40 and d["reorth"] == "full" and d["ms_reorth"] > 0
    assert abs(d["E0"] - e_ref) <= 1e-6 * abs(e_ref)
