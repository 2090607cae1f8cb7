"""The Python binding refuses vectors of the wrong length before any pointer reaches the
library (CPU only: the refusals happen before a device is touched).

A vector shorter than the basis would let a kernel read or write past its end, so every
wrapper compares element counts first.  The basis here is a stand-in object with a
known dimension and no library handle.
"""
import pytest

torch = pytest.importorskip("torch")

import paper_1804_05028_gb300 as ed  # noqa: E402


def fake_basis(dim=10, is_real=True):
    B = ed.Basis(None, (1.0,), (1.0,), 1, device=0)
    B._info = {"dim": dim, "is_real": int(is_real)}
    return B


def refused(fn, *a, **kw):
    with pytest.raises(ValueError) as e:
        fn(*a, **kw)
    return str(e.value)


def test_apply_H_lengths():
    B = fake_basis(10)
    assert "x has 9" in refused(B.apply_H, torch.zeros(9, dtype=torch.float64))
    assert "y has 11" in refused(B.apply_H, torch.zeros(10, dtype=torch.float64),
                                 torch.zeros(11, dtype=torch.float64))


def test_apply_H_rows_lengths_and_range():
    B = fake_basis(10)
    x = torch.zeros(10, dtype=torch.float64)
    assert "outside" in refused(B.apply_H_rows, x, 3, 11)
    assert "outside" in refused(B.apply_H_rows, x, 5, 4)
    assert "y has 5" in refused(B.apply_H_rows, x, 2, 6, torch.zeros(5, dtype=torch.float64))
    assert "x has 8" in refused(B.apply_H_rows, torch.zeros(8, dtype=torch.float64), 2, 6)


def test_apply_H_host_lengths():
    import numpy as np
    B = fake_basis(10)
    assert "10 elements" in refused(B.apply_H_host, np.zeros(9))
    assert "10 elements" in refused(B.apply_H_host, np.zeros(10), np.zeros(7))
    assert "10 elements" in refused(B.apply_H_host, torch.zeros(10), torch.zeros(3))


def test_dot_and_expectations_lengths():
    B = fake_basis(10)
    assert "y has 4" in refused(B.dot, torch.zeros(10, dtype=torch.float64),
                                torch.zeros(4, dtype=torch.float64))
    assert "x has 12" in refused(B.expect_classes, torch.zeros(12, dtype=torch.float64))


def test_lanczos_vector_lengths():
    B = fake_basis(10)
    assert "v0 has 3" in refused(B.lanczos, v0=torch.zeros(3, dtype=torch.float64))
    assert "psi has 30" in refused(B.lanczos, psi=torch.zeros(30, dtype=torch.float64))


def test_dot_noalloc_lengths():
    out = torch.zeros(2, dtype=torch.float64)
    assert "y has 5" in refused(ed.dot_noalloc, torch.zeros(6, dtype=torch.float64),
                                torch.zeros(5, dtype=torch.float64), out)


def test_batch_vector_lengths():
    bt = ed.Batch.__new__(ed.Batch)
    bt._h, bt.k = None, 4
    bt.bases = [fake_basis(3), fake_basis(0), fake_basis(5, is_real=False)]
    ok = [torch.zeros(12, dtype=torch.float32), torch.zeros(0, dtype=torch.float32),
          torch.zeros(20, dtype=torch.complex64)]
    short = [ok[0], ok[1], torch.zeros(19, dtype=torch.complex64)]
    assert "one x and one y" in refused(bt.set_vectors, ok[:2], ok[:2])
    assert "x[2] has 19" in refused(bt.set_vectors, short, ok)
    assert "y[0] has 11" in refused(bt.set_vectors, ok, [torch.zeros(11), ok[1], ok[2]])
