"""Descriptor validation of ed_build_basis, on the host: every refusal happens before any
CUDA call, so these run without a GPU.  Each case breaks one property that the paper's
construction needs (a group of site permutations with a 1-D character, bonds invariant
under it, a sublattice split that every element carries block onto block, Sec. III B)
and checks the error code and message."""
import numpy as np
import pytest

import paper_1804_05028_gb300 as ed
import workloads as w

INVALID, UNSTABLE, CUDA, UNSUPPORTED = 1, 2, 4, 7


def _build(p, **over):
    a = dict(n_sites=p.n_sites, n_sublat=p.n_sublat, bonds=p.bonds, bond_class=p.bond_class,
             n_classes=p.n_classes, perm=p.perm, phase_num=p.phase_num, phase_denom=p.phase_denom,
             n_up=p.n_up, flip=getattr(p, "flip", None))
    a.update(over)
    return ed.build_basis(**a, stream=0)


def _refused(p, code, text, **over):
    with pytest.raises(ed.EdError) as e:
        _build(p, **over)
    assert e.value.code == code, str(e.value)
    assert text in str(e.value), str(e.value)


@pytest.fixture(scope="module")
def chain6():
    ed.build()
    return w.chain(6, 2, k=1, n_up=3)       # labels: block 0 = even positions, block 1 = odd


def test_counts_out_of_range(chain6):
    p = chain6
    _refused(p, INVALID, "n_sublat", n_sublat=0)
    _refused(p, INVALID, "n_sublat", n_sublat=9)
    _refused(p, INVALID, "n_classes", n_classes=0)
    _refused(p, INVALID, "n_up out of range", n_up=7)
    _refused(p, INVALID, "n_up out of range", n_up=-1)
    _refused(p, INVALID, "bad irrep", phase_denom=0)


def test_split_must_divide_and_be_stable(chain6):
    p = chain6
    _refused(p, UNSTABLE, "does not divide", n_sublat=4)
    # position order as labels: blocks {0,1,2} and {3,4,5}; T1 sends 2 to 3
    q = w.chain(6, 1, k=1, n_up=3)
    _refused(q, UNSTABLE, "not stable", n_sublat=2)


def test_one_block_size_limit():
    q = w.chain(28, 1, k=0, n_up=14)
    _refused(q, UNSUPPORTED, "N <= 26")


def test_group_axioms(chain6):
    p = chain6
    bad = p.perm.copy()
    bad[1, 0] = bad[1, 1]                   # two sites onto one
    _refused(p, INVALID, "not a bijection", perm=bad)
    _refused(p, INVALID, "not closed", perm=p.perm[:4], phase_num=p.phase_num[:4])
    _refused(p, INVALID, "no identity", perm=p.perm[1:], phase_num=p.phase_num[1:])
    ph = p.phase_num.copy()
    ph[0] = 1                               # chi(e) = exp(2 pi i / 6)
    _refused(p, INVALID, "chi(identity)", phase_num=ph)
    ph = p.phase_num.copy()
    ph[2] = (ph[2] + 1) % p.phase_denom     # chi(T2) != chi(T1)^2
    _refused(p, INVALID, "not a homomorphism", phase_num=ph)


def test_bonds(chain6):
    p = chain6
    b = p.bonds.copy()
    b[0, 1] = b[0, 0]
    _refused(p, INVALID, "bad bond", bonds=b)
    c = np.array(p.bond_class).copy()
    c[0] = 1
    _refused(p, INVALID, "bad bond class", bond_class=c)
    dup = np.vstack([p.bonds, p.bonds[:1]])
    _refused(p, INVALID, "duplicate bond", bonds=dup, bond_class=np.zeros(len(dup), np.int32))
    _refused(p, INVALID, "not invariant", bonds=p.bonds[:5], bond_class=p.bond_class[:5])
    # two classes that the group mixes
    c2 = np.array(p.bond_class).copy()
    c2[0] = 1
    _refused(p, INVALID, "not invariant", bond_class=c2, n_classes=2)


def test_spin_flip_needs_half_filling():
    q = w.with_spin_flip(w.chain(6, 2, k=0, n_up=3), 0)
    _refused(q, INVALID, "n_up = N/2", n_up=2)


def test_valid_descriptor_reaches_the_device(chain6):
    """A valid sector passes validation; without a GPU the first CUDA call reports."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the build itself is covered by the GPU tests")
    with pytest.raises(ed.EdError) as e:
        _build(chain6)
    assert e.value.code == CUDA
