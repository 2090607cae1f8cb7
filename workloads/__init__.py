"""Seeded synthetic inputs for the symmetry-adapted spin-1/2 Hamiltonian.

Everything here is *problem data*: it is consumed unchanged by the CPU oracle, by
the tests and by the benchmark, and it holds none of the method's arithmetic (no
representative search, no matrix element, no eigensolver).

A :class:`Problem` describes one symmetry sector of a spin-1/2 model:

* ``n_sites`` N and the site labelling.  Label 0 is the most significant bit of
  the integer coding of a configuration and an up spin is a 1 (Sec. II, Eq. 1 and
  the ordering by ``int``).  Sites of sublattice X carry the labels
  ``X*N/n_sublat ... (X+1)*N/n_sublat - 1``, sublattice 0 being the most
  significant block (Sec. III B, site numbering below the stability definition).
* ``bonds``: pairs of labels, each with a coupling class (J1, J2, ...).  The
  Hamiltonian is H = sum_b J_c(b) [ Jz_c S^z_i S^z_j + (S^+_i S^-_j + h.c.)/2 ]
  (Eq. 21, with the exchange split into classes; Jz_c = 1 is Heisenberg).
* ``perm``: the symmetry group as site permutations; group element g carries the
  spin on label p to label ``perm[g, p]``.  The group acts on configurations by
  (g s)[perm[g, p]] = s[p].
* ``phase_num`` / ``phase_denom``: a one-dimensional irrep given exactly as
  chi(g) = exp(2 pi i phase_num[g] / phase_denom) (Sec. II restricts to 1-D
  irreps).
* ``n_up``: the number of up spins (the S^z sector).

Vectors on a basis are keyed by the *state*, not by its position, so that any
party that knows a representative can evaluate the input coefficient without
knowing where that state sits in somebody else's basis array.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import Sequence

import numpy as np

__all__ = [
    "Problem", "chain", "square_cluster", "square_torus", "tilted_square_40",
    "point_group_irreps", "momenta", "state_uniform", "state_gaussian",
    "splitmix64", "config_chain16", "config_square36", "config_square25_sectors",
    "config_tilted40", "C4V_OPS", "C4V_NAMES", "n_point_irreps", "with_spin_flip",
    "to_dict", "from_dict",
]


@dataclasses.dataclass
class Problem:
    name: str
    n_sites: int
    n_sublat: int
    bonds: np.ndarray          # (n_bonds, 2) int32 labels
    bond_class: np.ndarray     # (n_bonds,) int32
    n_classes: int
    perm: np.ndarray           # (n_sym, N) int32
    phase_denom: int
    phase_num: np.ndarray      # (n_sym,) int32
    n_up: int
    J: tuple                   # per class
    Jz: tuple                  # per class
    coords: np.ndarray | None = None   # (N, 2) real-space coordinate of each label
    sym_names: list | None = None
    flip: np.ndarray | None = None     # (n_sym,) uint8: element also reverses every spin

    @property
    def n_sym(self) -> int:
        return int(self.perm.shape[0])

    @property
    def n_bonds(self) -> int:
        return int(self.bonds.shape[0])

    def is_real(self) -> bool:
        """True when every character is +1 or -1."""
        twice = (2 * self.phase_num) % self.phase_denom
        return bool(np.all(twice == 0))

    def with_n_up(self, n_up: int) -> "Problem":
        return dataclasses.replace(self, n_up=int(n_up))

    def with_couplings(self, J: Sequence[float], Jz: Sequence[float] | None = None) -> "Problem":
        J = tuple(float(v) for v in J)
        Jz = tuple(float(v) for v in (Jz if Jz is not None else self.Jz))
        return dataclasses.replace(self, J=J, Jz=Jz)


def to_dict(p: Problem) -> dict:
    """A JSON-ready description of the sector: every field of Problem as plain lists."""
    arr = lambda a: None if a is None else np.asarray(a).tolist()
    return {"name": p.name, "n_sites": int(p.n_sites), "n_sublat": int(p.n_sublat),
            "bonds": arr(p.bonds), "bond_class": arr(p.bond_class), "n_classes": int(p.n_classes),
            "perm": arr(p.perm), "phase_denom": int(p.phase_denom), "phase_num": arr(p.phase_num),
            "n_up": int(p.n_up), "J": [float(v) for v in p.J], "Jz": [float(v) for v in p.Jz],
            "coords": arr(p.coords), "sym_names": None if p.sym_names is None else list(p.sym_names),
            "flip": arr(p.flip)}


def from_dict(d: dict) -> Problem:
    """The inverse of to_dict."""
    opt = lambda k, dt: None if d.get(k) is None else np.asarray(d[k], dtype=dt)
    return Problem(name=str(d["name"]), n_sites=int(d["n_sites"]), n_sublat=int(d["n_sublat"]),
                   bonds=np.asarray(d["bonds"], np.int32).reshape(-1, 2),
                   bond_class=np.asarray(d["bond_class"], np.int32), n_classes=int(d["n_classes"]),
                   perm=np.asarray(d["perm"], np.int32).reshape(-1, int(d["n_sites"])),
                   phase_denom=int(d["phase_denom"]), phase_num=np.asarray(d["phase_num"], np.int32),
                   n_up=int(d["n_up"]), J=tuple(float(v) for v in d["J"]),
                   Jz=tuple(float(v) for v in d["Jz"]), coords=opt("coords", np.float64),
                   sym_names=d.get("sym_names"), flip=opt("flip", np.uint8))


def with_spin_flip(p: Problem, parity: int) -> Problem:
    """The group G x Z2 of p's group and the reversal of every spin, for the S^z = 0
    sector (n_up = N/2), in the even (parity 0) or odd (parity 1) irrep of the flip.

    Element (g, f) acts as s -> g s with every spin reversed when f = 1; its character
    is chi(g) (-1)^(f parity).  The paper uses this symmetry in all its benchmarks
    (Sec. V, Table 1: "even" / "odd").
    """
    if 2 * p.n_up != p.n_sites:
        raise ValueError("the spin flip maps the sector to itself only at n_up = N/2")
    if getattr(p, "flip", None) is not None:
        raise ValueError("already has the spin flip")
    denom = math.lcm(p.phase_denom, 2)
    base = (p.phase_num.astype(np.int64) * (denom // p.phase_denom)) % denom
    odd = (base + (denom // 2 if parity else 0)) % denom
    names = p.sym_names or [f"g{i}" for i in range(p.n_sym)]
    return dataclasses.replace(
        p, name=f"{p.name}_flip{'odd' if parity else 'even'}",
        perm=np.concatenate([p.perm, p.perm]).astype(np.int32), phase_denom=denom,
        phase_num=np.concatenate([base, odd]).astype(np.int32),
        flip=np.concatenate([np.zeros(p.n_sym, np.uint8), np.ones(p.n_sym, np.uint8)]),
        sym_names=names + [n + "*F" for n in names])


# ----------------------------------------------------------------------------
# one-dimensional chain with periodic boundary conditions
# ----------------------------------------------------------------------------

def chain(N: int, n_sublat: int = 1, k: int = 0, n_up: int | None = None,
          J: float = 1.0, Jz: float = 1.0) -> Problem:
    """Periodic chain of N sites, translation group C_N, momentum index k.

    Position p belongs to sublattice p mod n_sublat; inside a sublattice the
    positions are labelled in increasing order (the labelling of the six-site
    examples of Sec. III A and III B).  T_n carries position p to p+n and
    chi(T_n) = exp(2 pi i k n / N).
    """
    if N % n_sublat:
        raise ValueError("n_sublat must divide N")
    m = N // n_sublat
    label = np.array([(p % n_sublat) * m + p // n_sublat for p in range(N)], dtype=np.int32)
    perm = np.empty((N, N), dtype=np.int32)
    for n in range(N):
        for p in range(N):
            perm[n, label[p]] = label[(p + n) % N]
    bonds = np.array([[label[p], label[(p + 1) % N]] for p in range(N)], dtype=np.int32)
    coords = np.zeros((N, 2))
    coords[label, 0] = np.arange(N)
    return Problem(
        name=f"chain{N}_k{k}_sub{n_sublat}", n_sites=N, n_sublat=n_sublat,
        bonds=bonds, bond_class=np.zeros(N, dtype=np.int32), n_classes=1,
        perm=perm, phase_denom=N,
        phase_num=np.array([(k * n) % N for n in range(N)], dtype=np.int32),
        n_up=N // 2 if n_up is None else n_up, J=(float(J),), Jz=(float(Jz),),
        coords=coords, sym_names=[f"T{n}" for n in range(N)])


# ----------------------------------------------------------------------------
# square-lattice clusters spanned by two superlattice vectors
# ----------------------------------------------------------------------------

# point operations of the square lattice, as integer 2x2 matrices acting on (x, y)
C4V_NAMES = ["E", "C4", "C2", "C4^3", "sx", "sy", "sd", "sd'"]
C4V_OPS = [
    np.array([[1, 0], [0, 1]]), np.array([[0, -1], [1, 0]]),
    np.array([[-1, 0], [0, -1]]), np.array([[0, 1], [-1, 0]]),
    np.array([[-1, 0], [0, 1]]), np.array([[1, 0], [0, -1]]),
    np.array([[0, 1], [1, 0]]), np.array([[0, -1], [-1, 0]]),
]


class _Cluster:
    """Integer points of Z^2 modulo the superlattice spanned by a1, a2."""

    def __init__(self, a1, a2):
        (a, b), (c, d) = a1, a2
        self.a1, self.a2 = (a, b), (c, d)
        self.det = a * d - b * c
        if self.det <= 0:
            raise ValueError("a1, a2 must be positively oriented")
        self.n = self.det
        keys = {}
        span = abs(a) + abs(b) + abs(c) + abs(d) + 1
        for x in range(-span, span + 1):
            for y in range(-span, span + 1):
                kk = self.key(x, y)
                if kk not in keys:
                    keys[kk] = self.canonical_xy(kk)
        if len(keys) != self.n:
            raise AssertionError("cluster enumeration failed")
        self.keys = keys

    def key(self, x, y):
        (a, b), (c, d) = self.a1, self.a2
        return ((d * x - c * y) % self.det, (-b * x + a * y) % self.det)

    def canonical_xy(self, kk):
        (a, b), (c, d) = self.a1, self.a2
        u, v = kk
        return ((a * u + c * v) // self.det, (b * u + d * v) // self.det)

    def in_lattice(self, x, y):
        return self.key(x, y) == (0, 0)


def square_cluster(a1, a2, *, point_ops: Sequence[int] | None = None,
                   momentum=(0, 0), point_irrep: int = 0, n_sublat: int = 4,
                   J1: float = 1.0, J2: float = 0.0, n_up: int | None = None,
                   name: str | None = None) -> Problem:
    """Square lattice on the torus spanned by a1, a2 (integer vectors).

    The group is the translations by every site times the point operations of
    C4v (indices into :data:`C4V_OPS`) that leave the superlattice invariant
    *and* the momentum invariant (the little group).  ``point_irrep`` indexes the
    one-dimensional irreps of that little group as listed by
    :func:`point_group_irreps`.  The character of (R|t), the map p -> R p + t, is
    exp(2 pi i (m1 u(t) + m2 v(t)) / det) * chi_R, where (u, v) are the
    superlattice coordinates of t scaled by det.

    Sublattices: n_sublat = 4 uses (x mod 2, y mod 2), 2 the checkerboard
    (x + y) mod 2, 1 a single block.  Within a sublattice the sites are labelled
    by increasing canonical (y, x).  Bonds of class 0 are the nearest neighbours
    (+x, +y), of class 1 the diagonal next-nearest neighbours (+x+y, +x-y).
    """
    cl = _Cluster(a1, a2)
    sites = sorted(cl.keys.values(), key=lambda p: (p[1], p[0]))
    N = len(sites)
    if n_sublat == 4:
        sub = lambda x, y: (x % 2) + 2 * (y % 2)
        if any(v % 2 for v in (*a1, *a2)):
            raise ValueError("4-sublattice split needs even superlattice vectors")
    elif n_sublat == 2:
        sub = lambda x, y: (x + y) % 2
        if any((v[0] + v[1]) % 2 for v in (a1, a2)):
            raise ValueError("checkerboard split needs even a1, a2 parities")
    elif n_sublat == 1:
        sub = lambda x, y: 0
    else:
        raise ValueError("n_sublat in {1, 2, 4}")
    blocks = [[s for s in sites if sub(*s) == X] for X in range(n_sublat)]
    if any(len(bk) != N // n_sublat for bk in blocks):
        raise ValueError("sublattices of unequal size")
    label_of = {}
    coords = np.zeros((N, 2))
    for X, bk in enumerate(blocks):
        for i, s in enumerate(bk):
            lab = X * (N // n_sublat) + i
            label_of[cl.key(*s)] = lab
            coords[lab] = s
    lab = lambda x, y: label_of[cl.key(x, y)]

    # point operations compatible with the cluster
    ops_all = range(len(C4V_OPS)) if point_ops is None else point_ops
    ops = []
    for r in ops_all:
        R = C4V_OPS[r]
        if all(cl.in_lattice(*(R @ np.array(v))) for v in (a1, a2)):
            ops.append(r)
    kphase = _kphase(cl, momentum)
    little = _little_group(cl, sites, ops, momentum)
    irreps = point_group_irreps([C4V_OPS[r] for r in little])
    chi_R = irreps[point_irrep]               # exponents e: chi = i**e
    denom = math.lcm(cl.det, 4)
    perm, pnum, names = [], [], []
    for ri, r in enumerate(little):
        R = C4V_OPS[r]
        for t in sites:
            row = np.empty(N, dtype=np.int32)
            for s in sites:
                img = R @ np.array(s) + np.array(t)
                row[lab(*s)] = lab(*img)
            perm.append(row)
            pnum.append((kphase(t) * (denom // cl.det) + chi_R[ri] * (denom // 4)) % denom)
            names.append(f"{C4V_NAMES[r]}+t{t}")
    bonds, bcls = [], []
    nn = [(1, 0), (0, 1)]
    nnn = [(1, 1), (1, -1)]
    for cls, dirs in ((0, nn), (1, nnn)):
        if cls == 1 and J2 == 0.0:
            continue
        for s in sites:
            for dx, dy in dirs:
                bonds.append((lab(*s), lab(s[0] + dx, s[1] + dy)))
                bcls.append(cls)
    bonds = np.array(bonds, dtype=np.int32)
    keyset = {tuple(sorted(b)) for b in bonds.tolist()}
    if len(keyset) != len(bonds):
        raise ValueError("cluster too small: duplicate bonds")
    n_classes = 2 if J2 != 0.0 else 1
    return Problem(
        name=name or f"square{N}_k{momentum}_ir{point_irrep}_sub{n_sublat}",
        n_sites=N, n_sublat=n_sublat, bonds=bonds,
        bond_class=np.array(bcls, dtype=np.int32), n_classes=n_classes,
        perm=np.array(perm, dtype=np.int32), phase_denom=denom,
        phase_num=np.array(pnum, dtype=np.int32),
        n_up=N // 2 if n_up is None else n_up,
        J=(float(J1), float(J2))[:n_classes], Jz=(1.0, 1.0)[:n_classes],
        coords=coords, sym_names=names)


def _kphase(cl, momentum):
    """Numerator (over det) of the momentum phase of a translation t."""
    m1, m2 = momentum

    def kphase(t):
        u, v = cl.key(*t)
        return (m1 * u + m2 * v) % cl.det
    return kphase


def _little_group(cl, sites, ops, momentum):
    """Point operations R with chi_k(R t) = chi_k(t) for every translation t."""
    kphase = _kphase(cl, momentum)
    return [r for r in ops
            if all(kphase(tuple(C4V_OPS[r] @ np.array(t))) == kphase(t) for t in sites)]


def n_point_irreps(a1, a2, momentum, point_ops=None) -> int:
    """Number of one-dimensional irreps of the little group of ``momentum``."""
    cl = _Cluster(a1, a2)
    sites = list(cl.keys.values())
    ops_all = range(len(C4V_OPS)) if point_ops is None else point_ops
    ops = [r for r in ops_all
           if all(cl.in_lattice(*(C4V_OPS[r] @ np.array(v))) for v in (a1, a2))]
    little = _little_group(cl, sites, ops, momentum)
    return len(point_group_irreps([C4V_OPS[r] for r in little]))


def square_torus(L: int, **kw) -> Problem:
    """L x L torus (a1 = (L, 0), a2 = (0, L))."""
    return square_cluster((L, 0), (0, L), **kw)


def tilted_square_40(**kw) -> Problem:
    """40-site square cluster spanned by (6, 2) and (-2, 6); point group C4."""
    return square_cluster((6, 2), (-2, 6), **kw)


def momenta(a1, a2):
    """Distinct momenta (m1, m2) of the cluster, as integer pairs modulo det."""
    cl = _Cluster(a1, a2)
    sites = list(cl.keys.values())
    seen, out = set(), []
    for m1 in range(cl.det):
        for m2 in range(cl.det):
            sig = tuple(((m1 * cl.key(*t)[0] + m2 * cl.key(*t)[1]) % cl.det) for t in sites)
            if sig not in seen:
                seen.add(sig)
                out.append((m1, m2))
            if len(out) == cl.n:
                return out
    return out


def point_group_irreps(mats):
    """All one-dimensional characters of a point group given by its matrices.

    A character is returned as a tuple of exponents e with chi = i**e, found by
    trying every assignment of fourth roots of unity and keeping the
    homomorphisms (enough for every subgroup of C4v).  The trivial irrep comes
    first; the rest are in lexicographic order of their exponent tuples.
    """
    n = len(mats)
    idx = {m.tobytes(): i for i, m in enumerate(mats)}
    prod = [[idx[(mats[a] @ mats[b]).astype(mats[0].dtype).tobytes()] for b in range(n)]
            for a in range(n)]
    out = []
    for es in itertools.product(range(4), repeat=n):
        if all((es[a] + es[b] - es[prod[a][b]]) % 4 == 0 for a in range(n) for b in range(n)):
            out.append(tuple(es))
    out.sort()
    return out


# ----------------------------------------------------------------------------
# state-keyed pseudo-random vectors
# ----------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014) on uint64."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _stream(states, seed: int, lane: int):
    s = np.asarray(states, dtype=np.uint64)
    with np.errstate(over="ignore"):
        off = np.uint64((int(seed) * 2 + lane + 1) * int(_GOLDEN) % (1 << 64))
        return splitmix64(s + off)


def state_uniform(states, seed: int) -> np.ndarray:
    """Coefficient x(s) in [-1, 1), a function of the configuration s and the seed."""
    z = _stream(states, seed, 0)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def state_gaussian(states, seed: int) -> np.ndarray:
    """Standard normal coefficient per configuration (Box-Muller on two streams)."""
    z1 = _stream(states, seed, 0)
    z2 = _stream(states, seed, 1)
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------
# the workloads: named configurations
# ----------------------------------------------------------------------------

def config_chain16(n_sublat: int = 2) -> Problem:
    """Heisenberg chain, N=16, periodic, J=1, Sz=0, C16, k=0."""
    return chain(16, n_sublat=n_sublat, k=0, n_up=8, J=1.0)


def config_square36(J2: float = 0.5, n_sublat: int = 4) -> Problem:
    """J1-J2 Heisenberg on the 6x6 torus, J1=1, Sz=0, 36 translations x C4v, Gamma-A1."""
    return square_torus(6, momentum=(0, 0), point_irrep=0, n_sublat=n_sublat,
                        J1=1.0, J2=J2, n_up=18, name=f"square36_J2={J2}_GammaA1")


def config_tilted40(n_sublat: int = 4) -> Problem:
    """Heisenberg J1 on the 40-site tilted square cluster, 40 translations x C4, Gamma-A."""
    return tilted_square_40(momentum=(0, 0), point_irrep=0, n_sublat=n_sublat,
                            J1=1.0, J2=0.0, n_up=20, name="tilted40_GammaA")


def config_square25_sectors(J2: float = 0.3, n_up_values=range(13, 26)):
    """Every (S^z = 1/2 .. 25/2, momentum, little-group 1-D irrep) sector of the 5x5 J1-J2
    torus (n_up = 13 .. 25), one sublattice (no split of 25 sites is stable under C4v)."""
    out = []
    for m in momenta((5, 0), (0, 5)):
        for ir in range(n_point_irreps((5, 0), (0, 5), m)):
            p = square_torus(5, momentum=m, point_irrep=ir, n_sublat=1, J1=1.0, J2=J2, n_up=0)
            for n_up in n_up_values:
                out.append(dataclasses.replace(p, n_up=n_up, name=f"sq25_k{m}_ir{ir}_up{n_up}"))
    return out
