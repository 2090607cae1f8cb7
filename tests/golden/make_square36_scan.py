#!/usr/bin/env python3
"""Write tests/golden/square36_scan_e0.json: the oracle's ground-state energies of the
6x6 J1-J2 sector (J1 = 1, S^z = 0, 36 translations x C4v, Gamma-A1, D = 31,566,122) at
J2 = 0.40, 0.45, 0.55 and 0.60 (0.50 is tests/golden/square36_e0.json).

Everything here comes from ``oracle/`` (plus the problem data and the seeded start
vector of ``workloads``):

* the basis by enumerating all 2^36 configurations and applying every group element
  (Alg. 3 on one process, Eqs. 3-4);
* H is linear in the exchange of each coupling class (Eq. 21), so the stored
  symmetry-adapted matrix is built once per class with that class's exchange alone:
  H(J2) = H_1 + J2 H_2 (about 1.2e9 entries each, 28 GB of host memory together);
* plain fp64 Lanczos with full reorthogonalisation on H(J2), started from the
  state-keyed uniform vector with seed 1805 (the library's default start vector).

It takes about three hours on 8 host cores.  Run from the repository root:

    python tests/golden/make_square36_scan.py [--cache DIR]

``--cache DIR`` reads or keeps the oracle basis there (basis.npy, stab.npy).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "square36_scan_e0.json")
SCAN = (0.40, 0.45, 0.55, 0.60)


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default=None)
    ap.add_argument("--seed", type=int, default=1805)
    args = ap.parse_args()
    p = workloads.config_square36(0.5)
    t_all = time.time()
    bs = stab = None
    if args.cache and os.path.exists(os.path.join(args.cache, "basis.npy")):
        bs = np.load(os.path.join(args.cache, "basis.npy"))
        stab = np.load(os.path.join(args.cache, "stab.npy"))
        log(f"basis from cache: {bs.size}")
    if bs is None:
        t0 = time.time()
        bs, stab = oracle.basis(p)
        log(f"oracle basis: {bs.size} states in {time.time() - t0:.0f} s")
        if args.cache:
            os.makedirs(args.cache, exist_ok=True)
            np.save(os.path.join(args.cache, "basis.npy"), bs)
            np.save(os.path.join(args.cache, "stab.npy"), stab)
    assert bs.size == oracle.dimension_formula(p)
    assert np.all(bs[1:] > bs[:-1])
    parts = []
    t0 = time.time()
    for c in range(p.n_classes):
        J = [0.0] * p.n_classes
        J[c] = 1.0
        S = oracle.stored_matrix(p.with_couplings(J, p.Jz), (bs, stab), chunk_rows=1 << 20,
                                 progress=lambda r, D: log(f"  class {c}: rows {r}/{D}")
                                 if r % (1 << 24) < (1 << 20) or r == D else None)
        log(f"class {c}: {S.nnz} off-diagonal entries")
        parts.append(S)
    t_build = time.time() - t0
    v0 = workloads.state_uniform(bs, args.seed)
    out = {"what": "oracle ground-state energies of the 6x6 J1-J2 torus sector (J1=1, Sz=0, "
                   "36 translations x C4v = 288 elements, Gamma-A1) for several J2",
           "source": "tests/golden/make_square36_scan.py (oracle/ only: brute-force basis over "
                     "2^36 configurations, one stored symmetry-adapted matrix per coupling "
                     "class, fp64 Lanczos with full reorthogonalisation on H1 + J2 H2)",
           "dim": int(bs.size), "offdiag_terms_per_class": [int(S.nnz) for S in parts],
           "start_vector": f"workloads.state_uniform(basis, {args.seed})",
           "lanczos_tol": 1e-13, "build_seconds": t_build,
           "host": f"{platform.machine()} {oracle.max_threads()} threads", "scan": []}
    for J2 in SCAN:
        t0 = time.time()
        E0, alpha, beta, steps = oracle.lanczos(
            lambda x: parts[0].matvec(x) + J2 * parts[1].matvec(x), v0, max_steps=300, tol=1e-13)
        log(f"J2 = {J2}: E0 = {E0!r} after {steps} steps ({time.time() - t0:.0f} s)")
        out["scan"].append({"J2": J2, "E0": float(E0), "lanczos_steps": int(steps),
                            "alpha": [float(a) for a in alpha[:5]],
                            "beta": [float(b) for b in beta[:5]]})
        out["total_seconds"] = time.time() - t_all
        with open(OUT, "w") as f:   # written after every point
            json.dump(out, f, indent=1)
            f.write("\n")
    log(f"wrote {OUT}")


if __name__ == "__main__":
    main()
