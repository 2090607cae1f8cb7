#!/usr/bin/env python3
"""Write tests/golden/square36_e0.json: the oracle's ground-state energy of the 6x6
J1-J2 sector (J1 = 1, J2 = 0.5, S^z = 0, 36 translations x C4v, Gamma-A1,
D = 31,566,122).

Everything here comes from ``oracle/`` (plus the problem data and the seeded start
vector of ``workloads``):

* the basis by enumerating all 2^36 configurations and applying every one of the 288
  group elements (Alg. 3's loop on one process, Eqs. 3-4);
* the whole symmetry-adapted Hamiltonian stored row by row (the stored-matrix
  alternative of Sec. IV; about 2.3e9 entries, 28 GB of host memory);
* plain fp64 Lanczos with full reorthogonalisation on it, started from the
  state-keyed uniform vector with seed 1805 (the library's default start vector).

It takes about two hours on 8 host cores.  Run from the repository root:

    python tests/golden/make_square36_e0.py [--cache DIR]

``--cache DIR`` keeps the oracle basis there (basis.npy, stab.npy) so that a rerun
skips the enumeration.
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "square36_e0.json")


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default=None)
    ap.add_argument("--seed", type=int, default=1805)
    args = ap.parse_args()
    p = workloads.config_square36(0.5)
    t_all = time.time()
    D_formula = oracle.dimension_formula(p)
    log(f"projection count D = {D_formula}")
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
    assert bs.size == D_formula, (bs.size, D_formula)
    assert np.all(bs[1:] > bs[:-1])
    t0 = time.time()
    S = oracle.stored_matrix(p, (bs, stab), chunk_rows=1 << 20,
                             progress=lambda r, D: log(f"  rows {r}/{D}"))
    t_build = time.time() - t0
    log(f"stored matrix: {S.nnz} off-diagonal entries in {t_build:.0f} s")
    v0 = workloads.state_uniform(bs, args.seed)
    # one timed stored-matrix product (the paper's stored-matrix alternative, host cores)
    S.matvec(v0)
    t0 = time.time()
    S.matvec(v0)
    t_spmv = time.time() - t0
    log(f"stored-matrix product: {t_spmv:.2f} s")
    t0 = time.time()
    E0, alpha, beta, steps = oracle.lanczos(S.matvec, v0, max_steps=300, tol=1e-13)
    t_lz = time.time() - t0
    log(f"E0 = {E0!r} after {steps} steps ({t_lz:.0f} s)")
    out = {
        "what": "oracle ground-state energy of the 6x6 J1-J2 torus sector (J1=1, J2=0.5, "
                "Sz=0, 36 translations x C4v = 288 elements, Gamma-A1)",
        "source": "tests/golden/make_square36_e0.py (oracle/ only: brute-force basis over "
                  "2^36 configurations, stored symmetry-adapted matrix, fp64 Lanczos with "
                  "full reorthogonalisation)",
        "dim": int(bs.size),
        "offdiag_terms": int(S.nnz),
        "start_vector": f"workloads.state_uniform(basis, {args.seed})",
        "E0": float(E0),
        "lanczos_steps": int(steps),
        "lanczos_tol": 1e-13,
        "alpha": [float(a) for a in alpha[:8]],
        "beta": [float(b) for b in beta[:8]],
        "stored_matrix_product": {
            "seconds": t_spmv, "cores": oracle.max_threads(),
            "nonzeros_per_s": (bs.size + S.nnz) / t_spmv,
            "host": f"{platform.machine()} {platform.processor() or ''}".strip(),
            "note": "CSR (uint32 columns, fp64 values), OpenMP over rows"},
        "build_seconds": t_build,
        "total_seconds": time.time() - t_all,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    log(f"wrote {OUT}")


if __name__ == "__main__":
    main()
