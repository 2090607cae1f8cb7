#!/usr/bin/env python3
"""Write tests/golden/square36_hv.json: the oracle's product y = H x on the whole 6x6
J1-J2 sector (J1 = 1, J2 = 0.5, S^z = 0, 36 translations x C4v, Gamma-A1,
D = 31,566,122) for the state-keyed vector x = workloads.state_uniform(basis, 1804).

The product comes from ``oracle/`` alone: the basis by enumerating all 2^36
configurations (Alg. 3 on one process, Eqs. 3-4), the stored symmetry-adapted matrix
(the stored-matrix alternative of Sec. IV; 2.34e9 entries, 28 GB of host memory) and its
CSR product in fp64.  y itself (253 MB) is not stored; the file holds what pins every
row in aggregate and some rows one by one:

* <x, y>, ||y||^2 and sum(y);
* the sums of y over 256 consecutive row blocks of equal length (the last shorter);
* y at 1024 rows drawn with numpy's default_rng(1806), and the basis states of those
  rows.

It takes about 80 minutes on 8 host cores.  Run from the repository root:

    python tests/golden/make_square36_hv.py [--cache DIR] [--states-only]

``--cache DIR`` reads or keeps the oracle basis there (basis.npy, stab.npy).
``--states-only`` adds the sampled rows' basis states to an existing file without
rebuilding the matrix.
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "square36_hv.json")
N_BLOCKS = 256
N_SAMPLE = 1024


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default=None)
    ap.add_argument("--states-only", action="store_true")
    args = ap.parse_args()
    p = workloads.config_square36(0.5)
    t_all = time.time()
    bs = stab = None
    if args.cache and os.path.exists(os.path.join(args.cache, "basis.npy")):
        bs = np.load(os.path.join(args.cache, "basis.npy"))
        stab = np.load(os.path.join(args.cache, "stab.npy"))
        log(f"basis from cache: {bs.size}")
    if bs is None:
        bs, stab = oracle.basis(p)
        log(f"oracle basis: {bs.size} states")
        if args.cache:
            os.makedirs(args.cache, exist_ok=True)
            np.save(os.path.join(args.cache, "basis.npy"), bs)
            np.save(os.path.join(args.cache, "stab.npy"), stab)
    assert bs.size == oracle.dimension_formula(p)
    D = bs.size
    if args.states_only:
        out = json.load(open(OUT))
        out["sample_states"] = [int(v) for v in bs[np.array(out["sample_rows"])]]
        with open(OUT, "w") as f:
            json.dump(out, f)
            f.write("\n")
        log(f"added the sampled rows' states to {OUT}")
        return
    S = oracle.stored_matrix(p, (bs, stab), chunk_rows=1 << 20,
                             progress=lambda r, n: log(f"  rows {r}/{n}")
                             if r % (1 << 24) < (1 << 20) or r == n else None)
    log(f"stored matrix: {S.nnz} off-diagonal entries")
    x = workloads.state_uniform(bs, 1804)
    y = S.matvec(x)
    blk = -(-D // N_BLOCKS)
    rows = np.sort(np.random.default_rng(1806).choice(D, N_SAMPLE, replace=False))
    out = {"what": "oracle product y = H x on the 6x6 J1-J2 torus sector (J1=1, J2=0.5, Sz=0, "
                   "Gamma-A1), x = workloads.state_uniform(basis, 1804)",
           "source": "tests/golden/make_square36_hv.py (oracle/ only: brute-force basis, stored "
                     "symmetry-adapted matrix, fp64 CSR product)",
           "dim": int(D), "offdiag_terms": int(S.nnz),
           "x_dot_y": float(np.dot(x, y)), "y_norm2": float(np.dot(y, y)), "y_sum": float(y.sum()),
           "block_rows": int(blk),
           "block_sums": [float(y[a:a + blk].sum()) for a in range(0, D, blk)],
           "abs_block_sums": [float(np.abs(y[a:a + blk]).sum()) for a in range(0, D, blk)],
           "sample_seed": 1806, "sample_rows": [int(r) for r in rows],
           "sample_y": [float(v) for v in y[rows]],
           "sample_states": [int(v) for v in bs[rows]],
           "host": f"{platform.machine()} {oracle.max_threads()} threads",
           "total_seconds": time.time() - t_all}
    with open(OUT, "w") as f:
        json.dump(out, f)
        f.write("\n")
    log(f"wrote {OUT}")


if __name__ == "__main__":
    main()
