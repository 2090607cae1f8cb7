"""Command line: ground-state energies of symmetry sectors described in JSON.

    python -m paper_1804_05028_gb300 describe NAME [--n-up K] [-o FILE]
        write the descriptor of a built-in sector (chain16, square36, tilted40) as JSON
    python -m paper_1804_05028_gb300 run FILE [--dtype f64|f32] [--max-steps M] [--tol T]
                                         [--fixed-steps K] [--reorth local|none|full]
        build the sector's basis on the current GPU, run Lanczos, print one JSON line
        (--fixed-steps runs exactly K steps; --reorth full keeps the whole Krylov basis
        on the device and sweeps against it)

A descriptor holds the fields of a sector: sites, sublattice count, bonds and their
coupling classes, the group as site permutations (and optional spin-flip bits), the
1-D irrep as integer phases chi(g) = exp(2 pi i phase_num[g] / phase_denom), n_up,
and the couplings J, Jz per class (the arguments of ed_build_basis and ed_lanczos).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def _workloads():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads
    return workloads


def _describe(args) -> int:
    w = _workloads()
    makers = {"chain16": w.config_chain16, "square36": w.config_square36,
              "tilted40": w.config_tilted40}
    if args.name not in makers:
        print(f"unknown sector {args.name!r}; one of {sorted(makers)}", file=sys.stderr)
        return 2
    p = makers[args.name]()
    if args.n_up is not None:
        p = p.with_n_up(args.n_up)
    text = json.dumps(w.to_dict(p))
    if args.output:
        with open(args.output, "w") as f:
            f.write(text + "\n")
    else:
        print(text)
    return 0


def _run(args) -> int:
    import numpy as np
    import torch

    import paper_1804_05028_gb300 as ed
    with open(args.file) as f:
        d = json.load(f)
    t0 = time.perf_counter()
    B = ed.build_basis(d["n_sites"], d["n_sublat"], np.asarray(d["bonds"]), d["bond_class"],
                       d["n_classes"], np.asarray(d["perm"]), d["phase_num"], d["phase_denom"],
                       d["n_up"], J=d["J"], Jz=d["Jz"], flip=d.get("flip"))
    build_s = time.perf_counter() - t0
    out = {"name": d.get("name"), "dim": B.dim, "is_real": B.is_real, "build_s": build_s}
    if B.dim:
        real = B.is_real
        dt = {"f64": torch.float64 if real else torch.complex128,
              "f32": torch.float32 if real else torch.complex64}[args.dtype]
        r = B.lanczos(dtype=dt, max_steps=args.max_steps, tol=args.tol,
                      fixed_steps=args.fixed_steps, reorth=args.reorth)
        out.update({"E0": r["E0"], "steps": r["steps"], "converged": r["converged"],
                    "dtype": args.dtype, "reorth": args.reorth, "ms_total": r["ms_total"],
                    "ms_apply": r["ms_apply"], "ms_reorth": r["ms_reorth"]})
    print(json.dumps(out))
    B.close()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_1804_05028_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("describe", help="write a built-in sector as a JSON descriptor")
    a.add_argument("name")
    a.add_argument("--n-up", type=int, default=None)
    a.add_argument("-o", "--output", default=None)
    a = sub.add_parser("run", help="ground-state energy of a sector described in JSON")
    a.add_argument("file")
    a.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    a.add_argument("--max-steps", type=int, default=400)
    a.add_argument("--tol", type=float, default=1e-13)
    a.add_argument("--fixed-steps", type=int, default=0)
    a.add_argument("--reorth", choices=["local", "none", "full"], default="local")
    args = ap.parse_args(argv)
    try:
        return _describe(args) if args.cmd == "describe" else _run(args)
    except Exception as e:          # report library errors as one line and a status
        print(f"error: {e}", file=sys.stderr)
        return 1


if __name__ == "__main__":
    sys.exit(main())
