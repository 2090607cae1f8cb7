#!/usr/bin/env python3
"""Throughput of the symmetry-adapted matrix-free H x inside Lanczos on GB300.

A step is one Lanczos iteration on the sector: the row-pull product y = H v
(representative search by sublattice coding, Limits lookup, gather) with the fused
<v, Hv> partials, the three-term update with the ||w|| partials, and the scaling of
the next vector.  Both precisions are timed on the same sector and start vector:
fp64 vectors, and fp32 vectors with fp64 alpha/beta and tridiagonal solve ("mixed").
The headline is the mixed form when its ground-state energy agrees with the fp64
one to |dE0/E0| <= 1e-9, else the fp64 form.

Metric: symmetrised H x nonzeros per second = (D diagonal terms + off-diagonal terms
whose target survives the projection) per product x products per second, summed over
ranks (each rank runs its own replica of the sector; weak scaling).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--batch-only]
       (N > 1: launched by torch.distributed.run, one rank per GPU)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "Symmetrized H·v nonzeros/s + HBM roofline %, mixed vs FP64 at |ΔE0/E0|≤1e-9"
UNIT = "nonzeros/s"
WORKLOADS = {
    "square36": ("J1-J2 Heisenberg 6x6 torus, J1=1 J2=0.5, Sz=0, 36 translations x C4v "
                 "(288), Gamma-A1", lambda: workloads.config_square36(0.5)),
    "tilted40": ("Heisenberg J1 40-site tilted square (6,2),(-2,6), Sz=0, 40 translations x "
                 "C4 (160), Gamma-A", workloads.config_tilted40),
    "chain16": ("Heisenberg chain N=16 periodic, Sz=0, C16, k=0", workloads.config_chain16),
}
# the product kernels and the code that lays out the tables and the index they read
KERNEL_SOURCES = ["paper_1804_05028_gb300/csrc/apply.cu",
                  "paper_1804_05028_gb300/csrc/apply_fast.cu",
                  "paper_1804_05028_gb300/csrc/sced_internal.cuh",
                  "paper_1804_05028_gb300/csrc/dfloat.cuh",
                  "paper_1804_05028_gb300/csrc/basis.cu",
                  "paper_1804_05028_gb300/csrc/capi.cu"]


def _code_only(src: str) -> str:
    """The source without comments and with whitespace collapsed, so that a comment edit
    does not detach the committed counters from the code they were taken on."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return " ".join(src.split())


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def profiled(workload: str, key: str, dtype: str):
    """A per-launch counter of the product kernel from the committed ncu summary
    (`traffic_bytes_per_launch`: dram__bytes_read.sum + dram__bytes_write.sum;
    `warp_instructions_per_launch`: smsp__inst_executed.sum), if the kernel source has
    not changed since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", f"apply_h_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(rf"{key}\[{dtype}\]:\s*([0-9]+)\s+source_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(2) != kernel_hash():
        return None
    return int(m.group(1))


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def alg_bytes(D: int, n_off: int, vec_bytes: int) -> int:
    """Bytes the method must move per product: per row the state (8), |Stab| (2), x_i and
    y_i; per off-diagonal term one gathered x_j."""
    return D * (8 + 2 + 2 * vec_bytes) + n_off * vec_bytes


def sector_bytes(D: int, n_off: int, vec_bytes: int) -> int:
    """As alg_bytes, but each random x_j gather costs the whole 32-byte DRAM sector it
    sits in (the bound if no gathered x_j ever hit in L2)."""
    return D * (8 + 2 + 2 * vec_bytes) + n_off * 32


def oracle_sample(p, n_cfg: int, seed: int):
    """Representatives of the sector found by the oracle itself: random configurations with
    n_up up spins, their brute-force representatives, the surviving ones, sorted and
    unique (the oracle cannot enumerate C(36,18) configurations in a bench run)."""
    import oracle
    rng = np.random.default_rng(seed)
    N, n_up = p.n_sites, p.n_up
    cfg = np.zeros(n_cfg, np.uint64)
    for a in range(0, n_cfg, 1 << 16):           # n_up distinct sites per configuration
        m = min(n_cfg, a + (1 << 16)) - a
        sites = np.argsort(rng.random((m, N)), axis=1)[:, :n_up].astype(np.uint64)
        cfg[a:a + m] = np.bitwise_or.reduce(np.uint64(1) << sites, axis=1)
    rep, _, _, kept = oracle.representatives(p, cfg)
    return np.unique(rep[kept])


def cpu_baseline(p, seconds: float, seed: int = 7):
    """The oracle's matrix-free rows (brute-force representatives) on a sample of rows,
    sized to about `seconds` of work on the host cores."""
    import oracle
    xf = lambda q: workloads.state_uniform(q, 1804)
    reps = oracle_sample(p, 1 << 18, seed)
    reps = reps[np.random.default_rng(seed).permutation(reps.size)]   # unbiased prefixes
    oracle.rows(p, reps[:16], xf)              # load the library, start the thread pool
    n, dt = 64, 0.0
    while True:                                # grow the calibration sample to >= 1 s
        pick = reps[:min(n, reps.size)]
        t0 = time.perf_counter()
        oracle.rows(p, pick, xf)
        dt = time.perf_counter() - t0
        if dt >= 1.0 or n >= reps.size:
            break
        n *= 4
    n = int(min(reps.size, max(64, n * seconds / max(dt, 1e-3))))
    pick = reps[:n]
    t0 = time.perf_counter()
    oracle.rows(p, pick, xf)
    dt = time.perf_counter() - t0
    _, nt, _, _ = oracle.columns(p, pick)
    nnz = int(n + nt.sum())
    return {"value": nnz / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} representatives found by the oracle from random configurations "
                      f"(matrix-free brute-force rows, fp64), {nnz} nonzeros in {dt:.1f}s"}


def stored_matrix_record(workload: str):
    """The oracle's stored-matrix product (the alternative of Sec. IV) as timed when the
    committed oracle E0 of this workload was written (tests/golden), for context: the
    28 GB matrix takes over an hour to build, so it is not rebuilt here."""
    path = os.path.join(ROOT, "tests", "golden", f"{workload}_e0.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    m = g.get("stored_matrix_product")
    if not m:
        return None
    return {"value": m["nonzeros_per_s"], "unit": UNIT, "cores": m["cores"],
            "seconds_per_product": m["seconds"], "build_seconds": g.get("build_seconds"),
            "host": m.get("host"), "kind": "oracle stored matrix (CSR), fp64",
            "note": "timed on the host that wrote " + os.path.relpath(path, ROOT) +
                    ", not in this run"}


def bench_batch(ed, torch, steps: int):
    """All 572 sectors of the 5x5 J1-J2 torus (S^z = 1/2 .. 25/2, every momentum and
    little-group 1-D irrep) in one persistent, graph-replayed launch with block vectors
    k = 1, 4, 8 (fp32 / complex fp32, Gaussian), and the same work through the plain
    per-sector product (ed_apply_H once per sector and vector, fp32 and fp64).  Returns
    per-k throughput in nonzero-vector products per second."""
    t0 = time.time()
    probs = workloads.config_square25_sectors(0.3)
    bases = ed.build_sectors(probs)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    nnz = 0
    per = []   # (D, off-diagonal terms, bytes per vector entry) of each non-empty sector
    for B in bases:
        if B.dim:
            t = B.count_terms()[1]
            nnz += B.dim + t
            per.append((B.dim, t, 4 if B.is_real else 8))
    pk, pk_kind = peaks()
    out = {"workload": "square25 J1-J2 (J2=0.3), 572 sectors, one launch", "sectors": len(bases),
           "dim_total": int(sum(B.dim for B in bases)), "nonzeros_per_product": nnz,
           "build_s": build_s,
           "l2": "inputs larger than L2: 6 whole-lattice tables of 268 MB each, basis %d MB"
                 % (sum(d for d, _, _ in per) * 8 >> 20)}
    g = torch.Generator(device="cuda").manual_seed(1804)
    nz = [B for B in bases if B.dim]
    for k in (1, 4, 8):
        xs = [torch.randn(B.dim * k, dtype=torch.float32 if B.is_real else torch.complex64,
                          device="cuda", generator=g) for B in bases]
        ys = [torch.empty_like(x) for x in xs]
        bt = ed.Batch(bases, k=k)
        bt.set_vectors(xs, ys)
        bt.apply()                         # tunes the tile, captures the graph
        for _ in range(3):
            bt.apply()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            bt.apply()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # per row: state, |Stab|, k entries of x_i and y_i; per term: k gathered entries
        ab = sum(d * (8 + 2 + 2 * k * b) + t * k * b for d, t, b in per)
        ach = ab / (ms * 1e-3) / 1e9
        # the same work through the plain per-sector product: k separate vectors per sector
        plain = {}
        cols = [(B, x.view(B.dim, k)) for B, x in zip(bases, xs) if B.dim]
        for name, real_dt, cplx_dt in (("f32", torch.float32, torch.complex64),
                                       ("f64", torch.float64, torch.complex128)):
            vx = [[X[:, v].contiguous().to(real_dt if B.is_real else cplx_dt) for v in range(k)]
                  for B, X in cols]
            vy = [[torch.empty_like(c) for c in row] for row in vx]
            def run():
                for (B, _), xr, yr in zip(cols, vx, vy):
                    for xc, yc in zip(xr, yr):
                        B.apply_H(xc, yc)
            run()
            torch.cuda.synchronize()
            reps = max(1, steps // 4)
            e0.record()
            for _ in range(reps):
                run()
            e1.record()
            torch.cuda.synchronize()
            plain[name] = e0.elapsed_time(e1) / reps
            del vx, vy
        out[f"k{k}"] = {"ms_per_apply": ms, "value": nnz * k / (ms * 1e-3),
                        "unit": "nonzero-vector products/s", **bt.info(),
                        "plain_f32_ms": plain["f32"], "plain_f64_ms": plain["f64"],
                        "batched_ms": ms,
                        "speedup_vs_plain_f32": plain["f32"] / ms,
                        "speedup_vs_plain_f64": plain["f64"] / ms,
                        "plain": f"ed_apply_H per sector and vector: {len(nz) * k} launches",
                        "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                     "frac": ach / pk["hbm_gbs"], "peak_kind": pk_kind,
                                     "alg_bytes_per_launch": ab}}
        bt.close()
        del xs, ys
    for B in bases:
        B.close()
    return out


def run_reference(args):
    """Reference arm: the oracle as it stands, on the host cores, same metric and config."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    desc, mk = WORKLOADS[args.workload]
    p = mk()
    # representatives of the sector from the oracle itself (it cannot enumerate C(36,18)
    # configurations)
    rng = np.random.default_rng(11)
    reps = oracle_sample(p, 4096, 11)
    xf = lambda q: workloads.state_uniform(q, 1804)
    # calibrate rows per step to about one second
    oracle.rows(p, reps[:16], xf)
    m = min(reps.size, 256)
    t0 = time.perf_counter()
    oracle.rows(p, reps[:m], xf)
    per_row = max((time.perf_counter() - t0) / m, 1e-6)
    n_rows = int(max(16, min(reps.size, 1.0 / per_row)))
    step_rows = [reps[np.sort(rng.choice(reps.size, n_rows, replace=False))] for _ in range(args.warmup + args.steps)]
    for k in range(args.warmup):
        oracle.rows(p, step_rows[k], xf)
    nnz = 0
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        oracle.rows(p, step_rows[k], xf)
    dt = time.perf_counter() - t0
    for k in range(args.warmup, args.warmup + args.steps):
        _, nt, _, _ = oracle.columns(p, step_rows[k])
        nnz += int(nt.sum()) + step_rows[k].size
    value = nnz / dt
    cfg = {"workload": args.workload, "description": desc, "dim": oracle.dimension_formula(p),
           "n_sublat": p.n_sublat, "n_sym": p.n_sym, "rows_per_step": n_rows}
    gpath = os.path.join(ROOT, "tests", "golden", f"{args.workload}_e0.json")
    if os.path.exists(gpath):   # the oracle's own term count of the whole sector
        g = json.load(open(gpath))
        cfg["offdiag_terms_per_product"] = g["offdiag_terms"]
        cfg["nonzeros_per_product"] = g["dim"] + g["offdiag_terms"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (state-keyed uniform[-1,1) vectors, seed 1804)",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{n_rows} sampled representative rows per step, matrix-free brute force"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def bench_sector(ed, torch, workload, p, steps, warmup, ctx, accuracy=True, full_reorth=False):
    """Lanczos steps on one sector, fp64 and mixed (fp32 vectors, fp64 scalars and local
    reorthogonalisation): per-step throughput, the product's roofline, the accuracy of the
    mixed form against fp64, and the end-to-end product through the host-buffer entry
    point.  With full_reorth the mixed accuracy run is repeated with the whole Krylov
    basis stored and reorthogonalised against."""
    world, rank, barrier, allmax = ctx["world"], ctx["rank"], ctx["barrier"], ctx["allmax"]
    B = ed.build_basis_from(p)
    info = B.info()
    D = info["dim"]
    n_flip, n_off = B.count_terms()
    nnz = D + n_off

    # accuracy of the mixed form against fp64 (untimed): full Lanczos runs to convergence
    acc = {}
    if accuracy:
        want_psi = D < 1e8   # the ground state costs a second pass; skip it on the 40-site sector
        psi64 = torch.empty(D, dtype=torch.float64, device="cuda") if want_psi else None
        r64 = B.lanczos(dtype=torch.float64, max_steps=400, psi=psi64)
        del psi64
        psi32 = torch.empty(D, dtype=torch.float32, device="cuda") if want_psi else None
        r32 = B.lanczos(dtype=torch.float32, max_steps=400, psi=psi32)
        acc = {"E0_f64": r64["E0"], "steps_f64": r64["steps"],
               "E0_mixed": r32["E0"], "steps_mixed": r32["steps"],
               "dE0_rel_mixed": abs(r32["E0"] - r64["E0"]) / abs(r64["E0"]),
               "reorth": "local (second Gram-Schmidt sweep against v_j, v_j-1, fp64 dots)"}
        if want_psi:
            acc.update({"rq_f64": r64["rq"], "rq_mixed": r32["rq"],
                        "dE0_rel_mixed_rq": abs(r32["rq"] - r64["E0"]) / abs(r64["E0"]),
                        "dE0_rel_f64_rq": abs(r64["rq"] - r64["E0"]) / abs(r64["E0"])})
        if full_reorth:
            m = r32["steps"] + 1
            kry = torch.empty((m + 1) * D, dtype=torch.float32, device="cuda")
            psi32 = torch.empty(D, dtype=torch.float32, device="cuda")
            rf = B.lanczos(dtype=torch.float32, max_steps=m, psi=psi32, reorth="full", krylov=kry)
            acc["full_reorth_mixed"] = {
                "E0": rf["E0"], "steps": rf["steps"], "rq": rf["rq"],
                "dE0_rel": abs(rf["E0"] - r64["E0"]) / abs(r64["E0"]),
                "dE0_rel_rq": abs(rf["rq"] - r64["E0"]) / abs(r64["E0"]),
                "reorth_ms_per_step": rf["ms_reorth"] / rf["steps"],
                "apply_ms_per_step": rf["ms_apply"] / rf["steps"],
                "store_bytes": kry.numel() * 4}
            del kry, psi32

    pk, pk_kind = peaks()
    n_sm = ctx["n_sm"]
    results = {}
    for name, dt, vb in (("f64", torch.float64, 8), ("mixed", torch.float32, 4)):
        # three Lanczos vectors; with fp32 a fourth for the low words of the product
        work = torch.empty((3 if name == "f64" else 4) * D, dtype=dt, device="cuda")
        B.lanczos(dtype=dt, fixed_steps=max(warmup, 1), work=work)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(ctx["local"]) as cs:
            e0.record()
            r = B.lanczos(dtype=dt, fixed_steps=steps, work=work)
            e1.record()
            torch.cuda.synchronize()
        barrier()
        ms = allmax(e0.elapsed_time(e1))
        apply_ms = r["ms_apply"] / steps
        ab = alg_bytes(D, n_off, vb)
        achieved = ab / (apply_ms * 1e-3) / 1e9
        clk = cs.summary()
        # instruction-issue roof: every SM issues at most one warp instruction per cycle on
        # each of its 4 schedulers, at the SM clock sampled during the timed region
        winst = profiled(workload, "warp_instructions_per_launch", name)
        issue_peak = 4 * n_sm * clk["sm_mhz"] * 1e6 / 1e9 if clk.get("sm_mhz") else None
        issue = None
        if winst is not None and issue_peak:
            ia = winst / (apply_ms * 1e-3) / 1e9
            issue = {"bound": "issue", "achieved": ia, "peak": issue_peak, "unit": "Gwarp-inst/s",
                     "frac": ia / issue_peak, "warp_instructions_per_launch": winst,
                     "peak_kind": f"4 schedulers x {n_sm} SMs x sampled SM clock"}
        results[name] = {
            "value": world * nnz * steps / (ms * 1e-3), "ms_per_step": ms / steps,
            "apply_ms": apply_ms, "reorth_ms": r["ms_reorth"] / steps, "clocks": clk,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "peak_kind": pk_kind,
                         "traffic": profiled(workload, "traffic_bytes_per_launch", name),
                         "alg_bytes_per_launch": ab,
                         "sector_bytes_per_launch": sector_bytes(D, n_off, vb)},
            "roofline_issue": issue,
            # per step: product, three-term update, scale, and the local sweep's
            # multi-dot, coefficient reduction and update
            "gpu_launches": 6 * steps + 2,
        }
        del work

    ok_mixed = (not acc) or acc["dE0_rel_mixed"] <= 1e-9
    head_name = "mixed" if ok_mixed else "f64"

    # end to end through the host-buffer entry point: H2D of x, product, D2H of y per step
    hd = torch.float32 if ok_mixed else torch.float64
    xh = torch.from_numpy(workloads.state_uniform(B.export()[0], 1804)).to(hd).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(max(warmup, 1)):
        B.apply_H_host(xh, yh)
    barrier()
    e2e_steps = max(2, steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        B.apply_H_host(xh, yh)
    torch.cuda.synchronize()
    t_e2e = allmax(time.perf_counter() - t0)
    eb = xh.numel() * xh.element_size()
    e2e = {"value": world * nnz * e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": eb,
           "d2h_bytes_per_step": eb, "ms_per_step": 1000 * t_e2e / e2e_steps, "steps": e2e_steps,
           "what": "ed_apply_H_host: pinned host x -> device, product, device -> pinned host y"}
    del xh, yh
    cfg = {"dim": D, "offdiag_terms_per_product": n_off, "exchange_terms_per_product": n_flip,
           "nonzeros_per_product": nnz, "n_sublat": p.n_sublat, "n_sym": p.n_sym,
           "step": "one Lanczos iteration (apply_H with fused <v,Hv>, update with ||w||, "
                   "local reorthogonalisation sweep, scale)",
           "l2": "inputs larger than L2: basis %d MB, each vector %d MB" % (D * 8 >> 20, D * (4 if head_name == 'mixed' else 8) >> 20),
           "index": {k: info[k] for k in ("prefix_rank_bits", "prefix_raw_bits", "postfix_bits", "n_keys", "max_bucket")},
           "basis_build_ms": info["build_ms"], "steps": steps}
    B.close()
    return {"results": results, "headline": head_name, "accuracy": acc, "e2e": e2e, "config": cfg}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="square36", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 40-site sector that the default run adds as 'large'")
    ap.add_argument("--batch-only", action="store_true",
                    help="time only the batched 5x5 sectors and print their JSON object")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_only:
        import torch
        import paper_1804_05028_gb300 as ed
        ed.build()
        print(json.dumps({"batch": bench_batch(ed, torch, max(args.steps, 5))}))
        return 0

    import torch
    import paper_1804_05028_gb300 as ed

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def allmax(v):
        if not dist:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    desc, mk = WORKLOADS[args.workload]
    p = mk()
    ed.build()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    ctx = {"world": world, "rank": rank, "local": local, "barrier": barrier, "allmax": allmax,
           "n_sm": n_sm}
    main_res = bench_sector(ed, torch, args.workload, p, args.steps, args.warmup, ctx,
                            accuracy=not args.no_accuracy, full_reorth=True)

    batch = None
    if not args.no_batch and args.workload == "square36":
        batch = bench_batch(ed, torch, max(args.steps, 5))

    large = None
    if not args.no_large and args.workload == "square36":
        _, mk40 = WORKLOADS["tilted40"]
        large = bench_sector(ed, torch, "tilted40", mk40(), max(2, args.steps // 6),
                             max(1, min(args.warmup, 2)), ctx, accuracy=not args.no_accuracy,
                             full_reorth=False)
        large = {"workload": "tilted40", "description": WORKLOADS["tilted40"][0], **large}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, args.cpu_seconds)
        sm = stored_matrix_record(args.workload)
        if sm:
            cpu["stored_matrix"] = sm

    if rank == 0:
        r = main_res
        head = r["results"][r["headline"]]
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 vectors / f64 scalars" if r["headline"] == "mixed" else "f64",
            "data": "synthetic (state-keyed uniform[-1,1) start vector, seed 1805)",
            "config": {"workload": args.workload, "description": desc, **r["config"],
                       "parallelism": f"replicas x{world}"},
            "roofline": head["roofline"], "roofline_issue": head["roofline_issue"],
            "clocks": head["clocks"], "gpu_launches": head["gpu_launches"],
            "e2e": r["e2e"], "cpu_baseline": cpu, "headline": r["headline"],
            "fp64": r["results"]["f64"], "mixed": r["results"]["mixed"], "accuracy": r["accuracy"],
            "batch": batch, "large": large, "n_sm": n_sm, "kernel_sha": kernel_hash(),
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
