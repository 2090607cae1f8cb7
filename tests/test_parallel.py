"""Row-sharded product and Lanczos with world sizes 2 and 3 on CPU (gloo).

The sharding logic (partition, all-gather of the input slices, scalar all-reduces)
is the product code in paper_1804_05028_gb300.parallel; the local rows come from the
oracle's matrix here, because the CUDA kernel needs a GPU (it is covered by the GPU
parity tests through the same ed_apply_H_rows entry point)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1804_05028_gb300.parallel import row_partition


def test_row_partition_covers_and_balances():
    for D, world in [(10, 3), (1, 4), (0, 2), (810, 2), (1000, 7)]:
        parts = row_partition(D, world)
        assert parts[0][0] == 0 and parts[-1][1] == D
        assert all(a <= b for a, b in parts)
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        # blocks of ceil(D / world) rows back to back, so the gathered slices need no
        # reordering: every block starts at r * m
        m = -(-D // world) if D else 0
        assert all(a == min(r * m, D) and b - a <= m for r, (a, b) in enumerate(parts))
    w = np.r_[np.full(50, 10.0), np.ones(50)]
    parts = row_partition(100, 2, w)
    loads = [w[a:b].sum() for a, b in parts]
    assert abs(loads[0] - loads[1]) <= 10.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    import workloads as w
    from paper_1804_05028_gb300.parallel import ShardedOperator, sharded_lanczos
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = w.chain(16, 2, k=3, n_up=8)                # a complex sector
        H, bs, _ = oracle.hamiltonian(p)
        Hc = H.tocsr()

        def local_apply(x_full, r0, r1):
            return torch.from_numpy(Hc[r0:r1] @ x_full.numpy())

        op = ShardedOperator(local_apply, bs.size, rank, world)
        x = w.state_uniform(bs, 1804) + 1j * w.state_uniform(bs, 1805)
        y_local = op.matvec(torch.from_numpy(x[op.r0:op.r1]))
        ok_mv = np.abs(y_local.numpy() - (Hc @ x)[op.r0:op.r1]).max() < 1e-13
        # a weighted partition (uneven slices, gathered through a reordering copy)
        wts = np.linspace(1.0, 5.0, bs.size)
        opw = ShardedOperator(local_apply, bs.size, rank, world, weights=wts)
        for _ in range(2):         # the preallocated buffers are reused
            y_w = opw.matvec(torch.from_numpy(x[opw.r0:opw.r1]))
            ok_mv = ok_mv and np.abs(y_w.numpy() - (Hc @ x)[opw.r0:opw.r1]).max() < 1e-13
        v0 = torch.from_numpy(x[op.r0:op.r1].copy())
        e, steps, a, b = sharded_lanczos(op, v0)
        e_ref = np.linalg.eigvalsh(H.toarray())[0]
        out[rank] = (bool(ok_mv), float(e), float(e_ref))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])          # 3 ranks: slices of unequal length
def test_sharded_lanczos_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
        assert pr.exitcode == 0
    for r in range(world):
        ok, e, e_ref = out[r]
        assert ok
        assert abs(e - e_ref) < 1e-10 * abs(e_ref)
    assert len({out[r][1] for r in range(world)}) == 1   # every rank holds the same E0
