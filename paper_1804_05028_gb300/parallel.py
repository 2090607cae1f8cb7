"""Row-sharded product and Lanczos across ranks (one GPU per rank).

The row-wise pull makes rows independent: rank r owns the contiguous rows
[r0, r1) of the sorted basis and the matching slice of every vector.  One product is
an all-gather of the input slices followed by the local rows (``ed_apply_H_rows``);
the Lanczos scalars are all-reduced.  This replaces the paper's hash-of-prefix
placement and buffered all-to-all of (state, coefficient) pairs (Sec. IV, Alg. 4),
which exist to balance a push; the pull needs neither.

Every collective goes through ``torch.distributed``; the local product is a callable
so that the same driver runs with the CUDA library (NCCL) or with any other local
operator (gloo on CPU in the tests).
"""
from __future__ import annotations

import math
from typing import Callable, List, Tuple

import numpy as np

__all__ = ["row_partition", "ShardedOperator", "sharded_lanczos", "cuda_local_apply"]


def row_partition(D: int, world: int, weights=None) -> List[Tuple[int, int]]:
    """Contiguous row ranges, one per rank, balanced by ``weights`` (row costs; equal
    costs when None).  Every range is half-open; together they cover [0, D)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if weights is None:
        cuts = [(D * r) // world for r in range(world + 1)]
    else:
        w = np.asarray(weights, dtype=np.float64)
        if w.size != D:
            raise ValueError("one weight per row")
        c = np.concatenate([[0.0], np.cumsum(w)])
        targets = c[-1] * np.arange(world + 1) / world
        cuts = list(np.searchsorted(c, targets, side="left"))
        cuts[0], cuts[-1] = 0, D
        for r in range(1, world + 1):
            cuts[r] = max(cuts[r], cuts[r - 1])
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


class ShardedOperator:
    """y_local = (H x)[r0:r1] from x_local = x[r0:r1] on every rank.

    local_apply(x_full, r0, r1) -> y_local computes the rank's rows from the whole
    input vector (for the CUDA library: ``Basis.apply_H_rows``).
    """

    def __init__(self, local_apply: Callable, D: int, rank: int, world: int, weights=None,
                 group=None):
        import torch.distributed as dist
        self.dist = dist
        self.local_apply = local_apply
        self.D, self.rank, self.world, self.group = D, rank, world, group
        self.parts = row_partition(D, world, weights)
        self.r0, self.r1 = self.parts[rank]
        self.sizes = [b - a for a, b in self.parts]

    def gather(self, x_local):
        """All ranks' slices concatenated in row order (the exchange step)."""
        import torch
        if self.world == 1:
            return x_local
        m = max(self.sizes)
        pad = torch.zeros(m, dtype=x_local.dtype, device=x_local.device)
        pad[: x_local.numel()] = x_local
        bufs = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(bufs, pad, group=self.group)
        return torch.cat([b[:s] for b, s in zip(bufs, self.sizes)])

    def matvec(self, x_local):
        return self.local_apply(self.gather(x_local), self.r0, self.r1)

    def dot(self, a_local, b_local) -> float:
        import torch
        v = torch.sum(torch.conj(a_local) * b_local).real.to(torch.float64).reshape(1)
        if self.world > 1:
            self.dist.all_reduce(v, group=self.group)
        return float(v.item())


def _lowest_ritz(alpha, beta):
    from scipy.linalg import eigh_tridiagonal
    return float(eigh_tridiagonal(np.asarray(alpha), np.asarray(beta), eigvals_only=True,
                                  select="i", select_range=(0, 0))[0])


def sharded_lanczos(op: ShardedOperator, v0_local, max_steps: int = 300, tol: float = 1e-13):
    """Plain Lanczos over the row shards: the product needs one all-gather, each of
    alpha and beta one scalar all-reduce.  Returns (E0, steps, alphas, betas)."""
    v = v0_local / math.sqrt(op.dot(v0_local, v0_local))
    v_prev = None
    alphas, betas = [], []
    e_old = None
    for k in range(max_steps):
        w = op.matvec(v)
        a = op.dot(v, w)
        w = w - a * v - (betas[-1] * v_prev if betas else 0)
        b = math.sqrt(max(op.dot(w, w), 0.0))
        alphas.append(a)
        e = _lowest_ritz(alphas, betas)
        if e_old is not None and abs(e - e_old) < tol * max(1.0, abs(e)):
            return e, k + 1, np.array(alphas), np.array(betas)
        e_old = e
        if b < 1e-14 * max(1.0, abs(a)) or len(alphas) >= op.D:
            return e, k + 1, np.array(alphas), np.array(betas)
        betas.append(b)
        v_prev, v = v, w / b
    return e_old, max_steps, np.array(alphas), np.array(betas)


def cuda_local_apply(basis):
    """local_apply for ShardedOperator backed by the CUDA library (ed_apply_H_rows)."""
    def f(x_full, r0, r1):
        return basis.apply_H_rows(x_full, r0, r1)
    return f
