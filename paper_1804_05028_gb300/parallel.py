"""Row-sharded product and Lanczos across ranks (one GPU per rank).

The row-wise pull makes rows independent: rank r owns the contiguous rows
[r0, r1) of the sorted basis and the matching slice of every vector.  One product is
an all-gather of the input slices followed by the local rows (``ed_apply_H_rows``);
the Lanczos scalars are all-reduced.  This replaces the paper's hash-of-prefix
placement and buffered all-to-all of (state, coefficient) pairs (Sec. IV, Alg. 4),
which exist to balance a push; the pull needs neither.

Where the arithmetic runs:

* CUDA tensors: the local rows (``ed_apply_H_rows``), the local dot products
  (``ed_dot_noalloc``), the three-term update with its norm (``ed_axpy_norm``) and the
  scaling (``ed_scale``) all run in the library's kernels, in place on three rotating
  slices; torch provides the buffers and the collectives (NCCL).
* CPU tensors (the gloo tests): the same driver with torch's CPU operations, and any
  local operator (the oracle's matrix in the tests).
* On the host, every rank: the tridiagonal eigenvalue (scipy), a few scalars per step.

The all-gather writes into one preallocated buffer per dtype and device: with the
default partition (blocks of ceil(D / world) rows, the last one shorter) the gathered
slices lie back to back, so the full input vector is a view of that buffer and no
per-product copy is made.  A weighted partition gathers into the same buffer and then
copies the slices once into a preallocated full vector.
"""
from __future__ import annotations

import math
from typing import Callable, List, Tuple

import numpy as np

__all__ = ["row_partition", "ShardedOperator", "sharded_lanczos", "cuda_local_apply"]


def row_partition(D: int, world: int, weights=None) -> List[Tuple[int, int]]:
    """Contiguous row ranges, one per rank; together they cover [0, D).

    Without weights: blocks of m = ceil(D / world) rows (the last ones shorter or empty),
    the layout whose all-gather needs no reordering.  With ``weights`` (row costs): cuts
    that balance the summed costs."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if weights is None:
        m = -(-D // world) if D else 0
        return [(min(r * m, D), min((r + 1) * m, D)) for r in range(world)]
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

    local_apply(x_full, r0, r1[, out]) -> y_local computes the rank's rows from the whole
    input vector (for the CUDA library: ``Basis.apply_H_rows``); it receives ``out`` when
    it has an attribute ``accepts_out`` set.
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
        self.m = max(self.sizes) if self.sizes else 0
        self.back_to_back = all(a == min(r * self.m, D) for r, (a, _) in enumerate(self.parts))
        self._bufs = {}

    def _buffers(self, like):
        import torch
        key = (like.dtype, str(like.device))
        if key not in self._bufs:
            pad = torch.zeros(self.m, dtype=like.dtype, device=like.device)
            flat = torch.empty(self.world * self.m, dtype=like.dtype, device=like.device)
            full = None if self.back_to_back else torch.empty(self.D, dtype=like.dtype,
                                                              device=like.device)
            extra = {}
            if like.is_cuda:
                extra["dot"] = torch.zeros(2, dtype=torch.float64, device=like.device)
                extra["norm2"] = torch.zeros(1, dtype=torch.float64, device=like.device)
                extra["scratch"] = torch.zeros(4096, dtype=torch.float64, device=like.device)
            self._bufs[key] = (pad, flat, full, extra)
        return self._bufs[key]

    def gather(self, x_local):
        """All ranks' slices in row order (the exchange step), in preallocated buffers."""
        if self.world == 1:
            return x_local
        pad, flat, full, _ = self._buffers(x_local)
        pad[: x_local.numel()].copy_(x_local)      # the tail of pad stays zero
        self.dist.all_gather_into_tensor(flat, pad, group=self.group)
        if self.back_to_back:
            return flat[: self.D]
        for r, (a, b) in enumerate(self.parts):
            full[a:b].copy_(flat[r * self.m: r * self.m + (b - a)])
        return full

    def matvec(self, x_local, out=None):
        x = self.gather(x_local)
        if out is not None and getattr(self.local_apply, "accepts_out", False):
            return self.local_apply(x, self.r0, self.r1, out)
        return self.local_apply(x, self.r0, self.r1)

    def _allreduce(self, t):
        if self.world > 1:
            self.dist.all_reduce(t, group=self.group)
        return t

    def dot(self, a_local, b_local) -> float:
        """Re <a, b> over all ranks."""
        import torch
        if a_local.is_cuda:
            import paper_1804_05028_gb300 as ed
            out = self._buffers(a_local)[3]["dot"]
            ed.dot_noalloc(a_local, b_local, out)
            v = out[:1]
        else:
            v = torch.sum(torch.conj(a_local) * b_local).real.to(torch.float64).reshape(1)
        return float(self._allreduce(v).item())

    def axpy_norm(self, w, v, vprev, a: float, b: float) -> float:
        """w <- w - a v - b vprev in place (vprev may be None); returns ||w||^2 over all
        ranks."""
        import torch
        if w.is_cuda:
            import paper_1804_05028_gb300 as ed
            ex = self._buffers(w)[3]
            ed.axpy_norm(w, v, vprev, a, b, ex["scratch"], ex["norm2"])
            n2 = ex["norm2"]
        else:
            w.sub_(a * v)
            if vprev is not None:
                w.sub_(b * vprev)
            n2 = torch.sum(torch.conj(w) * w).real.to(torch.float64).reshape(1)
        return float(self._allreduce(n2).item())

    def scale(self, x, s: float):
        if x.is_cuda:
            import paper_1804_05028_gb300 as ed
            ed.scale(x, s)
        else:
            x.mul_(s)
        return x


def _lowest_ritz(alpha, beta):
    from scipy.linalg import eigh_tridiagonal
    return float(eigh_tridiagonal(np.asarray(alpha), np.asarray(beta), eigvals_only=True,
                                  select="i", select_range=(0, 0))[0])


def sharded_lanczos(op: ShardedOperator, v0_local, max_steps: int = 300, tol: float = 1e-13):
    """Plain Lanczos over the row shards, in place on three rotating slices: the product
    needs one all-gather, alpha and beta one scalar all-reduce each.  Returns
    (E0, steps, alphas, betas)."""
    import torch
    v = v0_local.clone()
    op.scale(v, 1.0 / math.sqrt(op.dot(v, v)))
    vprev = torch.empty_like(v)
    wbuf = torch.empty_like(v)
    alphas, betas = [], []
    e_old = None
    for k in range(max_steps):
        w = op.matvec(v, out=wbuf)
        a = op.dot(v, w)
        b2 = op.axpy_norm(w, v, vprev if k else None, a, betas[-1] if betas else 0.0)
        b = math.sqrt(max(b2, 0.0))
        alphas.append(a)
        e = _lowest_ritz(alphas, betas)
        if e_old is not None and abs(e - e_old) < tol * max(1.0, abs(e)):
            return e, k + 1, np.array(alphas), np.array(betas)
        e_old = e
        if b < 1e-14 * max(1.0, abs(a)) or len(alphas) >= op.D:
            return e, k + 1, np.array(alphas), np.array(betas)
        betas.append(b)
        op.scale(w, 1.0 / b)
        # rotate: w becomes v, v becomes vprev, the old vprev buffer takes the next product
        if w is wbuf:
            vprev, v, wbuf = v, w, vprev
        else:                      # an operator that returned a fresh tensor
            vprev, v = v, w
    return e_old, max_steps, np.array(alphas), np.array(betas)


def cuda_local_apply(basis):
    """local_apply for ShardedOperator backed by the CUDA library (ed_apply_H_rows)."""
    def f(x_full, r0, r1, out=None):
        return basis.apply_H_rows(x_full, r0, r1, y=out)
    f.accepts_out = True
    return f
