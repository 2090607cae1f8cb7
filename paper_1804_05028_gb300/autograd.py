"""Differentiable ground-state energy: E0(J) with dE0/dJ_c through the adjoint product.

H(J) = sum_c J_c H_c (Eq. 21 split into coupling classes).  For the normalised ground
state psi of H(J), dE0/dJ_c = <psi|H_c|psi> (Hellmann-Feynman).  The backward pass
recomputes the Lanczos vectors to form psi (a second pass of the same recurrence, no
stored Krylov basis) and evaluates every <psi|H_c|psi> in one class-resolved pass of the
product kernel (ed_expect_classes).
"""
from __future__ import annotations

import torch

__all__ = ["ground_state_energy"]


class _GroundStateEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J, basis, Jz, kw):
        r = basis.lanczos(J=J.tolist(), Jz=Jz, **kw)
        ctx.basis, ctx.Jz, ctx.kw = basis, Jz, kw
        ctx.save_for_backward(J)
        return torch.tensor(r["E0"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad):
        (J,) = ctx.saved_tensors
        B = ctx.basis
        # the ground state in the forward pass's precision: fp64 by default; with fp32
        # vectors (the mixed form) psi is an fp32 vector and <psi|H_c|psi> is summed in
        # double from fp32 products
        mixed = ctx.kw.get("dtype") in (torch.float32, torch.complex64)
        if mixed:
            dt = torch.float32 if B.is_real else torch.complex64
        else:
            dt = torch.float64 if B.is_real else torch.complex128
        psi = torch.empty(B.dim, dtype=dt, device=f"cuda:{B.device}")
        kw = dict(ctx.kw)
        kw["dtype"] = dt
        kw.setdefault("tol_residual", 1e-10)   # dE0/dJ is first order in the state's error
        kw.setdefault("max_steps", 600)
        B.lanczos(J=J.tolist(), Jz=ctx.Jz, psi=psi, **kw)
        dE = torch.as_tensor(B.expect_classes(psi, Jz=ctx.Jz), dtype=torch.float64)
        return grad * dE, None, None, None


def ground_state_energy(basis, J, Jz=None, **lanczos_kw) -> torch.Tensor:
    """E0 as a differentiable function of the per-class exchange J (CPU float64 tensor).

    ``lanczos_kw`` goes to ``Basis.lanczos``; ``dtype=torch.float32`` (or complex64) runs
    both passes in the mixed form, whose gradient carries the fp32 ground state's error
    (first order in it, about 1e-7 relative) instead of fp64's."""
    if not isinstance(J, torch.Tensor):
        J = torch.tensor(J, dtype=torch.float64)
    return _GroundStateEnergy.apply(J, basis, Jz, lanczos_kw)
