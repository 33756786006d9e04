"""The Schwinger-model action S(q) = S_G + phi^dag (D^dag D)^{-1} phi as a
torch.autograd.Function.

forward         per-chain S (Eq. gauge_action + Eq. fer_action): one CG solve
backward        dS/dq = F (Eq. force): the adjoint solve is the force's own
                CG (chi, xi of Eq. chi_xi_vectors), recomputed, not stored
double backward (Hess S) v through ``sm_hvp`` (Eq. CFF and Eq. Z12 with f
                replaced by the incoming cotangent v), again recomputing
                chi and xi

Only q and phi are saved between passes; every solve is redone when needed.
phi is treated as a constant (no gradient).  All arithmetic runs in the CUDA
library; this module only wires the calls into autograd.
"""
from __future__ import annotations

import torch

from .binding import CG, Lattice


def _chain_index(lat: Lattice) -> torch.Tensor:
    idx = getattr(lat, "_chain_index", None)
    if idx is None:
        sizes = torch.as_tensor(lat.L.astype("int64") * lat.T.astype("int64"))
        idx = torch.repeat_interleave(torch.arange(lat.nchains), sizes).to(lat.device)
        lat._chain_index = idx
    return idx


class _Force(torch.autograd.Function):
    """F(q) = dS/dq; its vector-Jacobian product is the Hessian-vector
    product (the Hessian is symmetric)."""

    @staticmethod
    def forward(ctx, q, phi, lat, part, cg):
        ctx.save_for_backward(q, phi)
        ctx.lat, ctx.part, ctx.cg = lat, part, cg
        return lat.force(q, phi, part, cg)

    @staticmethod
    def backward(ctx, gF):
        q, phi = ctx.saved_tensors
        Hv = ctx.lat.hvp(q, phi, gF.contiguous(), ctx.part, ctx.cg)
        return Hv, None, None, None, None


class SchwingerAction(torch.autograd.Function):
    """Per-chain action S of the lattice batch ``lat`` for links q (float64
    (N, 2)) and pseudofermion phi (complex128 (N, 2)).  ``part`` selects
    'gauge', 'fermion' or 'full'."""

    @staticmethod
    def forward(ctx, q, phi, lat, part="full", cg=None):
        cg = cg or CG(tol=1e-12)
        want = {"gauge": ("SG",), "fermion": ("SF",), "full": ("SG", "SF")}[part]
        e = lat.energies(q=q, phi=phi if "SF" in want else None, cg=cg, want=want)
        S = sum(e[k] for k in want)
        ctx.save_for_backward(q, phi)
        ctx.lat, ctx.part, ctx.cg = lat, part, cg
        return S

    @staticmethod
    def backward(ctx, gS):
        q, phi = ctx.saved_tensors
        F = _Force.apply(q, phi, ctx.lat, ctx.part, ctx.cg)
        w = gS[_chain_index(ctx.lat)].unsqueeze(-1)
        return F * w, None, None, None, None


def action(q, phi, lat, part="full", cg=None):
    """S(q) per chain, differentiable twice in q."""
    return SchwingerAction.apply(q, phi, lat, part, cg)
