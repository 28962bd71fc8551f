"""Functional forms of the library's entry points on torch tensors.

    from paper_1808_01829_gb300 import functional as rhmc
    Y = rhmc.apply_mdagm(U, X, mass=0.01)                       # (A + sigma) X, Sec. IV operator
    X, info = rhmc.block_multishift_cg(U, B, shifts, 1e-8, mass=0.01)   # Algorithm 1
    S = rhmc.PseudofermionAction.apply(U, Phi, coeffs, 0.01)    # Eq. (RA) action, Eq. (force) gradient

The lattice extents are read from the link tensor's shape (Lt, Lz, Ly, Lx, 4,
3, 3).  One RhmcContext is kept per (device, extents, mass, boundary
condition); the links are staged into it again whenever a different tensor, or
the same tensor after an in-place change, is passed.  Every call goes through
the C ABI exactly as the RhmcContext methods do (no computation here).
"""
from __future__ import annotations

import weakref
from typing import Optional, Sequence

import torch

from .api import RhmcContext

_contexts: dict = {}


def context_for(U: torch.Tensor, mass: float, bc_t: int = -1) -> RhmcContext:
    """The cached context of U's lattice, with U staged."""
    if U.dim() != 7 or tuple(U.shape[4:]) != (4, 3, 3):
        raise ValueError(f"U must have shape (Lt, Lz, Ly, Lx, 4, 3, 3), got {tuple(U.shape)}")
    lt, lz, ly, lx = (int(d) for d in U.shape[:4])
    dev = U.device.index if U.device.index is not None else 0
    key = (U.device.type, dev, (lx, ly, lz, lt), float(mass), int(bc_t))
    ent = _contexts.get(key)
    if ent is None:
        ent = {"ctx": RhmcContext((lx, ly, lz, lt), mass, bc_t, device=dev), "ref": None, "version": None}
        _contexts[key] = ent
    staged = ent["ref"]() if ent["ref"] is not None else None
    if staged is not U or ent["version"] != U._version:
        ent["ctx"].set_gauge(U.detach().contiguous())
        ent["ref"], ent["version"] = weakref.ref(U), U._version
    return ent["ctx"]


def clear_contexts() -> None:
    """Destroy every cached context."""
    for ent in _contexts.values():
        ent["ctx"].close()
    _contexts.clear()


def apply_mdagm(U: torch.Tensor, X: torch.Tensor, mass: float, sigma: float = 0.0, bc_t: int = -1,
                precision: str = "fp64", out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """(A + sigma) X, A = 4m^2 - D_eo D_oe on the even sites (rhmc_apply_mdagm_mrhs)."""
    return context_for(U, mass, bc_t).apply_mdagm_mrhs(X, sigma, precision, out=out)


def block_multishift_cg(U: torch.Tensor, B: torch.Tensor, shifts: Sequence[float], tol: float, mass: float,
                        bc_t: int = -1, precision: str = "mixed", max_iter: int = 0):
    """X^(s) = (A + sigma_s)^-1 B for every shift, with the block solver SBCGrQ
    (rhmc_block_multishift_cg); returns (X [n_shifts][V/2][3][n], SolveInfo)."""
    return context_for(U, mass, bc_t).block_multishift_cg(B, shifts, tol, max_iter=max_iter, precision=precision)


def force(U: torch.Tensor, Phi: torch.Tensor, coeffs, tol: float, mass: float, bc_t: int = -1,
          precision: str = "mixed", max_iter: int = 0):
    """Action and force of Eqs. (RA), (force) with the rational approximation
    `coeffs` (remez.RationalApprox): returns (G [V][4][3][3], S, SolveInfo)."""
    return context_for(U, mass, bc_t).force(Phi, coeffs.alpha0, coeffs.alpha, coeffs.beta, tol,
                                            precision=precision, max_iter=max_iter)


class PseudofermionAction:
    """S_f(U, Phi) as a differentiable function of U and Phi (torch.autograd)."""

    @staticmethod
    def apply(U: torch.Tensor, Phi: torch.Tensor, coeffs, mass: float, tol: float = 1e-8, bc_t: int = -1,
              precision: str = "mixed", store="auto", max_iter: int = 0) -> torch.Tensor:
        from .action import pseudofermion_action

        ctx = context_for(U, mass, bc_t)
        return pseudofermion_action(U, Phi, ctx, coeffs, tol=tol, precision=precision, store=store,
                                    max_iter=max_iter)
