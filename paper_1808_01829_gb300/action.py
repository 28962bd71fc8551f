"""Pseudofermion action as a torch.autograd.Function (argument marshalling only).

    S_f(U, Phi) = sum_i phi_i^dagger R(A[U]) phi_i,
    R(x) = alpha_0 + sum_s alpha_s / (x + beta_s)          (Eqs. (RA), Sec. II)

forward  : stages U, solves (A + beta_s) X^(s) = Phi for all shifts and columns
           (rhmc_block_multishift_cg), S from rhmc_force with G = NULL;
backward : grad_U   = grad_S * G, G = dS/dRe U + i dS/dIm U from rhmc_force
           (the hand-written derivative of Eq. (force));
           grad_Phi = grad_S * 2 R(A) Phi (rhmc_rational_apply).
PyTorch's complex-gradient convention for a real loss L is dL/dRe z + i dL/dIm z,
the same convention as G.

The shifted solutions are kept from forward to backward when they fit the
memory budget (store="auto": at most half of the free device memory), otherwise
backward solves again.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import _lib
from .api import PRECISION, RhmcContext, _check_field, _doubles, _ptr, _stream


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U: torch.Tensor, Phi: torch.Tensor, rctx: RhmcContext, alpha0: float, alpha, beta, tol: float,
                precision: str = "mixed", store="auto", max_iter: int = 0):
        rctx.set_gauge(U.detach().contiguous())
        n = Phi.shape[-1]
        ns = len(beta)
        field_bytes = Phi.numel() * 16
        if store == "auto":
            free, _ = torch.cuda.mem_get_info(Phi.device)
            store = ns * field_bytes <= free // 2
        Phi_c = Phi.detach().contiguous()
        X = None
        if store:
            X, info = rctx.block_multishift_cg(Phi_c, beta, tol, max_iter=max_iter, precision=precision)
        S = ctypes.c_double(0.0)
        lib = rctx.lib
        rc = lib.rhmc_force(rctx._h, _ptr(Phi_c), n, float(alpha0), _doubles(alpha), _doubles(beta), ns, float(tol),
                            int(max_iter), PRECISION[precision], _ptr(X) if X is not None else None, None,
                            ctypes.byref(S), None, None, _stream(Phi_c))
        _lib.check(rc, "rhmc_force (action)")
        ctx.rctx = rctx
        ctx.coeffs = (float(alpha0), list(alpha), list(beta), float(tol), precision, int(max_iter))
        ctx.U_shape = U.shape
        ctx.save_for_backward(Phi_c, X if X is not None else torch.empty(0, device=Phi.device))
        ctx.stored = X is not None
        return torch.tensor(S.value, dtype=torch.float64, device=Phi.device)

    @staticmethod
    def backward(ctx, grad_S):
        Phi, X = ctx.saved_tensors
        rctx: RhmcContext = ctx.rctx
        alpha0, alpha, beta, tol, precision, max_iter = ctx.coeffs
        g = grad_S.to(torch.float64)
        grad_U = grad_Phi = None
        if not ctx.stored and (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]):
            X, _ = rctx.block_multishift_cg(Phi, beta, tol, max_iter=max_iter, precision=precision)
        if ctx.needs_input_grad[0]:
            G, _, _ = rctx.force(Phi, alpha0, alpha, beta, tol, precision=precision, X=X, max_iter=max_iter)
            grad_U = (G * g).reshape(ctx.U_shape)
        if ctx.needs_input_grad[1]:
            RPhi = torch.empty_like(Phi)
            _lib.check(rctx.lib.rhmc_rational_apply(rctx._h, _ptr(Phi), Phi.shape[-1], alpha0, _doubles(alpha),
                                                    len(alpha), _ptr(X), _ptr(RPhi), _stream(Phi)),
                       "rhmc_rational_apply")
            grad_Phi = 2.0 * g * RPhi
        return grad_U, grad_Phi, None, None, None, None, None, None, None, None


def pseudofermion_action(U: torch.Tensor, Phi: torch.Tensor, rctx: RhmcContext, coeffs, tol: float = 1e-8,
                         precision: str = "mixed", store="auto", max_iter: int = 0) -> torch.Tensor:
    """S_f(U, Phi) with the rational approximation `coeffs` (remez.RationalApprox)."""
    _check_field(U, "U")
    _check_field(Phi, "Phi")
    return PseudofermionAction.apply(U, Phi, rctx, coeffs.alpha0, coeffs.alpha, coeffs.beta, tol, precision, store,
                                     max_iter)
