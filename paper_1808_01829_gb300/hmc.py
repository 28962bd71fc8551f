"""RHMC trajectory over the C ABI (argument marshalling only).

Sec. II sets up the algorithm (momenta, pseudofermion heatbath, molecular
dynamics with the pseudofermion force, accept/reject); Sec. IV gives the run
parameters (Wilson gauge action, two-level OMF2 integrator with lambda = 1/6,
force solves at 1e-7, heatbath and accept/reject solves at 1e-14).  Every step
runs in librhmc.so: rhmc_gauge_action, rhmc_kinetic_energy,
rhmc_momenta_from_normals, rhmc_gauge_momentum, rhmc_momentum_update,
rhmc_link_update, rhmc_md_evolve and rhmc_hmc_trajectory.

Random numbers are inputs: the caller draws the momentum normals p
(float64 (Lt, Lz, Ly, Lx, 4, 8)), the heatbath Gaussians eta (complex128
(V/2, 3, n_pf), density exp(-|eta|^2)) and the accept/reject uniform u.
Fields: U and P complex128 (Lt, Lz, Ly, Lx, 4, 3, 3); G the same shape as U.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from .api import PRECISION, RhmcContext, _check_field, _ptr, _stream


@dataclass
class MdParams:
    """Two-level OMF2 molecular dynamics (rhmc_md_params_t)."""

    beta: float           # Wilson gauge coupling
    tau: float = 1.0      # trajectory length
    n_steps: int = 10     # outer steps (pseudofermion force)
    n_gauge: int = 3      # inner steps per outer drift (gauge force)
    lam: float = 1.0 / 6  # OMF2 parameter
    tol_md: float = 1e-7
    max_iter: int = 0
    precision: str = "mixed"

    def to_c(self) -> _lib.MdParams:
        return _lib.MdParams(float(self.beta), float(self.tau), int(self.n_steps), int(self.n_gauge),
                             float(self.lam), float(self.tol_md), int(self.max_iter), PRECISION[self.precision])


class _Rational:
    """rhmc_rational_t for coefficients with alpha0, alpha, beta (keeps the arrays alive)."""

    def __init__(self, coeffs):
        self.alpha = (ctypes.c_double * len(coeffs.alpha))(*[float(a) for a in coeffs.alpha])
        self.beta = (ctypes.c_double * len(coeffs.beta))(*[float(b) for b in coeffs.beta])
        self.c = _lib.Rational(len(coeffs.beta), float(coeffs.alpha0), self.alpha, self.beta)

    def ref(self):
        return ctypes.byref(self.c)


def _md_dict(m: _lib.MdInfo) -> dict:
    return {"force_evals": m.force_evals, "gauge_force_evals": m.gauge_force_evals,
            "solver_iters": m.solver_iters, "dirac_calls": m.dirac_calls, "max_rel_resid": m.max_rel_resid}


def _link_shape(ctx: RhmcContext):
    lx, ly, lz, lt = ctx.dims
    return (lt, lz, ly, lx, 4, 3, 3)


def gauge_action(ctx: RhmcContext, U: torch.Tensor, beta: float) -> float:
    _check_field(U, "U", _link_shape(ctx))
    S = ctypes.c_double()
    _lib.check(ctx.lib.rhmc_gauge_action(ctx._h, _ptr(U), float(beta), ctypes.byref(S), _stream(U)),
               "rhmc_gauge_action")
    return S.value


def kinetic_energy(ctx: RhmcContext, P: torch.Tensor) -> float:
    _check_field(P, "P", _link_shape(ctx))
    K = ctypes.c_double()
    _lib.check(ctx.lib.rhmc_kinetic_energy(ctx._h, _ptr(P), ctypes.byref(K), _stream(P)), "rhmc_kinetic_energy")
    return K.value


def momenta(ctx: RhmcContext, p: torch.Tensor) -> torch.Tensor:
    lx, ly, lz, lt = ctx.dims
    if p.dtype != torch.float64 or not p.is_cuda or not p.is_contiguous() or tuple(p.shape) != (lt, lz, ly, lx, 4, 8):
        raise ValueError("p must be a contiguous float64 CUDA tensor of shape (Lt, Lz, Ly, Lx, 4, 8)")
    P = torch.empty(_link_shape(ctx), dtype=torch.complex128, device=p.device)
    _lib.check(ctx.lib.rhmc_momenta_from_normals(ctx._h, _ptr(p), _ptr(P), _stream(p)), "rhmc_momenta_from_normals")
    return P


def gauge_kick(ctx: RhmcContext, U: torch.Tensor, P: torch.Tensor, beta: float, eps: float) -> None:
    """P += eps TA(U G_g^dagger) / 2 in place."""
    _check_field(U, "U", _link_shape(ctx))
    _check_field(P, "P", _link_shape(ctx))
    _lib.check(ctx.lib.rhmc_gauge_momentum(ctx._h, _ptr(U), _ptr(P), float(beta), float(eps), _stream(U)),
               "rhmc_gauge_momentum")


def momentum_kick(ctx: RhmcContext, U: torch.Tensor, G: torch.Tensor, P: torch.Tensor, eps: float) -> None:
    """P += eps TA(U G^dagger) / 2 in place."""
    for t, n in ((U, "U"), (P, "P")):
        _check_field(t, n, _link_shape(ctx))
    _check_field(G, "G")
    if G.numel() != U.numel():
        raise ValueError("G must have the link field's size")
    _lib.check(ctx.lib.rhmc_momentum_update(ctx._h, _ptr(U), _ptr(G), _ptr(P), float(eps), _stream(U)),
               "rhmc_momentum_update")


def link_update(ctx: RhmcContext, U: torch.Tensor, P: torch.Tensor, eps: float) -> None:
    """U <- exp(eps P) U in place."""
    _check_field(U, "U", _link_shape(ctx))
    _check_field(P, "P", _link_shape(ctx))
    _lib.check(ctx.lib.rhmc_link_update(ctx._h, _ptr(U), _ptr(P), float(eps), _stream(U)), "rhmc_link_update")


def md_evolve(ctx: RhmcContext, U: torch.Tensor, P: torch.Tensor, Phi, md_coeffs, params: MdParams) -> dict:
    """Molecular dynamics over one trajectory, U and P updated in place; Phi None is pure gauge."""
    _check_field(U, "U", _link_shape(ctx))
    _check_field(P, "P", _link_shape(ctx))
    n_pf = 0
    rat = None
    if Phi is not None:
        n_pf = Phi.shape[-1]
        _check_field(Phi, "Phi", ctx.field_shape(n_pf))
        rat = _Rational(md_coeffs)
    info = _lib.MdInfo()
    prm = params.to_c()
    _lib.check(ctx.lib.rhmc_md_evolve(ctx._h, _ptr(U), _ptr(P), _ptr(Phi) if Phi is not None else None, n_pf,
                                      rat.ref() if rat else None, ctypes.byref(prm), ctypes.byref(info),
                                      _stream(U)), "rhmc_md_evolve")
    return _md_dict(info)


def trajectory(ctx: RhmcContext, U: torch.Tensor, p: torch.Tensor, eta, heatbath, md, action, params: MdParams,
               tol_action: float = 1e-14, u: float = 0.0, want_phi: bool = False) -> dict:
    """One RHMC trajectory with accept/reject (rhmc_hmc_trajectory); U is replaced on accept.

    heatbath, md, action: rational approximations (alpha0, alpha, beta) of
    x^(+n_f/(8 n_pf)), x^(-n_f/(4 n_pf)) (force accuracy) and x^(-n_f/(4 n_pf))
    (accept/reject accuracy).  eta None: pure-gauge HMC."""
    _check_field(U, "U", _link_shape(ctx))
    lx, ly, lz, lt = ctx.dims
    if p.dtype != torch.float64 or not p.is_cuda or not p.is_contiguous() or tuple(p.shape) != (lt, lz, ly, lx, 4, 8):
        raise ValueError("p must be a contiguous float64 CUDA tensor of shape (Lt, Lz, Ly, Lx, 4, 8)")
    n_pf = 0
    rats = [None, None, None]
    phi = None
    if eta is not None:
        n_pf = eta.shape[-1]
        _check_field(eta, "eta", ctx.field_shape(n_pf))
        rats = [_Rational(heatbath), _Rational(md), _Rational(action)]
        if want_phi:
            phi = torch.empty_like(eta)
    info = _lib.HmcInfo()
    prm = params.to_c()
    _lib.check(ctx.lib.rhmc_hmc_trajectory(
        ctx._h, _ptr(U), _ptr(p), _ptr(eta) if eta is not None else None, n_pf,
        *[r.ref() if r else None for r in rats], ctypes.byref(prm), float(tol_action), float(u),
        _ptr(phi) if phi is not None else None, ctypes.byref(info), _stream(U)), "rhmc_hmc_trajectory")
    out = {"H_old": info.H_old, "H_new": info.H_new, "dH": info.dH, "K": tuple(info.K), "S_g": tuple(info.S_g),
           "S_f": tuple(info.S_f), "accepted": bool(info.accepted), "md": _md_dict(info.md)}
    if phi is not None:
        out["Phi"] = phi
    return out
