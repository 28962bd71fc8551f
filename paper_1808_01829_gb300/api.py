"""Torch-facing API over the C ABI (argument marshalling only).

Every step of the path runs in librhmc.so; this module converts torch tensors
to device pointers, passes the current CUDA stream and turns status codes into
exceptions.  Tensors are complex128 on a CUDA device in the layouts of
include/rhmc.h:

* gauge field U: (Lt, Lz, Ly, Lx, 4, 3, 3)
* a block of n fields on one parity: (V/2, 3, n)
* shifted solutions: (n_shifts, V/2, 3, n)
* force G: (V, 4, 3, 3)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _lib

PRECISION = {"fp64": _lib.RHMC_FP64, "mixed": _lib.RHMC_MIXED_FP32, "fp32": _lib.RHMC_MIXED_FP32,
             "df64": _lib.RHMC_DF64}


@dataclass
class SolveInfo:
    iters: int
    dirac_calls: int
    reliable_updates: int
    refinements: int
    refine_iters: int
    true_rel_resid_max: float
    phase1_rel_resid_max: float
    per_shift_resid: list
    phase1_ms: float = 0.0
    refine_ms: float = 0.0


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _check_field(t: torch.Tensor, name: str, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex128:
        raise ValueError(f"{name} must be complex128, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _doubles(xs):
    arr = (ctypes.c_double * len(xs))(*[float(x) for x in xs])
    return arr


class RhmcContext:
    """One lattice on one GPU (rhmc_create / rhmc_destroy)."""

    def __init__(self, dims: Sequence[int], mass: float, bc_t: int = -1, device: int = 0):
        self.lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the RHMC library has no CPU path")
        self.dims = tuple(int(d) for d in dims)
        self.mass = float(mass)
        self.bc_t = int(bc_t)
        self.device = torch.device("cuda", device)
        lat = _lib.Lattice((ctypes.c_int * 4)(*self.dims), self.mass, self.bc_t)
        h = ctypes.c_void_p()
        _lib.check(self.lib.rhmc_create(ctypes.byref(h), ctypes.byref(lat), int(device)), "rhmc_create")
        self._h = h
        V = 1
        for d in self.dims:
            V *= d
        self.V = V
        self.Vh = V // 2
        self.U = None

    def close(self):
        if getattr(self, "_h", None):
            self.lib.rhmc_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def field_shape(self, n: int):
        return (self.Vh, 3, n)

    # -- rhmc_set_gauge
    def set_gauge(self, U: torch.Tensor):
        lx, ly, lz, lt = self.dims
        _check_field(U, "U", (lt, lz, ly, lx, 4, 3, 3))
        _lib.check(self.lib.rhmc_set_gauge(self._h, _ptr(U), _stream(U)), "rhmc_set_gauge")
        self.U = U

    def workspace_bytes(self, n: int, nshift: int, precision: str = "mixed") -> int:
        return int(self.lib.rhmc_workspace_bytes(self._h, n, nshift, PRECISION[precision]))

    # -- rhmc_apply_mdagm_mrhs
    def apply_mdagm_mrhs(self, X: torch.Tensor, sigma: float = 0.0, precision: str = "fp64", out=None):
        n = X.shape[-1]
        _check_field(X, "X", self.field_shape(n))
        Y = torch.empty_like(X) if out is None else out
        _lib.check(self.lib.rhmc_apply_mdagm_mrhs(self._h, _ptr(X), _ptr(Y), n, float(sigma), PRECISION[precision],
                                                  _stream(X)), "rhmc_apply_mdagm_mrhs")
        return Y

    # -- rhmc_hop
    def hop(self, X: torch.Tensor, out_parity: int, precision: str = "fp64"):
        n = X.shape[-1]
        _check_field(X, "X", self.field_shape(n))
        Y = torch.empty_like(X)
        _lib.check(self.lib.rhmc_hop(self._h, _ptr(X), _ptr(Y), n, int(out_parity), PRECISION[precision],
                                     _stream(X)), "rhmc_hop")
        return Y

    def _info(self, info: _lib.Info, buf, ns, n):
        return SolveInfo(info.iters, info.dirac_calls, info.reliable_updates, info.refinements, info.refine_iters,
                         info.true_rel_resid_max, info.phase1_rel_resid_max,
                         [list(buf[q * n:(q + 1) * n]) for q in range(ns)], info.phase1_ms, info.refine_ms)

    # -- per-context launch settings (rhmc_ctx_tune_set / rhmc_ctx_tune_get)
    def tune_set(self, key: int, value: int):
        _lib.check(self.lib.rhmc_ctx_tune_set(self._h, int(key), int(value)), "rhmc_ctx_tune_set")

    def tune_get(self, key: int) -> int:
        return int(self.lib.rhmc_ctx_tune_get(self._h, int(key)))

    # -- rhmc_block_multishift_cg
    def block_multishift_cg(self, B: torch.Tensor, shifts: Sequence[float], tol: float, max_iter: int = 0,
                            precision: str = "mixed", out=None, workspace: Optional[torch.Tensor] = None,
                            allow_not_converged: bool = False):
        n = B.shape[-1]
        _check_field(B, "B", self.field_shape(n))
        ns = len(shifts)
        X = torch.empty((ns,) + tuple(B.shape), dtype=B.dtype, device=B.device) if out is None else out
        buf = (ctypes.c_double * (ns * n))()
        info = _lib.Info()
        info.per_shift_resid = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None
        rc = self.lib.rhmc_block_multishift_cg(self._h, _ptr(B), n, ns, _doubles(shifts), _ptr(X), float(tol),
                                               int(max_iter), PRECISION[precision], ws, ctypes.byref(info),
                                               _stream(B))
        _lib.check(rc, "rhmc_block_multishift_cg", allow=(2,) if allow_not_converged else ())
        return X, self._info(info, buf, ns, n)

    # -- rhmc_multishift_cg_pervector (FP64 per-vector SCG baseline)
    def multishift_cg_pervector(self, B: torch.Tensor, shifts: Sequence[float], tol: float, max_iter: int = 0,
                                out=None):
        n = B.shape[-1]
        _check_field(B, "B", self.field_shape(n))
        ns = len(shifts)
        X = torch.empty((ns,) + tuple(B.shape), dtype=B.dtype, device=B.device) if out is None else out
        info = _lib.Info()
        rc = self.lib.rhmc_multishift_cg_pervector(self._h, _ptr(B), n, ns, _doubles(shifts), _ptr(X), float(tol),
                                                   int(max_iter), None, ctypes.byref(info), _stream(B))
        _lib.check(rc, "rhmc_multishift_cg_pervector")
        return X, SolveInfo(info.iters, info.dirac_calls, 0, 0, 0, -1.0, -1.0, [])

    # -- rhmc_rational_solve (heatbath / action: R(A) Phi without per-shift solutions)
    def rational_solve(self, Phi: torch.Tensor, alpha0: float, alpha: Sequence[float], beta: Sequence[float],
                       tol: float, max_iter: int = 0, out=None, workspace: Optional[torch.Tensor] = None,
                       allow_not_converged: bool = False):
        n = Phi.shape[-1]
        _check_field(Phi, "Phi", self.field_shape(n))
        ns = len(beta)
        if len(alpha) != ns:
            raise ValueError("alpha and beta must have the same length")
        Y = torch.empty_like(Phi) if out is None else out
        buf = (ctypes.c_double * (ns * n))()
        info = _lib.Info()
        info.per_shift_resid = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None
        rc = self.lib.rhmc_rational_solve(self._h, _ptr(Phi), n, float(alpha0), _doubles(alpha), _doubles(beta), ns,
                                          float(tol), int(max_iter), _ptr(Y), ws, ctypes.byref(info), _stream(Phi))
        _lib.check(rc, "rhmc_rational_solve", allow=(2,) if allow_not_converged else ())
        return Y, self._info(info, buf, ns, n)

    # -- rhmc_force
    def force(self, Phi: torch.Tensor, alpha0: float, alpha: Sequence[float], beta: Sequence[float], tol: float,
              precision: str = "mixed", X: Optional[torch.Tensor] = None, max_iter: int = 0, out=None,
              workspace: Optional[torch.Tensor] = None):
        n = Phi.shape[-1]
        _check_field(Phi, "Phi", self.field_shape(n))
        ns = len(beta)
        if len(alpha) != ns:
            raise ValueError("alpha and beta must have the same length")
        if X is not None:
            _check_field(X, "X", (ns,) + tuple(Phi.shape))
        G = torch.empty((self.V, 4, 3, 3), dtype=torch.complex128, device=Phi.device) if out is None else out
        S = ctypes.c_double(0.0)
        buf = (ctypes.c_double * (ns * n))()
        info = _lib.Info()
        info.per_shift_resid = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None
        rc = self.lib.rhmc_force(self._h, _ptr(Phi), n, float(alpha0), _doubles(alpha), _doubles(beta), ns,
                                 float(tol), int(max_iter), PRECISION[precision],
                                 _ptr(X) if X is not None else None, _ptr(G), ctypes.byref(S), ws,
                                 ctypes.byref(info), _stream(Phi))
        _lib.check(rc, "rhmc_force")
        return G, S.value, self._info(info, buf, ns, n)

    # -- rhmc_force_lie (Lie-algebra force F = TA(U G^dagger) and the force norm)
    def force_lie(self, U: torch.Tensor, G: torch.Tensor, out=None, want_F: bool = True):
        """F_mu(x) = TA(U_mu(x) G_mu(x)^dagger) and sum_{x,mu,a} (F^a)^2 / 2 with
        F^a = Re tr(G^dagger T^a U), T^a = i lambda^a / 2.  Returns (F or None, norm2)."""
        for t, name in ((U, "U"), (G, "G")):
            _check_field(t, name, (self.V, 4, 3, 3))
        F = None
        if want_F:
            F = torch.empty_like(G) if out is None else out
            _check_field(F, "F", (self.V, 4, 3, 3))
        nrm = ctypes.c_double(0.0)
        rc = self.lib.rhmc_force_lie(self._h, _ptr(U), _ptr(G), _ptr(F) if F is not None else None,
                                     ctypes.byref(nrm), _stream(G))
        _lib.check(rc, "rhmc_force_lie")
        return F, nrm.value


def block_multishift_cg_batch(items, tol: float, max_iter: int = 0, precision: str = "mixed"):
    """Batched SBCGrQ over independent ensembles (rhmc_block_multishift_cg_batch).

    items: sequence of (RhmcContext, B, shifts).  Returns a list of (X, SolveInfo)
    in the same order.  Every context must have its gauge field set and may
    appear once."""
    n_items = len(items)
    arr = (_lib.BatchItem * n_items)()
    keep, outs = [], []
    for i, (rctx, B, shifts) in enumerate(items):
        n = B.shape[-1]
        _check_field(B, "B", rctx.field_shape(n))
        ns = len(shifts)
        X = torch.empty((ns,) + tuple(B.shape), dtype=B.dtype, device=B.device)
        sh = _doubles(shifts)
        buf = (ctypes.c_double * (ns * n))()
        info = _lib.Info()
        info.per_shift_resid = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
        arr[i] = _lib.BatchItem(rctx._h, B.data_ptr(), n, ns, ctypes.cast(sh, ctypes.POINTER(ctypes.c_double)),
                                X.data_ptr(), None, ctypes.pointer(info), 0)
        keep += [sh, buf, info]
        outs.append((rctx, X, info, buf, ns, n))
    lib = _lib.load()
    rc = lib.rhmc_block_multishift_cg_batch(arr, n_items, float(tol), int(max_iter), PRECISION[precision],
                                            _stream(items[0][1]))
    _lib.check(rc, "rhmc_block_multishift_cg_batch")
    return [(X, rctx._info(info, buf, ns, n)) for (rctx, X, info, buf, ns, n) in outs]
