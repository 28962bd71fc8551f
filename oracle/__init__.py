"""CPU oracle for the block multishift RHMC path (arXiv:1808.01829).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the benchmark's CPU-baseline leg; never by the product package.

``oracle.cpp`` is a plain FP64 C++ implementation (OpenMP over sites) of the
even-odd staggered operator, thin QR, SBCGrQ (Algorithm 1), scalar multishift
CG and the action/force of Eqs. (RA) and (force).  ``dense.py`` is a second,
independent numpy implementation used only on tiny lattices (dense matrices,
brute-force solves, finite differences) to pin the C++ one.

Every function here takes and returns numpy complex128 arrays in the layouts of
``paper_1808_01829_gb300.synthetic``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "invalid argument", 2: "not converged", 3: "breakdown"}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into a shared library (gcc, -O2, OpenMP); returns its path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
            lib.orc_hop.argtypes = [P, I, P, P, P, I, I]
            lib.orc_apply_A.argtypes = [P, D, I, P, P, P, I, D]
            lib.orc_apply_A_at.argtypes = [P, D, I, P, P, P, I, D, P, L]
            lib.orc_thin_qr.argtypes = [P, P, P, L, I]
            lib.orc_sbcgrq.argtypes = [P, D, I, P, P, I, I, P, P, D, D, I, I, P, P]
            lib.orc_scg.argtypes = [P, D, I, P, P, I, P, P, D, I, I, P]
            lib.orc_action.argtypes = [L, I, I, D, P, P, P]
            lib.orc_action.restype = D
            lib.orc_force.argtypes = [P, I, P, P, I, I, P, P]
            lib.orc_force_at.argtypes = [P, I, P, P, I, I, P, P, L, P]
            lib.orc_set_threads.argtypes = [I]
            lib.orc_max_threads.restype = I
            _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _check(rc, what):
    if rc == 1:
        raise ValueError(f"oracle {what}: invalid argument")
    return rc


def set_threads(t: int) -> None:
    _L().orc_set_threads(int(t))


def max_threads() -> int:
    return int(_L().orc_max_threads())


def hop(dims, U, psi, out_parity: int, bc_t: int = -1):
    """D psi on sites of parity out_parity; psi [Vh][3][n] lives on the other parity."""
    U, psi = _c128(U), _c128(psi)
    n = psi.shape[-1]
    out = np.empty_like(psi)
    _check(_L().orc_hop(_p(_dims(dims)), bc_t, _p(U), _p(psi), _p(out), n, out_parity), "hop")
    return out


def apply_A(dims, mass, U, X, sigma: float = 0.0, bc_t: int = -1):
    """(A + sigma) X, A = 4 m^2 - D_eo D_oe on even sites."""
    U, X = _c128(U), _c128(X)
    Y = np.empty_like(X)
    _check(_L().orc_apply_A(_p(_dims(dims)), mass, bc_t, _p(U), _p(X), _p(Y), X.shape[-1], sigma), "apply_A")
    return Y


def apply_A_at(dims, mass, U, X, sites, sigma: float = 0.0, bc_t: int = -1):
    """(A + sigma) X at the listed even-site ranks only; returns [len(sites)][3][n]."""
    U, X = _c128(U), _c128(X)
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    n = X.shape[-1]
    Y = np.empty((len(sites), 3, n), dtype=np.complex128)
    _check(_L().orc_apply_A_at(_p(_dims(dims)), mass, bc_t, _p(U), _p(X), _p(Y), n, sigma, _p(sites), len(sites)),
           "apply_A_at")
    return Y


def thin_qr(B):
    """Thin QR of a (rows, n) complex block; R upper triangular, positive real diagonal."""
    B = _c128(B)
    rows, n = B.shape
    Q = np.empty_like(B)
    R = np.empty((n, n), dtype=np.complex128)
    rc = _L().orc_thin_qr(_p(B), _p(Q), _p(R), rows, n)
    if rc:
        raise np.linalg.LinAlgError("thin_qr: rank deficient block")
    return Q, R


def sbcgrq(dims, mass, U, B, shifts, tol=1e-10, max_iter=10000, fixed_iters=0, tol_shift=0.0, bc_t=-1,
           want_history=False):
    """SBCGrQ (Algorithm 1).  Returns (X [nshift][Vh][3][n], iters, status[, history])."""
    U, B = _c128(U), _c128(B)
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    n = B.shape[-1]
    ns = len(shifts)
    X = np.empty((ns,) + B.shape, dtype=np.complex128)
    it = ctypes.c_int(0)
    kmax = fixed_iters if fixed_iters > 0 else max_iter
    hist = np.zeros(kmax + 1)
    rc = _L().orc_sbcgrq(_p(_dims(dims)), mass, bc_t, _p(U), _p(B), n, ns, _p(shifts), _p(X), tol, tol_shift,
                         max_iter, fixed_iters, ctypes.byref(it), _p(hist))
    _check(rc, "sbcgrq")
    if want_history:
        return X, it.value, rc, hist[: it.value + 1]
    return X, it.value, rc


def scg(dims, mass, U, b, shifts, tol=1e-10, max_iter=10000, fixed_iters=0, bc_t=-1):
    """Scalar multishift CG on one right-hand side b [Vh][3]; returns (x [nshift][Vh][3], iters, status)."""
    U, b = _c128(U), _c128(b)
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    ns = len(shifts)
    x = np.empty((ns,) + b.shape, dtype=np.complex128)
    it = ctypes.c_int(0)
    rc = _L().orc_scg(_p(_dims(dims)), mass, bc_t, _p(U), _p(b), ns, _p(shifts), _p(x), tol, max_iter,
                      fixed_iters, ctypes.byref(it))
    _check(rc, "scg")
    return x, it.value, rc


def action(alpha0, alpha, Phi, X):
    """S = sum_i [alpha_0 |phi_i|^2 + sum_s alpha_s phi_i^dagger X^(s) e_i]  (Eq. (RA))."""
    Phi, X = _c128(Phi), _c128(X)
    alpha = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    vh, _, n = Phi.shape
    return float(_L().orc_action(vh, n, len(alpha), float(alpha0), _p(alpha), _p(Phi), _p(X)))


def force(dims, U, X, alpha, bc_t=-1):
    """G = dS/dRe U + i dS/dIm U from the shifted solutions X [nshift][Vh][3][n]; [V][4][3][3]."""
    U, X = _c128(U), _c128(X)
    alpha = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    ns, vh, _, n = X.shape
    G = np.empty((2 * vh, 4, 3, 3), dtype=np.complex128)
    _check(_L().orc_force(_p(_dims(dims)), bc_t, _p(U), _p(X), n, ns, _p(alpha), _p(G)), "force")
    return G


def force_at(dims, U, X, alpha, links, bc_t=-1):
    """G at listed links (rows (lex, mu)); returns [len(links)][3][3]."""
    U, X = _c128(U), _c128(X)
    alpha = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    links = np.ascontiguousarray(np.asarray(links, dtype=np.int64).reshape(-1, 2))
    ns, vh, _, n = X.shape
    G = np.empty((len(links), 3, 3), dtype=np.complex128)
    _check(_L().orc_force_at(_p(_dims(dims)), bc_t, _p(U), _p(X), n, ns, _p(alpha), _p(links), len(links), _p(G)),
           "force_at")
    return G


def solve_and_force(dims, mass, U, Phi, alpha0, alpha, beta, tol=1e-12, max_iter=20000, bc_t=-1):
    """Full oracle force evaluation: SBCGrQ for all shifts, then S and G."""
    X, iters, rc = sbcgrq(dims, mass, U, Phi, beta, tol=tol, max_iter=max_iter, bc_t=bc_t)
    if rc != 0:
        raise RuntimeError(f"oracle sbcgrq: {STATUS.get(rc, rc)} after {iters} iterations")
    S = action(alpha0, alpha, Phi, X)
    G = force(dims, U, X, alpha, bc_t=bc_t)
    return S, G, X, iters
