"""Oracle of the RHMC trajectory around the pseudofermion force (Sec. II set-up,
Sec. IV run parameters): Wilson gauge action and its link derivative, the
exponential link update, the kinetic energy of the momenta, the pseudofermion
action, and the two-level second-order Omelyan (OMF2) integrator with the gauge
force on the inner level.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product package.

Conventions (shared with ``oracle.cpp`` and the library):

* gauge field U[t][z][y][x][mu][3][3] complex128, periodic in every direction;
  the antiperiodic temporal boundary belongs to the fermion operator only;
* Wilson action (Sec. IV: Wilson gauge action, beta = 5.12 in the paper's runs):
  S_g = beta sum_{x, mu<nu} (1 - Re tr Pi_{mu nu}(x) / 3),
  Pi_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger;
* derivatives in the convention of the pseudofermion force,
  G = dS/dRe U + i dS/dIm U, so that dS = Re tr(G^dagger dU); for S_g, with the
  staple sum V_mu(x) = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger
  + U_nu(x+mu-nu)^dagger U_mu(x-nu)^dagger U_nu(x-nu)] (every plaquette through the
  link is Re tr(U_mu(x) V)), G_g = -(beta / 3) V^dagger;
* momenta P_mu(x) = sum_a p^a T^a, T^a = i lambda^a / 2 (traceless anti-Hermitian),
  kinetic energy K = sum_{x,mu} sum_a (p^a)^2 / 2 = -sum tr(P^2); links evolve as
  dU/dtau = P U, so p^a is conjugate to the coordinate w of U -> exp(w T^a) U and
  dP/dtau = -sum_a (dS/dw^a) T^a = TA(U G^dagger) / 2 (dS/dw^a = tr(TA(U G^dagger) T^a),
  TA(M) = (M - M^dagger)/2 - tr(M - M^dagger)/6);
* H = K + S_g + S_f with S_f = sum_i phi_i^dagger R(A) phi_i (Eq. (RA));
* OMF2 step of length e for force F and drift D (Omelyan's second-order
  scheme, lambda = 1/6 in the paper's comparison runs):
  P += lambda e F; D(e/2); P += (1 - 2 lambda) e F; D(e/2); P += lambda e F;
  the two-level integrator (Sexton-Weingarten) applies it with the
  pseudofermion force on the outer level, whose drift D(e/2) is itself an OMF2
  integration of length e/2 with the gauge force in n_gauge steps.
"""
from __future__ import annotations

import numpy as np

import oracle

_AX = {0: 3, 1: 2, 2: 1, 3: 0}  # direction mu -> array axis of [t][z][y][x]


def _shift(A, mu, d):
    """Field at x + d mu (periodic)."""
    return np.roll(A, -d, axis=_AX[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def gauge_action(U, beta):
    """S_g = beta sum_{x, mu<nu} (1 - Re tr Pi_{mu nu}(x) / 3)."""
    S = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Um, Un = U[..., mu, :, :], U[..., nu, :, :]
            Pi = Um @ _shift(Un, mu, 1) @ _dag(_shift(Um, nu, 1)) @ _dag(Un)
            S += np.sum(1.0 - np.trace(Pi, axis1=-2, axis2=-1).real / 3.0)
    return float(beta * S)


def staples(U):
    """V_mu(x) such that the plaquettes through U_mu(x) sum to Re tr(U_mu(x) V_mu(x))."""
    V = np.zeros_like(U)
    for mu in range(4):
        Um = U[..., mu, :, :]
        for nu in range(4):
            if nu == mu:
                continue
            Un = U[..., nu, :, :]
            up = _shift(Un, mu, 1) @ _dag(_shift(Um, nu, 1)) @ _dag(Un)
            Un_m = _shift(Un, nu, -1)  # U_nu(x - nu)
            dn = _dag(_shift(Un_m, mu, 1)) @ _dag(_shift(Um, nu, -1)) @ Un_m
            V[..., mu, :, :] += up + dn
    return V


def gauge_G(U, beta):
    """G_g = dS_g/dRe U + i dS_g/dIm U = -(beta / 3) V^dagger."""
    return -(beta / 3.0) * _dag(staples(U))


def ta(M):
    """Traceless anti-Hermitian part."""
    A = 0.5 * (M - _dag(M))
    tr = np.trace(A, axis1=-2, axis2=-1) / 3.0
    return A - tr[..., None, None] * np.eye(3)


def momentum_force(U, G):
    """dP/dtau = TA(U G^dagger) / 2 for a total derivative G."""
    return 0.5 * ta(U @ _dag(G))


def kinetic(P):
    """K = -sum tr(P^2) = sum_a (p^a)^2 / 2."""
    return float(-np.sum(np.trace(P @ P, axis1=-2, axis2=-1).real))


def expm_ah(X):
    """exp(X) for anti-Hermitian X (stacked): X = i H with H Hermitian, so
    exp(X) = Q diag(exp(i h)) Q^dagger from the eigendecomposition H = Q diag(h) Q^dagger."""
    h, Q = np.linalg.eigh(-1j * X)
    return (Q * np.exp(1j * h)[..., None, :]) @ _dag(Q)


def drift(U, P, eps):
    """U <- exp(eps P) U, link by link."""
    return expm_ah(eps * P) @ U


def momenta_from_normals(p):
    """P = sum_a p^a T^a, T^a = i lambda^a / 2, for normals p of shape [...][8]."""
    from paper_1808_01829_gb300 import synthetic as syn

    T = 0.5j * syn.gell_mann()
    return np.einsum("...a,aij->...ij", p, T)


def momenta(dims, seed):
    """p^a ~ N(0, 1), P = sum_a p^a T^a, layout [t][z][y][x][mu][3][3]."""
    from paper_1808_01829_gb300 import synthetic as syn

    return momenta_from_normals(syn.momentum_normals(dims, seed))


def _flat(U):
    return np.ascontiguousarray(U.reshape(-1, 4, 3, 3))


def fermion_G(dims, mass, U, Phi, ra, tol, bc_t=-1):
    X, _, rc = oracle.sbcgrq(dims, mass, _flat(U), Phi, ra.beta, tol=tol, max_iter=50000, bc_t=bc_t)
    if rc != 0:
        raise RuntimeError(f"oracle sbcgrq: status {rc}")
    return oracle.force(dims, _flat(U), X, ra.alpha, bc_t=bc_t).reshape(U.shape)


def fermion_action(dims, mass, U, Phi, ra, tol, bc_t=-1):
    X, _, rc = oracle.sbcgrq(dims, mass, _flat(U), Phi, ra.beta, tol=tol, max_iter=50000, bc_t=bc_t)
    if rc != 0:
        raise RuntimeError(f"oracle sbcgrq: status {rc}")
    return oracle.action(ra.alpha0, ra.alpha, Phi, X)


def heatbath(dims, mass, U, eta, ra, tol, bc_t=-1):
    """Phi = R(A) eta = alpha0 eta + sum_s alpha_s (A + beta_s)^-1 eta, R the heatbath
    rational (x^(+n_f/(8 n_pf)) so that Phi^dagger A^(-n_f/(4 n_pf)) Phi = |eta|^2)."""
    X, _, rc = oracle.sbcgrq(dims, mass, _flat(U), eta, ra.beta, tol=tol, max_iter=50000, bc_t=bc_t)
    if rc != 0:
        raise RuntimeError(f"oracle sbcgrq: status {rc}")
    Phi = ra.alpha0 * eta
    for s, a in enumerate(ra.alpha):
        Phi = Phi + a * X[s]
    return Phi


def hamiltonian(dims, mass, U, P, Phi, beta, ra_action, tol, bc_t=-1):
    H = kinetic(P) + gauge_action(U, beta)
    if Phi is not None:
        H += fermion_action(dims, mass, U, Phi, ra_action, tol, bc_t)
    return H


def omf2(U, P, force, drift_fn, eps, lam):
    """One OMF2 step of length eps: P += lam eps F; D(eps/2); P += (1-2lam) eps F; D(eps/2); P += lam eps F."""
    P = P + lam * eps * force(U)
    U, P = drift_fn(U, P, 0.5 * eps)
    P = P + (1.0 - 2.0 * lam) * eps * force(U)
    U, P = drift_fn(U, P, 0.5 * eps)
    P = P + lam * eps * force(U)
    return U, P


def trajectory(dims, mass, U, P, Phi, beta, ra_md, tau, n_steps, n_gauge, lam, tol_md, bc_t=-1):
    """Two-level OMF2 molecular dynamics from (U, P) over length tau: n_steps outer
    steps with the pseudofermion force (none when Phi is None), each drift an OMF2
    integration with the gauge force in n_gauge steps.  Returns (U, P)."""

    def gforce(Uc):
        return momentum_force(Uc, gauge_G(Uc, beta))

    def fforce(Uc):
        if Phi is None:
            return np.zeros_like(Uc)
        return momentum_force(Uc, fermion_G(dims, mass, Uc, Phi, ra_md, tol_md, bc_t))

    def gauge_drift(Uc, Pc, length):
        e = length / n_gauge
        for _ in range(n_gauge):
            Uc, Pc = omf2(Uc, Pc, gforce, lambda a, b, t: (drift(a, b, t), b), e, lam)
        return Uc, Pc

    eps = tau / n_steps
    for _ in range(n_steps):
        U, P = omf2(U, P, fforce, gauge_drift, eps, lam)
    return U, P


def hmc_trajectory(dims, mass, U, p, eta, beta, ra_hb, ra_md, ra_act, tau, n_steps, n_gauge, lam, tol_md, tol_action,
                   u, bc_t=-1):
    """One RHMC trajectory (Sec. II): momenta from the normals p, heatbath Phi from
    eta (None: pure gauge), H at the start, molecular dynamics, H at the end, and
    acceptance when u < exp(-dH).  Returns (links after the step, record)."""
    P = momenta_from_normals(p)
    Phi = None if eta is None else heatbath(dims, mass, U, eta, ra_hb, tol_action, bc_t)
    H0 = hamiltonian(dims, mass, U, P, Phi, beta, ra_act, tol_action, bc_t)
    U1, P1 = trajectory(dims, mass, U, P, Phi, beta, ra_md, tau, n_steps, n_gauge, lam, tol_md, bc_t)
    H1 = hamiltonian(dims, mass, U1, P1, Phi, beta, ra_act, tol_action, bc_t)
    dH = H1 - H0
    acc = bool(dH <= 0 or u < np.exp(-dH))
    return (U1 if acc else U), {"H_old": H0, "H_new": H1, "dH": dH, "accepted": acc, "Phi": Phi, "U1": U1, "P1": P1}
