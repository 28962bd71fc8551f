"""Pins of the trajectory oracle (oracle/trajectory.py): Wilson action, its link
derivative, the link exponential, and the two-level OMF2 molecular dynamics of
Sec. IV.

* Wilson action of an abelian field with a constant plaquette in one plane
  against its closed form beta V (2/3)(1 - cos a);
* gauge invariance of the action under a random gauge transformation;
* the derivative G_g against central differences of S_g (random complex
  directions);
* the link exponential against scipy's expm, unitarity and unit determinant;
* the momentum force conserves H along the flow: dH/dtau = 0 to rounding for the
  exact equations of motion (directional derivative of H);
* OMF2: energy violation Delta H falls as dtau^2 (ratio 4 per halving, within
  25 %), and the trajectory is reversible (momenta flipped, run again: back to
  the start to 1e-11), with pure gauge at 4^4 and with two pseudofermions at 2^4.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import trajectory as tr
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx


def _abelian(dims, k):
    lx, ly, lz, lt = dims
    a = 2 * np.pi * k / ly
    U = syn.unit_links(dims).copy()
    y = np.arange(ly)
    ph = np.exp(1j * a * y)
    U[:, :, :, :, 0, 0, 0] = ph[None, None, :, None]
    U[:, :, :, :, 0, 1, 1] = np.conj(ph)[None, None, :, None]
    return U, a


@pytest.mark.parametrize("dims,k", [((4, 4, 4, 4), 1), ((2, 6, 4, 2), 2)])
def test_gauge_action_closed_form(dims, k):
    U, a = _abelian(dims, k)
    beta = 5.12
    V = np.prod(dims)
    assert abs(tr.gauge_action(U, beta) - beta * V * (2.0 / 3.0) * (1 - np.cos(a))) <= 1e-10 * beta * V
    assert abs(tr.gauge_action(syn.unit_links(dims), beta)) <= 1e-12


def test_gauge_action_gauge_invariant():
    dims = (4, 4, 4, 4)
    U = syn.random_links(dims, 0.5, 41)
    g = syn.random_gauge_transform(dims, 42)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ tr._dag(tr._shift(g, mu, 1))
    assert abs(tr.gauge_action(Ug, 5.12) - tr.gauge_action(U, 5.12)) <= 1e-10 * abs(tr.gauge_action(U, 5.12))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 2, 4)])
def test_gauge_derivative_central_differences(dims):
    beta = 5.12
    U = syn.random_links(dims, 0.5, 43)
    G = tr.gauge_G(U, beta)
    rng = np.random.default_rng(44)
    h = 1e-5
    for _ in range(4):
        W = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
        fd = (tr.gauge_action(U + h * W, beta) - tr.gauge_action(U - h * W, beta)) / (2 * h)
        an = float(np.sum(np.conj(G) * W).real)
        assert abs(fd - an) <= 1e-7 * abs(an) + 1e-9, (fd, an)


def test_link_exponential():
    P = tr.momenta((2, 2, 2, 2), 45)
    E = tr.expm_ah(0.7 * P)
    flat_p, flat_e = P.reshape(-1, 3, 3), E.reshape(-1, 3, 3)
    for k in range(0, flat_p.shape[0], 7):
        assert np.abs(flat_e[k] - scipy.linalg.expm(0.7 * flat_p[k])).max() <= 1e-13
    eye = np.eye(3)
    assert np.abs(E @ tr._dag(E) - eye).max() <= 1e-13
    assert np.abs(np.linalg.det(E) - 1).max() <= 1e-13
    # the momenta are traceless anti-Hermitian, K = sum (p^a)^2 / 2 > 0
    assert np.abs(P + tr._dag(P)).max() <= 1e-15 and np.abs(np.trace(P, axis1=-2, axis2=-1)).max() <= 1e-15
    assert tr.kinetic(P) > 0


def test_momentum_force_conserves_H_along_the_flow():
    """dH/dtau = dK/dtau + dS/dtau = -2 sum tr(P dP) + Re sum tr(G^dagger P U) = 0 with
    dP = TA(U G^dagger) / 2: both terms are computed independently and cancel."""
    dims, beta = (4, 4, 2, 2), 5.12
    U = syn.random_links(dims, 0.5, 46)
    P = tr.momenta(dims, 47)
    G = tr.gauge_G(U, beta)
    dP = tr.momentum_force(U, G)
    dK = float(-2 * np.sum(np.trace(P @ dP, axis1=-2, axis2=-1).real))
    dS = float(np.sum(np.conj(G) * (P @ U)).real)
    assert abs(dK + dS) <= 1e-11 * abs(dS)
    # dS/dtau along U(tau) = exp(tau P) U by central differences of S_g
    h = 1e-5
    fd = (tr.gauge_action(tr.drift(U, P, h), beta) - tr.gauge_action(tr.drift(U, P, -h), beta)) / (2 * h)
    assert abs(fd - dS) <= 1e-7 * abs(dS)


def _dH(dims, mass, U, P, Phi, beta, ra_md, ra_act, tau, n, n_gauge, tol):
    H0 = tr.hamiltonian(dims, mass, U, P, Phi, beta, ra_act, tol)
    U1, P1 = tr.trajectory(dims, mass, U, P, Phi, beta, ra_md, tau, n, n_gauge, 1.0 / 6.0, tol)
    H1 = tr.hamiltonian(dims, mass, U1, P1, Phi, beta, ra_act, tol)
    return H1 - H0, U1, P1


def test_omf2_pure_gauge_dH_scaling_and_reversibility():
    dims, beta, tau = (4, 4, 4, 4), 5.12, 0.5
    U = syn.random_links(dims, 0.3, 48)
    P = tr.momenta(dims, 49)
    dH = [abs(_dH(dims, 0.0, U, P, None, beta, None, None, tau, n, 1, 0.0)[0]) for n in (4, 8, 16)]
    assert 3.0 <= dH[0] / dH[1] <= 5.0 and 3.0 <= dH[1] / dH[2] <= 5.0, dH
    U1, P1 = tr.trajectory(dims, 0.0, U, P, None, beta, None, tau, 4, 2, 1.0 / 6.0, 0.0)
    U2, P2 = tr.trajectory(dims, 0.0, U1, -P1, None, beta, None, tau, 4, 2, 1.0 / 6.0, 0.0)
    assert np.abs(U2 - U).max() <= 1e-11 and np.abs(P2 + P).max() <= 1e-11


def test_omf2_with_pseudofermions_dH_scaling_and_reversibility():
    dims, mass, n_pf, beta, tau = (2, 2, 2, 4), 0.2, 2, 5.12, 0.3
    ra_md = rational_approx(-1.0 / (4 * n_pf), 0.1, 64.0, 8)
    U = syn.random_links(dims, 0.3, 50)
    P = tr.momenta(dims, 51)
    Phi = syn.gaussian_pseudofermions(dims, n_pf, 52)
    dH = [abs(_dH(dims, mass, U, P, Phi, beta, ra_md, ra_md, tau, n, 2, 1e-13)[0]) for n in (2, 4, 8)]
    assert 3.0 <= dH[0] / dH[1] <= 5.0 and 3.0 <= dH[1] / dH[2] <= 5.0, dH
    U1, P1 = tr.trajectory(dims, mass, U, P, Phi, beta, ra_md, tau, 2, 2, 1.0 / 6.0, 1e-13)
    U2, P2 = tr.trajectory(dims, mass, U1, -P1, Phi, beta, ra_md, tau, 2, 2, 1.0 / 6.0, 1e-13)
    assert np.abs(U2 - U).max() <= 1e-11 and np.abs(P2 + P).max() <= 1e-11


def test_heatbath_inverts_the_action():
    """Phi = R_hb(A) eta with R_hb ~ x^(1/16) and S_f = Phi^dagger R_act(A) Phi with
    R_act ~ x^(-1/8): R_hb R_act R_hb ~ 1 on the spectrum, so S_f = |eta|^2 up to the
    rationals' relative errors (Sec. II heatbath, Sec. IV accuracies)."""
    dims, mass, n_pf = (4, 4, 4, 4), 0.1, 2
    ra_hb = rational_approx(1.0 / 16, 1e-3, 64.0, 8)
    ra_act = rational_approx(-1.0 / 8, 1e-3, 64.0, 8)
    U = syn.random_links(dims, 0.5, 53)
    eta = syn.gaussian_pseudofermions(dims, n_pf, 54)
    Phi = tr.heatbath(dims, mass, U, eta, ra_hb, 1e-13)
    Sf = tr.fermion_action(dims, mass, U, Phi, ra_act, 1e-13)
    e2 = float(np.sum(np.abs(eta) ** 2))
    assert abs(Sf - e2) <= (ra_act.error + 2 * ra_hb.error) * e2 + 1e-10 * e2, (Sf, e2)
    # a wrong sign of the heatbath power would be far off
    assert abs(tr.fermion_action(dims, mass, U, eta, ra_act, 1e-13) - e2) > 1e-3 * e2


def test_hmc_trajectory_record():
    """The accept/reject step: H from its parts, acceptance when u < exp(-dH), and the
    links returned are the trial links on accept and the old ones on reject."""
    dims, beta = (2, 2, 2, 4), 5.12
    U = syn.random_links(dims, 0.3, 55)
    p = syn.momentum_normals(dims, 56)
    P = tr.momenta_from_normals(p)
    args = (dims, 0.0, U, p, None, beta, None, None, None, 0.5, 2, 1, 1.0 / 6.0, 0.0, 0.0)
    Uacc, rec = tr.hmc_trajectory(*args, 0.0)
    assert abs(rec["H_old"] - (tr.kinetic(P) + tr.gauge_action(U, beta))) <= 1e-12 * rec["H_old"]
    assert rec["accepted"] and Uacc is rec["U1"]
    Urej, rec2 = tr.hmc_trajectory(*args, 1.0)
    assert rec2["dH"] == rec["dH"]
    assert rec2["accepted"] == (rec["dH"] <= 0) and (Urej is U) == (rec["dH"] > 0)
