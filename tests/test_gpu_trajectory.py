"""GPU parity of the RHMC trajectory pieces against the trajectory oracle (Sec. II
set-up, Sec. IV run parameters: Wilson gauge action, two-level OMF2 integrator,
heatbath and accept/reject solves).

Tolerances (FP64 on both sides):
* gauge action, kinetic energy: 1e-12 relative (sums of ~1e3-1e6 terms, each
  exact to a few ulp);
* momenta from normals: 1e-15 absolute (one product per entry);
* kicks: 1e-13 of the largest momentum entry (a product of up to four SU(3)
  matrices per staple);
* link exponential: 1e-13, also past the scaling threshold (squarings double the
  rounding each time; the cases need at most 5);
* molecular dynamics: pure gauge 1e-11 (rounding of ~100 kernel steps, the GPU
  merging consecutive kicks); with pseudofermions the force solves stop at
  1e-12 on both sides, a relative force error of at most tol / lambda_min(A)
  ~ 1e-12 / 4m^2, so links and momenta agree to 1e-8;
* Hamiltonian: H to 1e-11 relative, dH to 1e-7 absolute (solves at 1e-13).
"""
import numpy as np
import pytest

from gpu_util import make_ctx, need_gpu, to_gpu
from oracle import trajectory as tr
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx

pytestmark = pytest.mark.gpu

BETA = 5.12


def _hmc():
    from paper_1808_01829_gb300 import hmc

    return hmc


def _rats(n_pf):
    """Heatbath x^(1/(8 n_pf)) and action / MD x^(-1/(4 n_pf)), n_f = 1, on [1e-3, 64]."""
    return (rational_approx(1.0 / (8 * n_pf), 1e-3, 64.0, 8), rational_approx(-1.0 / (4 * n_pf), 1e-3, 64.0, 8))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2)])
def test_actions_and_momenta(dims):
    need_gpu()
    hmc = _hmc()
    U = syn.random_links(dims, 0.5, 300)
    ctx = make_ctx(dims, 0.1, U)
    Ug = to_gpu(U)
    Sg = hmc.gauge_action(ctx, Ug, BETA)
    So = tr.gauge_action(U, BETA)
    assert abs(Sg - So) <= 1e-12 * abs(So)
    assert abs(hmc.gauge_action(ctx, to_gpu(syn.unit_links(dims)), BETA)) <= 1e-12 * np.prod(dims)
    p = syn.momentum_normals(dims, 301)
    P = hmc.momenta(ctx, to_gpu(p))
    Po = tr.momenta_from_normals(p)
    assert np.abs(P.cpu().numpy() - Po).max() <= 1e-15 * np.abs(Po).max() * 4
    K = hmc.kinetic_energy(ctx, P)
    assert abs(K - tr.kinetic(Po)) <= 1e-12 * tr.kinetic(Po)
    # K = sum (p^a)^2 / 2 (generators normalised tr(T^a T^b) = -delta/2)
    assert abs(K - 0.5 * np.sum(p ** 2)) <= 1e-12 * K
    ctx.close()


def test_gauge_action_abelian_closed_form():
    """U_x = diag(e^{i a y}, e^{-i a y}, 1): the (x, y) plaquettes have Re tr = 1 + 2 cos a."""
    need_gpu()
    hmc = _hmc()
    dims = (4, 6, 2, 4)
    lx, ly, lz, lt = dims
    a = 2 * np.pi / ly
    U = syn.unit_links(dims).copy()
    ph = np.exp(1j * a * np.arange(ly))
    U[:, :, :, :, 0, 0, 0] = ph[None, None, :, None]
    U[:, :, :, :, 0, 1, 1] = np.conj(ph)[None, None, :, None]
    ctx = make_ctx(dims, 0.1, U)
    S = hmc.gauge_action(ctx, to_gpu(U), BETA)
    V = np.prod(dims)
    assert abs(S - BETA * V * (2.0 / 3.0) * (1 - np.cos(a))) <= 1e-12 * BETA * V
    ctx.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 2)])
def test_kicks(dims):
    need_gpu()
    hmc = _hmc()
    U = syn.random_links(dims, 0.5, 302)
    P0 = tr.momenta(dims, 303)
    ctx = make_ctx(dims, 0.1, U)
    Ug, eps = to_gpu(U), 0.37
    P = to_gpu(P0)
    hmc.gauge_kick(ctx, Ug, P, BETA, eps)
    ref = P0 + eps * tr.momentum_force(U, tr.gauge_G(U, BETA))
    assert np.abs(P.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    rng = np.random.default_rng(304)
    G = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    P = to_gpu(P0)
    hmc.momentum_kick(ctx, Ug, to_gpu(G.reshape(-1, 4, 3, 3)), P, -eps)
    ref = P0 - eps * tr.momentum_force(U, G)
    assert np.abs(P.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    # the kicks keep P traceless anti-Hermitian
    Pn = P.cpu().numpy()
    assert np.abs(Pn + tr._dag(Pn)).max() <= 1e-14 * np.abs(Pn).max()
    assert np.abs(np.trace(Pn, axis1=-2, axis2=-1)).max() <= 1e-14 * np.abs(Pn).max()
    ctx.close()


@pytest.mark.parametrize("eps", [0.0, 0.05, 0.7, -4.0])
def test_link_update(eps):
    """exp(eps P) U against the oracle's eigendecomposition exponential; |eps P|_F
    spans no scaling (0.05) to five squarings (4.0)."""
    need_gpu()
    hmc = _hmc()
    dims = (4, 2, 4, 2)
    U = syn.random_links(dims, 0.5, 305)
    P = tr.momenta(dims, 306)
    ctx = make_ctx(dims, 0.1, U)
    Ug = to_gpu(U)
    hmc.link_update(ctx, Ug, to_gpu(P), eps)
    got = Ug.cpu().numpy()
    assert np.abs(got - tr.drift(U, P, eps)).max() <= 1e-13
    eye = np.eye(3)
    assert np.abs(got @ tr._dag(got) - eye).max() <= 1e-13
    assert np.abs(np.linalg.det(got) - 1).max() <= 1e-13
    ctx.close()


def test_md_pure_gauge_matches_oracle_and_reverses():
    need_gpu()
    hmc = _hmc()
    dims, tau = (4, 4, 4, 4), 0.5
    U = syn.random_links(dims, 0.3, 307)
    P0 = tr.momenta(dims, 308)
    ctx = make_ctx(dims, 0.1, U)
    prm = hmc.MdParams(beta=BETA, tau=tau, n_steps=4, n_gauge=2, lam=1.0 / 6)
    Ug, Pg = to_gpu(U), to_gpu(P0)
    info = hmc.md_evolve(ctx, Ug, Pg, None, None, prm)
    Uo, Po = tr.trajectory(dims, 0.0, U, P0, None, BETA, None, tau, 4, 2, 1.0 / 6, 0.0)
    assert np.abs(Ug.cpu().numpy() - Uo).max() <= 1e-11
    assert np.abs(Pg.cpu().numpy() - Po).max() <= 1e-11
    assert info["force_evals"] == 0 and info["gauge_force_evals"] == 2 * 4 * (2 * 2 + 1)
    Pg.neg_()
    hmc.md_evolve(ctx, Ug, Pg, None, None, prm)
    assert np.abs(Ug.cpu().numpy() - U).max() <= 1e-11
    assert np.abs(Pg.cpu().numpy() + P0).max() <= 1e-11
    ctx.close()


def test_md_pure_gauge_dH_scaling():
    """OMF2 is second order: dH falls by 4 per halving of the step (25 %)."""
    need_gpu()
    hmc = _hmc()
    dims, tau = (8, 8, 8, 8), 0.5
    U = syn.random_links(dims, 0.3, 309)
    p = to_gpu(syn.momentum_normals(dims, 310))
    ctx = make_ctx(dims, 0.1, U)
    dH = []
    for n in (4, 8, 16):
        Ug = to_gpu(U)
        P = hmc.momenta(ctx, p)
        H0 = hmc.kinetic_energy(ctx, P) + hmc.gauge_action(ctx, Ug, BETA)
        hmc.md_evolve(ctx, Ug, P, None, None, hmc.MdParams(beta=BETA, tau=tau, n_steps=n, n_gauge=1))
        dH.append(abs(hmc.kinetic_energy(ctx, P) + hmc.gauge_action(ctx, Ug, BETA) - H0))
    assert 3.0 <= dH[0] / dH[1] <= 5.0 and 3.0 <= dH[1] / dH[2] <= 5.0, dH
    ctx.close()


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-8), ("mixed", 1e-10, 1e-6)])
def test_md_with_pseudofermions_matches_oracle(precision, tol, bound):
    need_gpu()
    hmc = _hmc()
    dims, mass, n_pf, tau = (4, 4, 4, 4), 0.1, 2, 0.2
    _, ra = _rats(n_pf)
    U = syn.random_links(dims, 0.5, 311)
    P0 = tr.momenta(dims, 312)
    Phi = syn.gaussian_pseudofermions(dims, n_pf, 313)
    ctx = make_ctx(dims, mass, U)
    prm = hmc.MdParams(beta=BETA, tau=tau, n_steps=2, n_gauge=2, tol_md=tol, precision=precision)
    Ug, Pg = to_gpu(U), to_gpu(P0)
    info = hmc.md_evolve(ctx, Ug, Pg, to_gpu(Phi), ra, prm)
    Uo, Po = tr.trajectory(dims, mass, U, P0, Phi, BETA, ra, tau, 2, 2, 1.0 / 6, 1e-12)
    assert info["force_evals"] == 2 * 2 + 1
    assert info["max_rel_resid"] <= tol
    assert np.abs(Ug.cpu().numpy() - Uo).max() <= bound
    assert np.abs(Pg.cpu().numpy() - Po).max() <= bound * np.abs(Po).max()
    ctx.close()


def test_md_with_pseudofermions_reverses():
    need_gpu()
    hmc = _hmc()
    dims, mass, n_pf, tau = (4, 4, 4, 4), 0.1, 2, 0.3
    _, ra = _rats(n_pf)
    U = syn.random_links(dims, 0.5, 314)
    P0 = tr.momenta(dims, 315)
    Phi = to_gpu(syn.gaussian_pseudofermions(dims, n_pf, 316))
    ctx = make_ctx(dims, mass, U)
    prm = hmc.MdParams(beta=BETA, tau=tau, n_steps=3, n_gauge=2, tol_md=1e-13, precision="fp64")
    Ug, Pg = to_gpu(U), to_gpu(P0)
    hmc.md_evolve(ctx, Ug, Pg, Phi, ra, prm)
    Pg.neg_()
    hmc.md_evolve(ctx, Ug, Pg, Phi, ra, prm)
    assert np.abs(Ug.cpu().numpy() - U).max() <= 1e-10
    assert np.abs(Pg.cpu().numpy() + P0).max() <= 1e-10 * np.abs(P0).max()
    ctx.close()


@pytest.mark.parametrize("u", [0.0, 0.999999])
def test_hmc_trajectory_matches_oracle(u):
    """Whole trajectory: momenta, heatbath, H, molecular dynamics, H, accept/reject."""
    need_gpu()
    hmc = _hmc()
    dims, mass, n_pf, tau = (4, 4, 4, 4), 0.1, 2, 0.3
    ra_hb, ra = _rats(n_pf)
    U = syn.random_links(dims, 0.5, 317)
    p = syn.momentum_normals(dims, 318)
    eta = syn.gaussian_pseudofermions(dims, n_pf, 319)
    ctx = make_ctx(dims, mass, U)
    prm = hmc.MdParams(beta=BETA, tau=tau, n_steps=2, n_gauge=2, tol_md=1e-12, precision="fp64")
    Ug = to_gpu(U)
    rec = hmc.trajectory(ctx, Ug, to_gpu(p), to_gpu(eta), ra_hb, ra, ra, prm, tol_action=1e-13, u=u, want_phi=True)
    Uo, ro = tr.hmc_trajectory(dims, mass, U, p, eta, BETA, ra_hb, ra, ra, tau, 2, 2, 1.0 / 6, 1e-12, 1e-13, u)
    assert np.abs(rec["Phi"].cpu().numpy() - ro["Phi"]).max() <= 1e-11 * np.abs(ro["Phi"]).max()
    assert abs(rec["H_old"] - ro["H_old"]) <= 1e-11 * abs(ro["H_old"])
    assert abs(rec["H_new"] - ro["H_new"]) <= 1e-11 * abs(ro["H_new"]) + 1e-7
    assert abs(rec["dH"] - ro["dH"]) <= 1e-7
    # S_f at the start is |eta|^2 up to the rationals' errors
    e2 = float(np.sum(np.abs(eta) ** 2))
    assert abs(rec["S_f"][0] - e2) <= (ra.error + 2 * ra_hb.error) * e2 + 1e-10 * e2
    if abs(np.exp(-ro["dH"]) - u) > 1e-6:
        assert rec["accepted"] == ro["accepted"]
        assert np.abs(Ug.cpu().numpy() - Uo).max() <= 1e-8
    ctx.close()


def test_pure_gauge_hmc_full_size():
    """24^4 (the force workload's lattice), pure gauge: unitary links after the
    trajectory, the action against the oracle on the new links, and dH falling
    by 4 per halving of the step (dH is extensive: ~60 at this volume and step)."""
    need_gpu()
    hmc = _hmc()
    dims = (24, 24, 24, 24)
    U = syn.random_links(dims, 0.3, syn.seed_gauge(3))
    ctx = make_ctx(dims, 0.01, U)
    p = to_gpu(syn.momentum_normals(dims, 320))
    dH = []
    for n in (4, 8):
        Ug = to_gpu(U)
        rec = hmc.trajectory(ctx, Ug, p, None, None, None, None, hmc.MdParams(beta=BETA, tau=0.5, n_steps=n,
                                                                           n_gauge=2), u=0.0)
        assert rec["accepted"] and abs(rec["dH"]) <= 1e-3 * rec["H_old"]
        dH.append(abs(rec["dH"]))
    assert 3.0 <= dH[0] / dH[1] <= 5.0, dH
    U1 = Ug.cpu().numpy()
    rng = np.random.default_rng(321)
    idx = rng.integers(0, U1.reshape(-1, 3, 3).shape[0], 512)
    W = U1.reshape(-1, 3, 3)[idx]
    assert np.abs(W @ tr._dag(W) - np.eye(3)).max() <= 1e-13
    assert abs(rec["S_g"][1] - tr.gauge_action(U1, BETA)) <= 1e-12 * rec["S_g"][1]
    ctx.close()


def test_hmc_trajectory_mixed_md_close_to_oracle():
    """The bench's setting: force solves in mixed precision at 1e-9 (the MD is then an
    approximation of the oracle's 1e-12 one at the level of the solves' tolerance) with the
    heatbath and both actions in FP64 at 1e-13: H at the start agrees to 1e-11, dH to a
    bound set by the force errors (1e-9 / 4m^2 relative over tau = 0.3)."""
    need_gpu()
    hmc = _hmc()
    dims, mass, n_pf, tau = (4, 4, 4, 4), 0.1, 2, 0.3
    ra_hb, ra = _rats(n_pf)
    U = syn.random_links(dims, 0.5, 322)
    p = syn.momentum_normals(dims, 323)
    eta = syn.gaussian_pseudofermions(dims, n_pf, 324)
    ctx = make_ctx(dims, mass, U)
    prm = hmc.MdParams(beta=BETA, tau=tau, n_steps=2, n_gauge=2, tol_md=1e-9, precision="mixed")
    rec = hmc.trajectory(ctx, to_gpu(U), to_gpu(p), to_gpu(eta), ra_hb, ra, ra, prm, tol_action=1e-13, u=0.0)
    _, ro = tr.hmc_trajectory(dims, mass, U, p, eta, BETA, ra_hb, ra, ra, tau, 2, 2, 1.0 / 6, 1e-12, 1e-13, 0.0)
    assert abs(rec["H_old"] - ro["H_old"]) <= 1e-11 * abs(ro["H_old"])
    assert abs(rec["dH"] - ro["dH"]) <= 1e-4 * (1.0 + abs(ro["dH"]))
    assert rec["md"]["max_rel_resid"] <= 1e-9 and rec["md"]["force_evals"] == 5
    ctx.close()
