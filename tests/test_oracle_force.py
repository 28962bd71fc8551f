"""Pins of the oracle's pseudofermion action and force (Eqs. (RA), (force)).

* central finite differences of the action, computed by the independent dense
  numpy implementation (dense LU solves), against Re <G, V> for random
  unconstrained complex link directions V and for Lie-algebra directions;
* the action against the dense eigendecomposition form phi^dagger R(A) phi;
* gauge covariance G[U^g, g Phi] = g(x) G[U, Phi] g(x+mu)^dagger;
* linearity in the rational coefficients alpha_s;
* the sampled-link evaluation agrees with the full one;
* the Lie-algebra components F^a = Re tr(G^dagger T^a U) are the derivatives of
  the action along U -> exp(w T^a) U, link by link (finite differences), and the
  projection TA(U G^dagger) carries the same information: F = -2 sum_a F^a T^a,
  sum_a (F^a)^2 / 2 = |F|_F^2 / 4.
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1808_01829_gb300 import synthetic as syn

ALPHA0 = 0.7
ALPHA = [0.02, 0.11, 0.3, 0.9]
BETA = [0.004, 0.05, 0.6, 7.0]


def _solve(dims, mass, U, Phi):
    X, _, rc = oracle.sbcgrq(dims, mass, U, Phi, BETA, tol=1e-13, max_iter=5000)
    assert rc == 0
    return X


@pytest.mark.parametrize("dims,n,bc", [((2, 2, 2, 2), 2, -1), ((4, 4, 4, 4), 2, -1), ((2, 4, 2, 4), 3, 1)])
def test_force_matches_finite_differences(dims, n, bc):
    mass = 0.1
    U = syn.random_links(dims, 0.5, 1020)
    Phi = syn.gaussian_pseudofermions(dims, n, 2020)
    X, _, rc = oracle.sbcgrq(dims, mass, U, Phi, BETA, tol=1e-13, max_iter=5000, bc_t=bc)
    assert rc == 0
    G = oracle.force(dims, U, X, ALPHA, bc_t=bc)
    rng = np.random.default_rng(21)
    for _ in range(4):
        V = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
        an = np.vdot(G.reshape(-1), V.reshape(-1)).real
        fd = dense.fd_directional(dims, mass, U, Phi, ALPHA0, ALPHA, BETA, V, h=1e-5, bc_t=bc)
        fd2 = dense.fd_directional(dims, mass, U, Phi, ALPHA0, ALPHA, BETA, V, h=5e-6, bc_t=bc)
        assert abs(fd - an) <= 1e-6 * abs(an)
        assert abs(fd2 - an) <= 1e-6 * abs(an)


def test_force_lie_direction():
    """U -> exp(h T) U with T anti-Hermitian traceless: dS/dh = Re tr(G^dagger T U) summed."""
    dims, mass = (2, 2, 2, 2), 0.1
    U = syn.random_links(dims, 0.5, 1021)
    Phi = syn.gaussian_pseudofermions(dims, 2, 2021)
    G = oracle.force(dims, U, _solve(dims, mass, U, Phi), ALPHA).reshape(U.shape)
    rng = np.random.default_rng(3)
    H = np.einsum("...a,aij->...ij", rng.standard_normal(U.shape[:-2] + (8,)), syn.gell_mann()) / 2
    T = 1j * H
    h = 1e-5

    def S_at(hh):
        w, v = np.linalg.eigh(H)
        E = np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * hh * w), v.conj())
        return dense.action(dims, mass, E @ U, Phi, ALPHA0, ALPHA, BETA)

    fd = (S_at(h) - S_at(-h)) / (2 * h)
    an = np.sum(np.conj(G) * (T @ U)).real
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_action_matches_dense_rational_form():
    dims, mass = (4, 4, 4, 4), 0.1
    U = syn.random_links(dims, 0.5, 1022)
    Phi = syn.gaussian_pseudofermions(dims, 3, 2022)
    S = oracle.action(ALPHA0, ALPHA, Phi, _solve(dims, mass, U, Phi))
    Sd = dense.action_rational(dims, mass, U, Phi, ALPHA0, ALPHA, BETA)
    assert abs(S - Sd) <= 1e-11 * abs(Sd)


def test_force_gauge_covariance():
    dims, mass = (4, 4, 4, 4), 0.1
    U = syn.random_links(dims, 0.5, 1023)
    Phi = syn.gaussian_pseudofermions(dims, 2, 2023)
    g = syn.random_gauge_transform(dims)
    from test_oracle_operator import _apply_g, _gauge_transform

    Ug = _gauge_transform(dims, U, g)
    G = oracle.force(dims, U, _solve(dims, mass, U, Phi), ALPHA).reshape(U.shape)
    Gg = oracle.force(dims, Ug, _solve(dims, mass, Ug, _apply_g(dims, g, Phi, 0)), ALPHA).reshape(U.shape)
    for mu, ax in ((0, 3), (1, 2), (2, 1), (3, 0)):
        gp = np.roll(g, -1, axis=ax)
        expect = g @ G[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
        np.testing.assert_allclose(Gg[..., mu, :, :], expect, atol=1e-9 * np.abs(G).max())


def test_force_linear_in_alpha():
    dims, mass = (4, 4, 4, 4), 0.05
    U = syn.random_links(dims, 0.5, 1024)
    Phi = syn.gaussian_pseudofermions(dims, 2, 2024)
    X = _solve(dims, mass, U, Phi)
    G = oracle.force(dims, U, X, ALPHA)
    parts = sum(oracle.force(dims, U, X[s:s + 1], [ALPHA[s]]) for s in range(len(ALPHA)))
    np.testing.assert_allclose(G, parts, atol=1e-13 * np.abs(G).max())


def test_force_at_matches_full():
    dims = (4, 2, 4, 6)
    U = syn.random_links(dims, 0.5, 1025)
    X = np.stack([syn.gaussian_pseudofermions(dims, 3, 2025 + s) for s in range(2)])
    G = oracle.force(dims, U, X, [0.4, 1.3])
    links = [(0, 0), (1, 3), (37, 2), (191, 1), (190, 3)]
    Gs = oracle.force_at(dims, U, X, [0.4, 1.3], links)
    for k, (lex, mu) in enumerate(links):
        np.testing.assert_allclose(Gs[k], G[lex, mu], atol=1e-13)


def test_lie_components_are_single_link_derivatives():
    """F^a at one link and generator = (S(exp(wT^a)U) - S(exp(-wT^a)U)) / 2w with only
    that link rotated (dense solves), for several links and all eight generators."""
    dims, mass = (2, 2, 2, 2), 0.1
    U = syn.random_links(dims, 0.5, 1031)
    Phi = syn.gaussian_pseudofermions(dims, 2, 2031)
    G = oracle.force(dims, U, _solve(dims, mass, U, Phi), ALPHA).reshape(U.shape)
    Fa = dense.lie_components(U, G)
    lam = dense.gell_mann_matrices()
    h = 1e-5
    for (t, z, y, x, mu) in [(0, 0, 0, 0, 0), (1, 0, 1, 0, 3), (0, 1, 1, 1, 2)]:
        for a in range(8):
            w, v = np.linalg.eigh(lam[a] / 2)  # exp(i h lambda/2) = v exp(i h w) v^dagger

            def S_at(hh):
                Up = U.copy()
                E = (v * np.exp(1j * hh * w)) @ v.conj().T
                Up[t, z, y, x, mu] = E @ U[t, z, y, x, mu]
                return dense.action(dims, mass, Up, Phi, ALPHA0, ALPHA, BETA)

            fd = (S_at(h) - S_at(-h)) / (2 * h)
            an = Fa[t, z, y, x, mu, a]
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (t, z, y, x, mu, a, fd, an)


def test_ta_projection_matches_components():
    """TA(U G^dagger) = -2 sum_a F^a T^a, traceless and anti-Hermitian, and the norm
    from the eight components equals |TA(U G^dagger)|_F^2 / 4 (random links, random G)."""
    rng = np.random.default_rng(33)
    U = syn.random_links((2, 2, 2, 4), 0.7, 1032)
    G = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    F = dense.force_lie(U, G)
    Fa = dense.lie_components(U, G)
    T = 0.5j * dense.gell_mann_matrices()
    assert np.allclose(F, -2 * np.einsum("...a,aij->...ij", Fa, T), atol=1e-13, rtol=0)
    assert np.allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-13)
    assert np.allclose(F, -np.swapaxes(F.conj(), -1, -2), atol=1e-13)
    assert abs(dense.force_norm2(U, G) - 0.25 * np.sum(np.abs(F) ** 2)) <= 1e-12 * dense.force_norm2(U, G)
    # the Gell-Mann matrices: Hermitian, traceless, tr(l^a l^b) = 2 delta_ab, closed under [.,.] with f^123 = 1
    lam = dense.gell_mann_matrices()
    assert np.allclose(np.einsum("aij,bji->ab", lam, lam), 2 * np.eye(8), atol=1e-14)
    assert np.allclose(lam, np.swapaxes(lam.conj(), -1, -2))
    assert np.allclose(np.trace(lam, axis1=-2, axis2=-1), 0)
    assert np.allclose(lam[0] @ lam[1] - lam[1] @ lam[0], 2j * lam[2])
