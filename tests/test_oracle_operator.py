"""Pins of the oracle's even-odd staggered operator (Sec. IV) against what the
mathematics fixes: closed-form free-field spectrum, an independent dense
construction (even-even block of M^dagger M), hermiticity, D_oe = -D_eo^dagger,
positivity bounds and gauge covariance."""
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1808_01829_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "free_field_spectrum.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                lx, ly, lz, lt, bc, m, lam, mult = line.split()
                rows.append(((int(lx), int(ly), int(lz), int(lt)), int(bc), float(m), float(lam), int(mult)))
    return rows


def _dense_from_oracle(dims, mass, U, bc_t=-1):
    """Dense matrix of the oracle's A, column by column."""
    vh = syn.volume(dims) // 2
    N = 3 * vh
    cols = []
    for c0 in range(0, N, 48):
        E = np.eye(N, dtype=np.complex128)[:, c0:c0 + 48].reshape(vh, 3, -1)
        cols.append(oracle.apply_A(dims, mass, U, E, bc_t=bc_t).reshape(N, -1))
    return np.concatenate(cols, axis=1)


@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 2), -1), ((2, 2, 2, 2), 1), ((4, 4, 4, 4), 1)])
def test_free_field_golden_hand_values(dims, bc):
    rows = [r for r in _golden_rows() if r[0] == dims and r[1] == bc]
    assert rows
    for mass in sorted({r[2] for r in rows}):
        w = np.linalg.eigvalsh(_dense_from_oracle(dims, mass, syn.unit_links(dims), bc))
        expect = np.concatenate([np.full(mult, lam) for (_, _, m, lam, mult) in rows if m == mass])
        np.testing.assert_allclose(np.sort(w), np.sort(expect), atol=1e-12)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 2, 6)])
@pytest.mark.parametrize("bc", [-1, 1])
def test_free_field_closed_form(dims, bc):
    mass = 0.07
    w = np.linalg.eigvalsh(_dense_from_oracle(dims, mass, syn.unit_links(dims), bc))
    np.testing.assert_allclose(np.sort(w), dense.free_field_spectrum(dims, mass, bc), atol=1e-12)


def test_free_field_plane_wave_large():
    """On 8^4 an even-projected plane wave is an eigenvector with the closed-form eigenvalue."""
    dims, mass = (8, 8, 8, 8), 0.05
    lex = dense.parity_lex(dims, 0)
    x = lex % 8
    y = (lex // 8) % 8
    z = (lex // 64) % 8
    t = lex // 512
    p = np.array([2 * np.pi * 1 / 8, 2 * np.pi * 3 / 8, 0.0, (2 * 2 + 1) * np.pi / 8])
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    X = np.zeros((len(lex), 3, 1), dtype=np.complex128)
    X[:, 1, 0] = phase
    Y = oracle.apply_A(dims, mass, syn.unit_links(dims), X)
    lam = 4 * mass ** 2 + 4 * np.sum(np.sin(p) ** 2)
    np.testing.assert_allclose(Y, lam * X, atol=1e-12)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 4, 2)])
@pytest.mark.parametrize("bc", [-1, 1])
def test_matches_dense_mdagm_even_block(dims, bc):
    """Oracle's two-hop A equals the even-even block of (2m + D)^dagger (2m + D) built independently."""
    mass = 0.1
    U = syn.random_links(dims, 0.5, 1001)
    A_or = _dense_from_oracle(dims, mass, U, bc)
    A_dn = dense.dense_A(dims, mass, U, bc)
    assert np.abs(A_or - A_dn).max() <= 1e-13 * np.abs(A_dn).max()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (4, 6, 2, 8)])
def test_hermitian_and_doe_is_minus_deo_dagger(dims):
    U = syn.random_links(dims, 0.5, 1002)
    n = 3
    X = syn.gaussian_pseudofermions(dims, n, 2001)
    Z = syn.gaussian_pseudofermions(dims, n, 2002)
    AX = oracle.apply_A(dims, 0.05, U, X)
    AZ = oracle.apply_A(dims, 0.05, U, Z)
    lhs = np.einsum("abi,abi->i", Z.conj(), AX)
    rhs = np.einsum("abi,abi->i", AZ.conj(), X)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)
    # <y_o, D_oe x_e> = -<D_eo y_o, x_e>  (Z plays an odd-site field)
    Doe_x = oracle.hop(dims, U, X, 1)
    Deo_z = oracle.hop(dims, U, Z, 0)
    l2 = np.einsum("abi,abi->i", Z.conj(), Doe_x)
    r2 = -np.einsum("abi,abi->i", Deo_z.conj(), X)
    np.testing.assert_allclose(l2, r2, rtol=1e-13)


def test_positivity_bounds_dense():
    dims, mass = (4, 4, 4, 4), 0.02
    U = syn.random_links(dims, 0.5, 1003)
    w = np.linalg.eigvalsh(_dense_from_oracle(dims, mass, U))
    assert w.min() >= 4 * mass ** 2 - 1e-12
    assert w.max() <= 4 * mass ** 2 + 64 + 1e-12


def test_positivity_power_iteration_8x4():
    """lambda_max of A on 8^4 stays below 4m^2 + 64 (||D|| <= 8)."""
    dims, mass = (8, 8, 8, 8), 0.01
    U = syn.random_links(dims, 0.5, 1004)
    X = syn.gaussian_pseudofermions(dims, 1, 2003)
    lam = 0.0
    for _ in range(40):
        Y = oracle.apply_A(dims, mass, U, X)
        lam = np.vdot(X, Y).real / np.vdot(X, X).real
        X = Y / np.linalg.norm(Y)
    assert 4 * mass ** 2 < lam <= 4 * mass ** 2 + 64


def _gauge_transform(dims, U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dagger in the (T,Z,Y,X,mu,3,3) layout."""
    Ug = np.empty_like(U)
    for mu, ax in ((0, 3), (1, 2), (2, 1), (3, 0)):
        gp = np.roll(g, -1, axis=ax)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    return Ug


def _apply_g(dims, g, X, parity):
    lex = dense.parity_lex(dims, parity)
    gf = g.reshape(-1, 3, 3)[lex]
    return np.einsum("hab,hbi->hai", gf, X)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 4)])
def test_gauge_covariance(dims):
    U = syn.random_links(dims, 0.5, 1005)
    g = syn.random_gauge_transform(dims)
    X = syn.gaussian_pseudofermions(dims, 2, 2004)
    Ug = _gauge_transform(dims, U, g)
    lhs = oracle.apply_A(dims, 0.1, Ug, _apply_g(dims, g, X, 0))
    rhs = _apply_g(dims, g, oracle.apply_A(dims, 0.1, U, X), 0)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13 * np.abs(rhs).max())


def test_apply_at_matches_full():
    dims = (4, 4, 2, 6)
    U = syn.random_links(dims, 0.5, 1006)
    X = syn.gaussian_pseudofermions(dims, 3, 2005)
    full = oracle.apply_A(dims, 0.03, U, X, sigma=0.25)
    sites = [0, 1, 17, 95]
    np.testing.assert_allclose(oracle.apply_A_at(dims, 0.03, U, X, sites, sigma=0.25), full[sites], atol=1e-13)


def test_links_are_su3():
    U = syn.random_links((2, 2, 2, 2), 0.5, 1007).reshape(-1, 3, 3)
    eye = np.einsum("kab,kcb->kac", U, U.conj())
    np.testing.assert_allclose(eye, np.broadcast_to(np.eye(3), eye.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(U), 1.0, atol=1e-13)
