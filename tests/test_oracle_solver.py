"""Pins of the oracle's SBCGrQ (Algorithm 1) and scalar multishift CG.

* dense brute force: X^(s) = (A + sigma_s)^-1 B by LU on 2^4 and 4^4;
* n_pf = 1: the block solver's iterates equal scalar multishift CG's (Sec. III:
  BCG is CG for one right-hand side, SBCGrQ reduces to SCG);
* Galerkin optimality: after k iterations every shifted iterate X^(s)_k is the
  minimiser of Tr[E^dagger (A + sigma_s) E] over the block Krylov space
  {B, A B, ..., A^(k-1) B} (Sec. III: BCG minimises this trace; the Krylov
  space is shift invariant), computed by explicit projection;
* one shift (N_s = 1) is BCGrQ: the smallest shift's iterates do not depend on the
  other shifts;
* a duplicated shift gives identical solutions; the true residual is below the
  tolerance; the rigorous bound ||X - X*|| <= ||R|| / (lambda_min + sigma);
* breakdown and non-convergence are reported, not crashed on.
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1808_01829_gb300 import synthetic as syn

SHIFTS = [0.002, 0.03, 0.4, 5.0, 60.0]


def _setup(dims, n, eps=0.5, seed=0):
    U = syn.random_links(dims, eps, 1000 + seed)
    B = syn.gaussian_pseudofermions(dims, n, 2000 + seed)
    return U, B


@pytest.mark.parametrize("dims,n", [((2, 2, 2, 2), 2), ((4, 4, 4, 4), 2), ((4, 4, 4, 4), 5), ((2, 4, 2, 4), 3)])
def test_sbcgrq_matches_dense_lu(dims, n):
    mass = 0.1
    U, B = _setup(dims, n)
    X, iters, rc = oracle.sbcgrq(dims, mass, U, B, SHIFTS, tol=1e-13, max_iter=2000)
    assert rc == 0
    A = dense.dense_A(dims, mass, U)
    for s, sig in enumerate(SHIFTS):
        Xd = dense.vec_to_field(dense.solve(A, dense.field_to_vec(B), sig), n)
        assert np.linalg.norm(X[s] - Xd) <= 1e-11 * np.linalg.norm(Xd)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8)])
def test_n1_block_iterates_equal_scalar_multishift_cg(dims):
    mass = 0.05
    U, B = _setup(dims, 1, seed=1)
    Xb, _, rc1 = oracle.sbcgrq(dims, mass, U, B, SHIFTS, fixed_iters=20)
    xs, _, rc2 = oracle.scg(dims, mass, U, B[..., 0], SHIFTS, fixed_iters=20)
    assert rc1 == 0 and rc2 == 0
    for s in range(len(SHIFTS)):
        assert np.linalg.norm(Xb[s][..., 0] - xs[s]) <= 1e-12 * np.linalg.norm(xs[s])
    # converged iteration counts agree within one
    _, kb, _ = oracle.sbcgrq(dims, mass, U, B, SHIFTS, tol=1e-9)
    _, ks, _ = oracle.scg(dims, mass, U, B[..., 0], SHIFTS, tol=1e-9)
    assert abs(kb - ks) <= 1


@pytest.mark.parametrize("k", [1, 2, 3])
def test_galerkin_optimality_all_shifts(k):
    dims, mass, n = (4, 4, 4, 4), 0.1, 3
    U, B = _setup(dims, n, seed=2)
    X, _, rc = oracle.sbcgrq(dims, mass, U, B, SHIFTS, fixed_iters=k)
    assert rc == 0
    A = dense.dense_A(dims, mass, U)
    Bv = dense.field_to_vec(B)
    A0 = A + SHIFTS[0] * np.eye(A.shape[0])
    blocks, cur = [], Bv
    for _ in range(k):
        blocks.append(cur)
        cur = A0 @ cur
    K, _ = np.linalg.qr(np.concatenate(blocks, axis=1))
    for s, sig in enumerate(SHIFTS):
        As = A + sig * np.eye(A.shape[0])
        Xopt = K @ np.linalg.solve(K.conj().T @ As @ K, K.conj().T @ Bv)
        got = dense.field_to_vec(X[s])
        assert np.linalg.norm(got - Xopt) <= 1e-10 * np.linalg.norm(Xopt), (s, k)


def test_duplicate_shift_gives_identical_solution():
    dims, mass = (4, 4, 4, 4), 0.1
    U, B = _setup(dims, 2, seed=3)
    shifts = [0.01, 0.01, 0.5, 0.5]
    X, _, rc = oracle.sbcgrq(dims, mass, U, B, shifts, tol=1e-12)
    assert rc == 0
    assert np.linalg.norm(X[1] - X[0]) <= 1e-13 * np.linalg.norm(X[0])
    assert np.linalg.norm(X[3] - X[2]) <= 1e-13 * np.linalg.norm(X[2])


@pytest.mark.parametrize("dims,mass,n", [((8, 8, 8, 8), 0.05, 4), ((4, 4, 4, 8), 0.02, 3)])
def test_true_residual_and_error_bound(dims, mass, n):
    U, B = _setup(dims, n, seed=4)
    tol = 1e-10
    X, iters, rc = oracle.sbcgrq(dims, mass, U, B, SHIFTS, tol=tol)
    assert rc == 0
    bn = np.linalg.norm(B, axis=(0, 1))
    for s, sig in enumerate(SHIFTS):
        R = B - oracle.apply_A(dims, mass, U, X[s], sigma=sig)
        rn = np.linalg.norm(R, axis=(0, 1))
        assert np.all(rn <= 2 * tol * bn), (s, rn / bn)
        if dims == (4, 4, 4, 8):
            A = dense.dense_A(dims, mass, U)
            Xd = dense.vec_to_field(dense.solve(A, dense.field_to_vec(B), sig), n)
            lam_min = 4 * mass ** 2
            err = np.linalg.norm(X[s] - Xd, axis=(0, 1))
            assert np.all(err <= rn / (lam_min + sig) * (1 + 1e-6) + 1e-14 * np.linalg.norm(Xd))


def test_iterations_decrease_with_npf():
    """Block Krylov space grows by n_pf per iteration: more columns, fewer iterations (Eq. (convergence_bound))."""
    dims, mass = (8, 8, 8, 8), 0.01
    U = syn.random_links(dims, 0.5, 1010)
    its = []
    for n in (1, 4, 8):
        B = syn.gaussian_pseudofermions(dims, n, 2010)
        _, k, rc = oracle.sbcgrq(dims, mass, U, B, [1e-4], tol=1e-8)
        assert rc == 0
        its.append(k)
    assert its[0] > its[1] > its[2]


def test_breakdown_on_rank_deficient_block():
    dims = (4, 4, 4, 4)
    U, B = _setup(dims, 2, seed=5)
    B[..., 1] = B[..., 0]
    X, _, rc = oracle.sbcgrq(dims, 0.1, U, B, SHIFTS, tol=1e-10)
    assert rc == 3


def test_not_converged_status():
    dims = (4, 4, 4, 4)
    U, B = _setup(dims, 2, seed=6)
    _, k, rc = oracle.sbcgrq(dims, 0.01, U, B, SHIFTS, tol=1e-12, max_iter=3)
    assert rc == 2 and k == 3


def test_thin_qr():
    rng = np.random.default_rng(7)
    B = rng.standard_normal((200, 6)) + 1j * rng.standard_normal((200, 6))
    Q, R = oracle.thin_qr(B)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(Q @ R, B, atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0)
    d = np.diag(R)
    assert np.all(d.real > 0) and np.allclose(d.imag, 0)
    # unique thin QR: agrees with numpy's after fixing the diagonal phase
    Qn, Rn = np.linalg.qr(B)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    np.testing.assert_allclose(Q, Qn * ph[None, :], atol=1e-12)


def test_single_shift_is_bcgrq():
    """N_s = 1 reduces SBCGrQ to BCGrQ: the smallest shift's iterates do not depend on
    the other shifts (the base recursion never reads them), so a fixed number of
    iterations gives the same X^(0) with or without them, to rounding of the same
    operations."""
    dims, mass, n = (4, 4, 4, 4), 0.05, 3
    U, B = _setup(dims, n, seed=7)
    for iters in (1, 7, 20):
        X1, _, rc1 = oracle.sbcgrq(dims, mass, U, B, [SHIFTS[0]], fixed_iters=iters)
        Xm, _, rcm = oracle.sbcgrq(dims, mass, U, B, SHIFTS, fixed_iters=iters)
        assert rc1 == 0 and rcm == 0
        assert np.linalg.norm(X1[0] - Xm[0]) <= 1e-14 * np.linalg.norm(Xm[0])
