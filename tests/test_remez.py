"""Pins of the rational approximation of Eq. (RA).

* Chebyshev alternation: 2N+2 alternating extrema of equal magnitude (the
  defining property of the unique minimax approximation);
* alpha_j > 0, beta_j > 0 (Sec. II) and poles outside [a, b];
* the error on a dense grid never exceeds the levelled error;
* r = -1/2 reproduces Zolotarev's closed form (Jacobi elliptic functions);
* the matrix function R(A) phi approximates A^r phi within the bound, with
  A^r from a dense eigendecomposition;
* the stated accuracy levels of Sec. IV are reachable: relative error < 1e-7
  with about 15 shifts, < 1e-15 with about 30.
"""
import numpy as np
import pytest

from oracle import dense
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import STANDARD, rational_approx, remez

mp = pytest.importorskip("mpmath")


def _rel_err(ra, x):
    return ra(x) / x ** ra.r - 1.0


@pytest.fixture(scope="module")
def small():
    return remez(-0.25, 1e-2, 50.0, 5)


def test_alternation(small):
    ext = np.array(small.extrema)
    assert len(ext) == 2 * 5 + 2
    e = _rel_err(small, ext)
    assert np.all(np.sign(e[1:]) == -np.sign(e[:-1]))
    assert np.max(np.abs(e)) / np.min(np.abs(e)) - 1 < 1e-3
    assert ext[0] == pytest.approx(1e-2) and ext[-1] == pytest.approx(50.0)


@pytest.mark.parametrize("params", STANDARD)
def test_standard_positive_and_bounded(params):
    ra = rational_approx(*params)
    assert ra.alpha0 > 0
    # x^r is a Stieltjes function for -1 < r < 0 (positive residues); for
    # 0 < r < 1, x^r = x * x^(r-1) makes every residue negative
    sgn = 1 if params[0] < 0 else -1
    assert all(sgn * a > 0 for a in ra.alpha)
    assert all(b > 0 for b in ra.beta)
    x = np.exp(np.linspace(np.log(ra.a), np.log(ra.b), 100_000))
    assert np.max(np.abs(_rel_err(ra, x))) <= ra.error * (1 + 1e-3) + 1e-14


def test_zolotarev_closed_form():
    """x^(-1/2) on [a, b]: the minimax relative approximation of type (n, n)
    has its poles at -a c_(2m-1), c_l = sn^2(l K'/(2n+1); k') / cn^2(l K'/(2n+1); k'),
    k'^2 = 1 - a/b (Zolotarev)."""
    a, b, n = 1e-3, 2.0, 7
    ra = remez(-0.5, a, b, n, equi_tol=1e-6)
    mp.mp.dps = 40
    m1 = 1 - mp.mpf(a) / b
    K = mp.ellipk(m1)
    c = [mp.ellipfun("sn", l * K / (2 * n + 1), m=m1) ** 2 / mp.ellipfun("cn", l * K / (2 * n + 1), m=m1) ** 2
         for l in range(1, 2 * n + 1)]
    poles = sorted(float(a * c[2 * m - 2]) for m in range(1, n + 1))
    np.testing.assert_allclose(ra.beta, poles, rtol=1e-7)
    # the numerator roots are the even-index constants
    zeros = sorted(float(a * c[2 * m - 1]) for m in range(1, n + 1))
    for z in zeros:
        assert abs(ra(np.array([-z]))[0]) < 1e-6 * ra.alpha0 * 1e3


def test_matrix_function_bound():
    dims, mass = (4, 4, 4, 4), 0.1
    ra = rational_approx(-1.0 / 8, 1e-3, 64.0, 8)
    U = syn.random_links(dims, 0.3, 1000)
    Phi = syn.gaussian_pseudofermions(dims, 2, 2000)
    A = dense.dense_A(dims, mass, U)
    w = np.linalg.eigvalsh(A)
    assert ra.a <= w.min() and w.max() <= ra.b
    B = dense.field_to_vec(Phi)
    RB = ra.alpha0 * B + sum(al * dense.solve(A, B, be) for al, be in zip(ra.alpha, ra.beta))
    exact = dense.field_to_vec(dense.matrix_power_apply(dims, mass, U, Phi, ra.r))
    assert np.linalg.norm(RB - exact) <= ra.error * np.linalg.norm(exact) * (1 + 1e-6)


@pytest.mark.slow
def test_paper_accuracy_levels():
    """Sec. IV: force approximations < 1e-7 with ~15 shifts; heatbath < 1e-15 with ~30."""
    assert rational_approx(-1.0 / 64, 4e-4, 64.0, 16).error < 1e-7
    # the 24-pole heatbath set is cached (its exchange takes minutes at the
    # working precision); the grid check below re-evaluates it independently,
    # in FP64, whose rounding over 25 terms adds a few 1e-16
    hb = rational_approx(1.0 / 128, 4e-4, 64.0, 24)
    assert hb.error < 1e-15
    x = np.exp(np.linspace(np.log(hb.a), np.log(hb.b), 200_000))
    assert np.max(np.abs(hb(x) / x ** (1.0 / 128) - 1)) < 4e-15
