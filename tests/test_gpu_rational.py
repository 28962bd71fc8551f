"""rhmc_rational_solve: R(A) Phi of Eq. (RA) by the block multishift solve
without per-shift solutions (the pseudofermion heatbath and the action need
only the rational sum), FP64.  Checked against the oracle's solutions combined
with the same coefficients, against rhmc_block_multishift_cg +
rhmc_rational_apply, and against the action from rhmc_force."""
import numpy as np
import pytest

import oracle
from gpu_util import make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx

pytestmark = pytest.mark.gpu

CASES = [
    # dims, mass, n, (r, a, b, N), eps, tol
    ((4, 4, 4, 4), 0.1, 2, (-1.0 / 8, 1e-3, 64.0, 8), 0.3, 1e-12),   # action: x^(-1/8)
    ((4, 4, 4, 4), 0.1, 2, (1.0 / 16, 1e-3, 64.0, 8), 0.3, 1e-14),   # heatbath: x^(+1/16), negative residues
    ((8, 8, 8, 8), 0.05, 4, (1.0 / 32, 2e-3, 64.0, 12), 0.5, 1e-13),
    ((4, 6, 4, 8), 0.03, 5, (-1.0 / 20, 1e-3, 64.0, 6), 0.5, 1e-12),
]


def _oracle_sum(dims, mass, U, Phi, ra):
    Xo, _, rc = oracle.sbcgrq(dims, mass, U, Phi, ra.beta, tol=1e-14, max_iter=20000)
    assert rc == 0
    return ra.alpha0 * Phi + sum(a * Xo[s] for s, a in enumerate(ra.alpha))


def _bound(Phi, ra, mass, tol):
    # a column residual r_s <= tol ||Phi|| moves X^(s) by at most r_s / (4 m^2 + beta_s)
    pn = np.linalg.norm(Phi.reshape(-1, Phi.shape[-1]), axis=0)
    return pn * tol * sum(abs(a) / (4 * mass ** 2 + b) for a, b in zip(ra.alpha, ra.beta))


@pytest.mark.parametrize("dims,mass,n,rp,eps,tol", CASES)
def test_rational_solve_matches_oracle(dims, mass, n, rp, eps, tol):
    need_gpu()
    ra = rational_approx(*rp)
    U = syn.random_links(dims, eps, 1260)
    Phi = syn.gaussian_pseudofermions(dims, n, 2260)
    ctx = make_ctx(dims, mass, U)
    Y, info = ctx.rational_solve(to_gpu(Phi), ra.alpha0, ra.alpha, ra.beta, tol)
    assert info.phase1_rel_resid_max <= tol
    assert info.true_rel_resid_max <= 10 * tol
    Yo = _oracle_sum(dims, mass, U, Phi, ra)
    err = np.linalg.norm((Y.cpu().numpy() - Yo).reshape(-1, n), axis=0)
    yn = np.linalg.norm(Yo.reshape(-1, n), axis=0)
    assert np.all(err <= 10 * _bound(Phi, ra, mass, tol) + 1e-12 * yn), err / yn
    ctx.close()


def test_rational_solve_agrees_with_stored_solutions_and_action():
    need_gpu()
    dims, mass, n = (8, 4, 4, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1261)
    Phi = syn.gaussian_pseudofermions(dims, n, 2261)
    ctx = make_ctx(dims, mass, U)
    P = to_gpu(Phi)
    tol = 1e-12
    Y, _ = ctx.rational_solve(P, ra.alpha0, ra.alpha, ra.beta, tol)
    X, _ = ctx.block_multishift_cg(P, ra.beta, tol, precision="fp64")
    from paper_1808_01829_gb300.api import _ptr, _doubles, _stream
    import torch

    Y2 = torch.empty_like(P)
    assert ctx.lib.rhmc_rational_apply(ctx._h, _ptr(P), n, ra.alpha0, _doubles(ra.alpha), len(ra.alpha), _ptr(X),
                                       _ptr(Y2), _stream(P)) == 0
    y, y2 = Y.cpu().numpy(), Y2.cpu().numpy()
    assert np.all(np.linalg.norm((y - y2).reshape(-1, n), axis=0) <= 2 * _bound(Phi, ra, mass, tol)
                  + 1e-12 * np.linalg.norm(y2.reshape(-1, n), axis=0))
    # the action S = sum_i Re phi_i^dagger R(A) phi_i, as rhmc_force reports it
    _, S, _ = ctx.force(P, ra.alpha0, ra.alpha, ra.beta, tol, precision="fp64", X=X)
    S_rs = float(np.real(np.vdot(Phi, y)))
    assert abs(S_rs - S) <= 1e-10 * abs(S)
    # no per-shift solutions: far less workspace than the stored-solution solve
    assert ctx.lib.rhmc_rational_solve_bytes(ctx._h, n, len(ra.beta)) < \
        ctx.lib.rhmc_workspace_bytes(ctx._h, n, len(ra.beta), 0)
    ctx.close()
