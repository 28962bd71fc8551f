"""GPU parity against the FP64 oracle at the two largest single-lattice workloads.

* 16^3 x 32, m = 0.02, n_pf = 8, 14 shifts of x^(-1/32) on [1e-3, 64], mixed
  precision, tol 1e-8: every (shift, column) solution of SBCGrQ (Algorithm 1)
  against the oracle solved to 1e-13 (true residual with the oracle's operator
  and the solution-error bound), and the force of Eq. (force) against the
  oracle's force, both from the oracle's solutions (bound of the solve) and
  from the GPU's own solutions (kernel-level parity, 1e-12).
* 24^4, m = 0.01, n_pf = 16, 16 shifts of x^(-1/64) on [4e-4, 64], mixed, tol
  1e-8 (the force-evaluation workload): every (shift, column) true residual
  of the GPU's solutions with the oracle's operator, which bounds the solution
  error rigorously (||X - X*|| <= ||R|| / (4m^2 + sigma_s) since
  lambda_min(A) >= 4m^2); the force computed on the GPU from those solutions
  against the oracle's force on 64 sampled links (t-boundary and wrap links
  included) at 1e-12; the force of the full call (solve inside) against the
  force from the separately solved X within the solution-error bound.

Every number these tests compare is printed (pytest -s) as a per-result error.
"""
import numpy as np
import pytest

import oracle
from gpu_util import check_solution, force_bound, make_ctx, need_gpu, sample_links, to_gpu
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx

pytestmark = pytest.mark.gpu


def _link_rows(dims, links):
    """Index rows of G [V][4][3][3] for (lex, mu) pairs."""
    return np.ascontiguousarray(links[:, 0]), np.ascontiguousarray(links[:, 1])


def test_mixed_16x16x16x32_npf8_solutions_and_force_match_oracle():
    need_gpu()
    dims, mass, n, tol = (16, 16, 16, 32), 0.02, 8, 1e-8
    ra = rational_approx(-1.0 / 32, 1e-3, 64.0, 14)
    U = syn.random_links(dims, 0.5, syn.seed_gauge(2))
    Phi = syn.gaussian_pseudofermions(dims, n, syn.seed_phi(2))
    ctx = make_ctx(dims, mass, U)
    Pd = to_gpu(Phi)
    Xg_d, info = ctx.block_multishift_cg(Pd, ra.beta, tol, precision="mixed")
    assert info.true_rel_resid_max <= tol
    G, S, finfo = ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, tol, precision="mixed")
    Gx, _, _ = ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, tol, X=Xg_d)
    Xg, G, Gx = Xg_d.cpu().numpy(), G.cpu().numpy(), Gx.cpu().numpy()
    ctx.close()

    Xo, iters, rc = oracle.sbcgrq(dims, mass, U, Phi, ra.beta, tol=1e-13, max_iter=20000)
    assert rc == 0
    worst_r, worst_e = check_solution(dims, mass, U, Phi, ra.beta, Xg, tol, Xo)
    Go = oracle.force(dims, U, Xo, ra.alpha)
    So = oracle.action(ra.alpha0, ra.alpha, Phi, Xo)
    bound = force_bound(mass, Phi, ra.beta, Xo, tol)
    ferr = np.linalg.norm(G - Go) / np.linalg.norm(Go)
    serr = abs(S - So) / abs(So)
    assert ferr <= bound and serr <= bound, (ferr, serr, bound)
    # kernel-level: the oracle's force of the GPU's own solutions
    Gox = oracle.force(dims, U, Xg, ra.alpha)
    kerr = np.linalg.norm(Gx - Gox) / np.linalg.norm(Gox)
    assert kerr <= 1e-12, kerr
    print(f"\n16^3x32 n_pf=8 mixed: GPU {info.iters} iters (oracle {iters}), max true resid/tol {worst_r:.3f}, "
          f"max solution err/bound {worst_e:.3f}, force err {ferr:.2e} (bound {bound:.2e}), action err {serr:.2e}, "
          f"force kernel err {kerr:.2e}")


def test_force_workload_24x4_npf16_parity():
    need_gpu()
    dims, mass, n, tol = (24, 24, 24, 24), 0.01, 16, 1e-8
    ra = rational_approx(-1.0 / 64, 4e-4, 64.0, 16)
    U = syn.random_links(dims, 0.5, syn.seed_gauge(3))
    Phi = syn.gaussian_pseudofermions(dims, n, syn.seed_phi(3))
    ctx = make_ctx(dims, mass, U)
    Pd = to_gpu(Phi)
    # the force evaluation as timed (solve inside the call)
    G, S, finfo = ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, tol, precision="mixed")
    assert finfo.true_rel_resid_max <= tol
    # the same solve through the solver entry point, and the force from its X
    Xg_d, info = ctx.block_multishift_cg(Pd, ra.beta, tol, precision="mixed")
    Gx, Sx, _ = ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, tol, X=Xg_d)
    links = sample_links(dims, 64, 4242)
    rows, mus = (to_gpu(a) for a in _link_rows(dims, links))
    Gs = G[rows, mus].cpu().numpy()
    Gxs = Gx[rows, mus].cpu().numpy()
    gdiff = float((G - Gx).norm() / Gx.norm())
    Xg = Xg_d.cpu().numpy()
    del Xg_d
    ctx.close()

    worst_r, _ = check_solution(dims, mass, U, Phi, ra.beta, Xg, tol)
    Go = oracle.force_at(dims, U, Xg, ra.alpha, links)
    kerr = np.linalg.norm(Gxs - Go) / np.linalg.norm(Go)
    kerr_link = max(np.linalg.norm(Gxs[k] - Go[k]) / np.linalg.norm(Go[k]) for k in range(len(links)))
    assert kerr <= 1e-12 and kerr_link <= 1e-11, (kerr, kerr_link)
    # the full call's force against the force from the separately solved X: both come
    # from solves with every true residual <= tol, so they differ by at most twice the
    # error a solve to tol allows
    bound = 2 * force_bound(mass, Phi, ra.beta, Xg, tol)
    assert gdiff <= bound, (gdiff, bound)
    sample_err = np.linalg.norm(Gs - Go) / np.linalg.norm(Go)
    assert abs(S - Sx) <= bound * abs(Sx)
    print(f"\n24^4 n_pf=16 mixed: {info.iters} iters, max true resid/tol {worst_r:.3f} (oracle operator), "
          f"force kernel err on 64 links {kerr:.2e} (worst link {kerr_link:.2e}), full call vs given-X force "
          f"{gdiff:.2e} (sampled {sample_err:.2e}, bound {bound:.2e})")
