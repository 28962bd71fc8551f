"""PseudofermionAction (torch.autograd.Function over the C ABI): gradients against
central finite differences of the action (Eq. (force) as the derivative of
Eq. (RA)'s action), store vs recompute of the solutions, and the action against
the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx

pytestmark = pytest.mark.gpu


def _action(rctx, U, Phi, ra, tol, prec):
    from paper_1808_01829_gb300.action import pseudofermion_action

    return float(pseudofermion_action(U, Phi, rctx, ra, tol=tol, precision=prec))


@pytest.mark.parametrize("dims,mass,n,rp", [((4, 4, 4, 4), 0.1, 2, (-1.0 / 8, 1e-3, 64.0, 8)),
                                             ((8, 8, 8, 8), 0.05, 4, (-1.0 / 16, 2e-3, 64.0, 12))])
def test_gradients_match_finite_differences(dims, mass, n, rp):
    torch = need_gpu()
    from paper_1808_01829_gb300.action import pseudofermion_action

    ra = rational_approx(*rp)
    U0 = syn.random_links(dims, 0.5, 1400)
    P0 = syn.gaussian_pseudofermions(dims, n, 2400)
    rctx = make_ctx(dims, mass, U0)
    U = to_gpu(U0).requires_grad_(True)
    Phi = to_gpu(P0).requires_grad_(True)
    S = pseudofermion_action(U, Phi, rctx, ra, tol=1e-12, precision="fp64")
    S.backward()
    # action against the oracle
    Xo, _, _ = oracle.sbcgrq(dims, mass, U0, P0, ra.beta, tol=1e-13)
    So = oracle.action(ra.alpha0, ra.alpha, P0, Xo)
    assert abs(float(S.detach()) - So) <= 1e-10 * abs(So)
    rng = np.random.default_rng(7)
    h = 1e-4
    for _ in range(3):
        V = to_gpu(rng.standard_normal(U0.shape) + 1j * rng.standard_normal(U0.shape))
        fd = (_action(rctx, (U + h * V).detach(), Phi.detach(), ra, 1e-12, "fp64")
              - _action(rctx, (U - h * V).detach(), Phi.detach(), ra, 1e-12, "fp64")) / (2 * h)
        an = float(torch.vdot(U.grad.reshape(-1), V.reshape(-1)).real)
        assert abs(fd - an) <= 1e-6 * abs(an)
        W = to_gpu(rng.standard_normal(P0.shape) + 1j * rng.standard_normal(P0.shape))
        fdp = (_action(rctx, U.detach(), (Phi + h * W).detach(), ra, 1e-12, "fp64")
               - _action(rctx, U.detach(), (Phi - h * W).detach(), ra, 1e-12, "fp64")) / (2 * h)
        anp = float(torch.vdot(Phi.grad.reshape(-1), W.reshape(-1)).real)
        assert abs(fdp - anp) <= 1e-6 * abs(anp)
    rctx.close()


def test_store_and_recompute_agree():
    torch = need_gpu()
    from paper_1808_01829_gb300.action import pseudofermion_action

    dims, mass, n = (8, 4, 4, 8), 0.05, 3
    ra = rational_approx(-1.0 / 12, 1e-3, 64.0, 5)
    U0 = syn.random_links(dims, 0.5, 1401)
    P0 = syn.gaussian_pseudofermions(dims, n, 2401)
    rctx = make_ctx(dims, mass, U0)
    grads = []
    for store in (True, False):
        U = to_gpu(U0).requires_grad_(True)
        S = pseudofermion_action(U, to_gpu(P0), rctx, ra, tol=1e-10, precision="fp64", store=store)
        S.backward()
        grads.append(U.grad.clone())
    assert torch.allclose(grads[0], grads[1], rtol=0, atol=1e-9 * float(grads[0].abs().max()))
    rctx.close()


def test_force_workload_directional_derivatives():
    """24^4, n_pf = 16, 16 shifts (the force workload).

    * The backward pass (Eq. (force)) against central differences (h = 1e-5) of
      the action on 32 random complex link directions.  Gradient and actions
      come from solves to 1e-11 (FP64-accurate results of the mixed solver), so
      the comparison measures the derivative and its kernels, not the solver's
      stopping error.  Bound per direction: 1e-6 |Re<G, V>| + 1e-13 |S| / h, the
      second term being the resolution of S itself (an FP64 sum of V/2 * 3 * n
      products, left by the solves with about 1e-13 relative rounding), which the
      difference quotient divides by h.
    * The gradient of the production solve (tol 1e-8) against that one, norm-wise,
      within the force error a solve to 1e-8 allows:
      2 max_s tol ||Phi|| / ((4m^2 + beta_s) ||X^(s)||)."""
    torch = need_gpu()
    from paper_1808_01829_gb300.action import pseudofermion_action

    dims, mass, n = (24, 24, 24, 24), 0.01, 16
    ra = rational_approx(-1.0 / 64, 4e-4, 64.0, 16)
    U0 = syn.random_links(dims, 0.5, syn.seed_gauge(3))
    P0 = syn.gaussian_pseudofermions(dims, n, syn.seed_phi(3))
    rctx = make_ctx(dims, mass, U0)
    Phi = to_gpu(P0)
    grads = {}
    for tol in (1e-8, 1e-11):
        U = to_gpu(U0).requires_grad_(True)
        S = pseudofermion_action(U, Phi, rctx, ra, tol=tol, precision="mixed")
        S.backward()
        grads[tol] = U.grad
    U = to_gpu(U0)
    G = grads[1e-11]
    S0 = abs(_action(rctx, U, Phi, ra, 1e-11, "mixed"))
    gen = torch.Generator(device=U.device)
    gen.manual_seed(11)
    h = 1e-5
    worst = 0.0
    for _ in range(32):
        V = torch.randn(U0.shape, dtype=torch.complex128, device=U.device, generator=gen)
        fd = (_action(rctx, U + h * V, Phi, ra, 1e-11, "mixed")
              - _action(rctx, U - h * V, Phi, ra, 1e-11, "mixed")) / (2 * h)
        an = float(torch.vdot(G.reshape(-1), V.reshape(-1)).real)
        tol_fd = 1e-6 * abs(an) + 1e-13 * S0 / h
        worst = max(worst, abs(fd - an) / tol_fd)
        assert abs(fd - an) <= tol_fd, (fd, an, S0)
    X, _ = rctx.block_multishift_cg(Phi, ra.beta, 1e-11, precision="mixed")
    xn = [float(X[s].norm()) for s in range(len(ra.beta))]
    del X
    bound = 2 * max(1e-8 * float(Phi.norm()) / ((4 * mass ** 2 + b) * xn[s]) for s, b in enumerate(ra.beta)) + 1e-10
    gerr = float((grads[1e-8] - G).norm() / G.norm())
    assert gerr <= bound, (gerr, bound)
    print(f"\n24^4 force vs central differences (h = 1e-5), 32 directions: worst difference / bound {worst:.2f}; "
          f"tol 1e-8 gradient vs tol 1e-11 gradient {gerr:.2e} (bound {bound:.2e})")
    rctx.close()
