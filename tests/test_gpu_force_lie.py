"""rhmc_force_lie (Lie-algebra force F = TA(U G^dagger) and the force norm
sum_a (F^a)^2 / 2 of Sec. II) against the oracle's component-wise definition,
on random links and forces, in place and norm-only, and on the force of an
actual solve."""
import numpy as np
import pytest

import oracle
from oracle import dense
from gpu_util import make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6), (6, 4, 4, 8)])
def test_force_lie_matches_oracle(dims):
    need_gpu()
    rng = np.random.default_rng(51)
    U = syn.random_links(dims, 0.6, 1051)
    G = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    ctx = make_ctx(dims, 0.1, U)
    V = int(np.prod(dims))
    Ug, Gg = to_gpu(U.reshape(V, 4, 3, 3)), to_gpu(G.reshape(V, 4, 3, 3))
    F, n2 = ctx.force_lie(Ug, Gg)
    Fo = dense.force_lie(U, G).reshape(V, 4, 3, 3)
    n2o = dense.force_norm2(U, G)
    assert np.max(np.abs(F.cpu().numpy() - Fo)) <= 1e-13 * np.max(np.abs(Fo))
    assert abs(n2 - n2o) <= 1e-12 * n2o
    # norm only, then in place over G: the same numbers
    _, n2b = ctx.force_lie(Ug, Gg, want_F=False)
    assert n2b == n2
    F2, n2c = ctx.force_lie(Ug, Gg, out=Gg)
    assert n2c == n2
    assert np.array_equal(Gg.cpu().numpy(), F.cpu().numpy())
    ctx.close()


def test_force_lie_of_a_solve():
    """F and F^2 of the library's own force on a small ensemble match the oracle's
    component-wise definition applied to the oracle's force."""
    need_gpu()
    dims, mass, n = (4, 4, 4, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1052)
    Phi = syn.gaussian_pseudofermions(dims, n, 2052)
    ctx = make_ctx(dims, mass, U)
    V = int(np.prod(dims))
    G, _, _ = ctx.force(to_gpu(Phi), ra.alpha0, ra.alpha, ra.beta, 1e-12, precision="fp64")
    F, n2 = ctx.force_lie(to_gpu(U.reshape(V, 4, 3, 3)), G)
    Xo, _, rc = oracle.sbcgrq(dims, mass, U, Phi, ra.beta, tol=1e-13)
    assert rc == 0
    Go = oracle.force(dims, U, Xo, ra.alpha).reshape(U.shape)
    Fo = dense.force_lie(U, Go).reshape(V, 4, 3, 3)
    n2o = dense.force_norm2(U, Go)
    assert np.linalg.norm(F.cpu().numpy() - Fo) <= 1e-9 * np.linalg.norm(Fo)
    assert abs(n2 - n2o) <= 1e-9 * n2o
    ctx.close()
