"""GPU parity of the multi-RHS staggered operator against the oracle (Sec. IV).

FP64: 1e-12 relative per column; FP32 kernel: 1e-6.  Sizes span several CTA
tiles with a ragged tail (odd site counts per tile, n not dividing 256), both
boundary conditions, n = 1 (no staging) to 16."""
import numpy as np
import pytest

import oracle
from gpu_util import colrel, make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

CASES = [
    ((4, 4, 4, 4), 2, -1),
    ((8, 8, 8, 8), 4, -1),
    ((4, 2, 6, 4), 3, 1),
    ((6, 4, 4, 2), 12, -1),
    ((8, 4, 4, 6), 16, 1),
    ((4, 4, 4, 8), 1, -1),
    ((2, 2, 2, 2), 5, -1),
]


@pytest.mark.parametrize("dims,n,bc", CASES)
def test_hop_fp64_fp32(dims, n, bc):
    need_gpu()
    U = syn.random_links(dims, 0.5, 1100)
    X = syn.gaussian_pseudofermions(dims, n, 2100)
    ctx = make_ctx(dims, 0.1, U, bc)
    for par in (0, 1):
        ref = oracle.hop(dims, U, X, par, bc_t=bc)
        got = ctx.hop(to_gpu(X), par, "fp64").cpu().numpy()
        assert colrel(got, ref) <= 1e-12
        got32 = ctx.hop(to_gpu(X), par, "fp32").cpu().numpy()
        assert colrel(got32, ref) <= 1e-6
        gotdf = ctx.hop(to_gpu(X), par, "df64").cpu().numpy()
        assert colrel(gotdf, ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("dims,n,bc", CASES)
@pytest.mark.parametrize("sigma", [0.0, 0.37])
def test_apply_mdagm(dims, n, bc, sigma):
    need_gpu()
    mass = 0.05
    U = syn.random_links(dims, 0.5, 1101)
    X = syn.gaussian_pseudofermions(dims, n, 2101)
    ctx = make_ctx(dims, mass, U, bc)
    ref = oracle.apply_A(dims, mass, U, X, sigma=sigma, bc_t=bc)
    got = ctx.apply_mdagm_mrhs(to_gpu(X), sigma, "fp64").cpu().numpy()
    assert colrel(got, ref) <= 1e-12
    got32 = ctx.apply_mdagm_mrhs(to_gpu(X), sigma, "fp32").cpu().numpy()
    assert colrel(got32, ref) <= 1e-6
    gotdf = ctx.apply_mdagm_mrhs(to_gpu(X), sigma, "df64").cpu().numpy()
    assert colrel(gotdf, ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 4), 2), ((6, 4, 4, 2), 6), ((8, 4, 4, 6), 10), ((4, 6, 4, 4), 14),
                                    ((8, 8, 8, 8), 16)])
def test_hop_fp32_kernel_variants(dims, n):
    """Every FP32 hop kernel (cp.async-staged tiles, register staged, all
    directions in flight) and every right-hand-sides-per-thread choice give the
    same operator (1e-6)."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    mass, sigma = 0.05, 0.21
    U = syn.random_links(dims, 0.5, 1102)
    X = syn.gaussian_pseudofermions(dims, n, 2102)
    ctx = make_ctx(dims, mass, U)
    refs = [oracle.hop(dims, U, X, par) for par in (0, 1)]
    refA = oracle.apply_A(dims, mass, U, X, sigma=sigma)
    try:
        for mode in (1, 2, 3, 4):
            for R in (1, 2, 4):
                if n % R:
                    continue
                lib.rhmc_tune_set(8, mode)
                lib.rhmc_tune_set(0, R)
                for par in (0, 1):
                    got = ctx.hop(to_gpu(X), par, "fp32").cpu().numpy()
                    assert colrel(got, refs[par]) <= 1e-6, (mode, R, par)
                got = ctx.apply_mdagm_mrhs(to_gpu(X), sigma, "fp32").cpu().numpy()
                assert colrel(got, refA) <= 1e-6, (mode, R)
    finally:
        lib.rhmc_tune_set(8, 0)
        lib.rhmc_tune_set(0, 0)
    ctx.close()


def test_apply_full_size_sampled():
    """24^4, n = 16 (the force workload's launch configuration): sampled even sites against the oracle."""
    need_gpu()
    dims, mass, n = (24, 24, 24, 24), 0.01, 16
    U = syn.random_links(dims, 0.5, syn.seed_gauge(3))
    X = syn.gaussian_pseudofermions(dims, n, syn.seed_phi(3))
    ctx = make_ctx(dims, mass, U)
    rng = np.random.default_rng(0)
    sites = np.concatenate([[0, 1, ctx.Vh - 1], rng.integers(0, ctx.Vh, 61)])
    ref = oracle.apply_A_at(dims, mass, U, X, sites)
    got = ctx.apply_mdagm_mrhs(to_gpu(X), 0.0, "fp64").cpu().numpy()[sites]
    assert colrel(got, ref) <= 1e-12
    got32 = ctx.apply_mdagm_mrhs(to_gpu(X), 0.0, "fp32").cpu().numpy()[sites]
    assert colrel(got32, ref) <= 1e-6
    gotdf = ctx.apply_mdagm_mrhs(to_gpu(X), 0.0, "df64").cpu().numpy()[sites]
    assert colrel(gotdf, ref) <= 1e-12
    ctx.close()


def test_free_field_eigenvector_gpu():
    """Property at any size: an even-projected plane wave is an eigenvector with the closed-form eigenvalue."""
    need_gpu()
    dims, mass = (16, 16, 16, 32), 0.02
    from oracle import dense

    lex = dense.parity_lex(dims, 0)
    x, y, z, t = lex % 16, (lex // 16) % 16, (lex // 256) % 16, lex // 4096
    p = np.array([2 * np.pi * 3 / 16, 2 * np.pi * 5 / 16, 2 * np.pi / 16, 7 * np.pi / 32])
    X = np.zeros((len(lex), 3, 2), dtype=np.complex128)
    X[:, 0, 0] = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    X[:, 2, 1] = X[:, 0, 0]
    ctx = make_ctx(dims, mass, syn.unit_links(dims))
    got = ctx.apply_mdagm_mrhs(to_gpu(X), 0.0, "fp64").cpu().numpy()
    lam = 4 * mass ** 2 + 4 * np.sum(np.sin(p) ** 2)
    assert np.abs(got - lam * X).max() <= 1e-12 * lam
    ctx.close()


def test_errors_are_reported():
    torch = need_gpu()
    from paper_1808_01829_gb300._lib import RhmcError

    dims = (4, 4, 4, 4)
    from paper_1808_01829_gb300.api import RhmcContext

    ctx = RhmcContext(dims, 0.1)
    X = to_gpu(syn.gaussian_pseudofermions(dims, 2, 1))
    with pytest.raises(RhmcError, match="NO_GAUGE"):
        ctx.apply_mdagm_mrhs(X)
    ctx.set_gauge(to_gpu(syn.unit_links(dims)))
    with pytest.raises(RhmcError, match="INVALID_ARG"):
        ctx.block_multishift_cg(X, [0.1, -1.0], 1e-8)
    with pytest.raises(ValueError):
        ctx.apply_mdagm_mrhs(X.to(torch.complex64))
    ctx.close()


@pytest.mark.parametrize("bc", [-1, 1])
def test_fp32_hop_12_real_links(bc):
    """SU(3) links: the FP32 hop reading two rows per link and rebuilding the third
    (with the staggered phase and boundary sign) agrees with the full records and the
    oracle; links off SU(3) must not take that path."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n, sigma = (4, 6, 4, 8), 0.05, 16, 0.13
    X = syn.gaussian_pseudofermions(dims, n, 2104)
    for scale in (1.0, 1.05):
        U = syn.random_links(dims, 0.5, 1104) * scale
        ref = oracle.apply_A(dims, mass, U, X, sigma=sigma, bc_t=bc)
        ctx = make_ctx(dims, mass, U, bc)
        try:
            for mode in (1, 0):
                lib.rhmc_tune_set(10, mode)
                got = ctx.apply_mdagm_mrhs(to_gpu(X), sigma, "fp32").cpu().numpy()
                assert colrel(got, ref) <= 1e-6, (scale, mode)
        finally:
            lib.rhmc_tune_set(10, 0)
        ctx.close()
