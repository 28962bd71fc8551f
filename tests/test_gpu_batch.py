"""Batched ensembles (rhmc_block_multishift_cg_batch) and captured-graph solves:
every member of a batch of uneven lattices, widths and shift sets matches the
oracle as a standalone solve does; graph and eager execution agree; the
autotuner leaves results unchanged."""
import numpy as np
import pytest

import oracle
from gpu_util import make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn
from paper_1808_01829_gb300.remez import rational_approx
from test_gpu_solver import _check_solution

pytestmark = pytest.mark.gpu

MEMBERS = [
    ((4, 4, 4, 4), 0.1, 2, (-1.0 / 8, 1e-3, 64.0, 8)),
    ((6, 6, 4, 4), 0.05, 4, (-1.0 / 16, 2e-3, 64.0, 12)),
    ((4, 4, 4, 8), 0.05, 8, (-1.0 / 32, 2e-3, 64.0, 12)),
    ((8, 4, 4, 4), 0.05, 12, (-1.0 / 48, 2e-3, 64.0, 12)),
]


def test_batch_members_match_oracle():
    need_gpu()
    from paper_1808_01829_gb300.api import block_multishift_cg_batch

    items, refs = [], []
    for k, (dims, mass, n, rp) in enumerate(MEMBERS):
        ra = rational_approx(*rp)
        U = syn.random_links(dims, 0.5, 1500 + k)
        B = syn.gaussian_pseudofermions(dims, n, 2500 + k)
        ctx = make_ctx(dims, mass, U)
        items.append((ctx, to_gpu(B), ra.beta))
        refs.append((dims, mass, U, B, ra.beta))
    out = block_multishift_cg_batch(items, 1e-9, precision="mixed")
    for (X, info), (dims, mass, U, B, shifts) in zip(out, refs):
        assert info.true_rel_resid_max <= 1e-9
        Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, shifts, tol=1e-13)
        _check_solution(dims, mass, U, B, shifts, X.cpu().numpy(), 1e-9, Xo)
    for ctx, _, _ in items:
        ctx.close()


def test_graph_and_eager_agree():
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n = (8, 8, 8, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1510)
    B = syn.gaussian_pseudofermions(dims, n, 2510)
    ctx = make_ctx(dims, mass, U)
    res = {}
    try:
        for mode in (2, 1, 1):  # eager, graph (capture), graph (replay)
            lib.rhmc_tune_set(7, mode)
            X, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-10, precision="fp64")
            res.setdefault(mode, []).append(X.cpu().numpy())
    finally:
        lib.rhmc_tune_set(7, 0)
    # the same kernels in the same order: identical results
    assert np.array_equal(res[2][0], res[1][0])
    assert np.array_equal(res[1][0], res[1][1])
    ctx.close()


def test_autotune_keeps_results(tmp_path):
    need_gpu()
    from paper_1808_01829_gb300 import autotune

    dims, mass, n = (8, 8, 4, 8), 0.05, 16
    ra = rational_approx(-1.0 / 64, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1520)
    B = to_gpu(syn.gaussian_pseudofermions(dims, n, 2520))
    ctx = make_ctx(dims, mass, U)
    try:
        X0, _ = ctx.block_multishift_cg(B, ra.beta, 1e-9, precision="mixed")
        settings = autotune.tune(ctx, n, shifts=ra.beta, cache=str(tmp_path / "tune.json"))
        assert set(settings) == {8, 19, 20}  # hop, base-step and Gram tiles
        X1, info = ctx.block_multishift_cg(B, ra.beta, 1e-9, precision="mixed")
        assert info.true_rel_resid_max <= 1e-9
        assert np.linalg.norm((X1 - X0).cpu().numpy()) <= 1e-6 * np.linalg.norm(X0.cpu().numpy())
        # applied to this context only; cached: a second call only applies
        assert all(ctx.tune_get(k) == v for k, v in settings.items())
        assert autotune.tune(ctx, n, cache=str(tmp_path / "tune.json")) == settings
    finally:
        autotune.reset(ctx)
    ctx.close()


def test_refinement_lanes_agree():
    """Defect corrections spread over concurrent lanes give bit-identical solutions to
    corrections run in turn (each shift's correction is the same deterministic kernels)."""
    need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    dims, mass, n = (8, 8, 8, 8), 0.05, 4
    ra = rational_approx(-1.0 / 16, 2e-3, 64.0, 12)
    U = syn.random_links(dims, 0.5, 1530)
    B = syn.gaussian_pseudofermions(dims, n, 2530)
    ctx = make_ctx(dims, mass, U)
    out = {}
    try:
        for lanes in (1, 4):
            lib.rhmc_tune_set(9, lanes)
            X, info = ctx.block_multishift_cg(to_gpu(B), ra.beta, 1e-10, precision="mixed")
            assert info.refinements > 0 and info.true_rel_resid_max <= 1e-10
            out[lanes] = X.cpu().numpy()
    finally:
        lib.rhmc_tune_set(9, 0)
    assert np.array_equal(out[1], out[4])
    Xo, _, _ = oracle.sbcgrq(dims, mass, U, B, ra.beta, tol=1e-13)
    _check_solution(dims, mass, U, B, ra.beta, out[4], 1e-10, Xo)
    ctx.close()
