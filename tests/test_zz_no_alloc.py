"""rhmc_apply_mdagm_mrhs_noalloc: the allocation-free FP64 operator application.

It exists for callers that cannot allocate device memory at call time (stream
capture, fixed memory budgets, frameworks that own allocation).  Through the
C ABI it must agree with rhmc_apply_mdagm_mrhs (FP64) and with the oracle's
operator to the tolerance of the other GPU tests (1e-12 relative per column),
on two calls in a row, and reject problems larger than its fixed scratch with INVALID_ARG.
This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest

import oracle

from gpu_util import colrel, need_gpu

pytestmark = pytest.mark.gpu


def _ctx(lib, dims, mass):
    from paper_1808_01829_gb300 import _lib

    h = ctypes.c_void_p()
    lat = _lib.Lattice((ctypes.c_int * 4)(*dims), mass, -1)
    assert lib.rhmc_create(ctypes.byref(h), ctypes.byref(lat), 0) == 0
    return h


def test_noalloc_matches_apply_mdagm_twice():
    torch = need_gpu()
    from paper_1808_01829_gb300 import _build, _lib
    from paper_1808_01829_gb300 import synthetic as syn

    _build.build()
    lib = _lib.load()
    dims, mass, n = (8, 4, 6, 8), 0.05, 5
    h = _ctx(lib, dims, mass)
    U = torch.from_numpy(syn.random_links(dims, 0.5, 1300)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rhmc_set_gauge(h, ctypes.c_void_p(U.data_ptr()), stream) == 0
    for call, sigma in enumerate((0.0, 0.21)):
        X = torch.from_numpy(syn.gaussian_pseudofermions(dims, n, 2300 + call)).cuda()
        Yref = torch.empty_like(X)
        Y = torch.full_like(X, float("nan"))
        rc = lib.rhmc_apply_mdagm_mrhs(h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Yref.data_ptr()), n,
                                       sigma, _lib.RHMC_FP64, stream)
        assert rc == 0
        rc = lib.rhmc_apply_mdagm_mrhs_noalloc(h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n,
                                               sigma, stream)
        assert rc == 0, lib.rhmc_last_error()
        torch.cuda.synchronize()
        assert colrel(Y.cpu().numpy(), Yref.cpu().numpy()) <= 1e-12
        # and directly against the FP64 oracle's (A + sigma) X
        Yo = oracle.apply_A(dims, mass, U.cpu().numpy(), X.cpu().numpy(), sigma=sigma)
        assert colrel(Y.cpu().numpy(), Yo) <= 1e-12
    lib.rhmc_destroy(h)


def test_noalloc_rejects_oversize_and_missing_gauge():
    torch = need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 16^3 x 32 with 16 right-hand sides needs 50 MB of scratch: above the fixed 32 MiB
    dims, n = (16, 16, 16, 32), 16
    h = _ctx(lib, dims, 0.02)
    X = torch.zeros((16 * 16 * 16 * 16, 3, n), dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    rc = lib.rhmc_apply_mdagm_mrhs_noalloc(h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n, 0.0,
                                           stream)
    assert rc == 6  # gauge not set yet
    from paper_1808_01829_gb300 import synthetic as syn

    U = torch.from_numpy(syn.unit_links(dims)).cuda()
    assert lib.rhmc_set_gauge(h, ctypes.c_void_p(U.data_ptr()), stream) == 0
    rc = lib.rhmc_apply_mdagm_mrhs_noalloc(h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n, 0.0,
                                           stream)
    assert rc == 1 and b"scratch" in lib.rhmc_last_error()
    # within the limit (n = 8: 25 MB) it runs
    X8 = torch.zeros((16 * 16 * 16 * 16, 3, 8), dtype=torch.complex128, device="cuda")
    Y8 = torch.empty_like(X8)
    rc = lib.rhmc_apply_mdagm_mrhs_noalloc(h, ctypes.c_void_p(X8.data_ptr()), ctypes.c_void_p(Y8.data_ptr()), 8, 0.0,
                                           stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert float(Y8.abs().max()) == 0.0
    lib.rhmc_destroy(h)
