"""Failure detection without a GPU fault: a bounded device-side wait that
nothing completes gives up after its time limit, the host reads the timeout
status, and the CUDA context stays usable."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from gpu_util import colrel, make_ctx, need_gpu, to_gpu
from paper_1808_01829_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    torch = need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.time()
    rc = lib.rhmc_selftest_bounded_wait(0, 0.2, stream)
    dt = time.time() - t0
    assert rc == 5, lib.rhmc_last_error()  # RHMC_ERR_DEVICE_TIMEOUT
    assert b"bounded device wait expired" in lib.rhmc_last_error()
    assert 0.1 < dt < 10.0
    assert lib.rhmc_selftest_bounded_wait(0, 3.0, stream) == 1  # limit out of range: INVALID_ARG
    # the context is intact: an operator application still matches the oracle
    dims, mass, n = (4, 4, 4, 4), 0.1, 3
    U = syn.random_links(dims, 0.3, 1270)
    X = syn.gaussian_pseudofermions(dims, n, 2270)
    ctx = make_ctx(dims, mass, U)
    got = ctx.apply_mdagm_mrhs(to_gpu(X), 0.0, "fp64").cpu().numpy()
    assert colrel(got, oracle.apply_A(dims, mass, U, X)) <= 1e-12
    ctx.close()
