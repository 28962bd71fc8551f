"""The FP64 reciprocal and square-root helpers of the n x n coefficient step
(Newton-Raphson refinement of an FP32 estimate; Algorithm 1's alpha_k, rho_k and
shifted coefficients use them) against CUDA's IEEE 1.0 / x and sqrt, and against
numpy's correctly rounded results, over a log-spaced sweep of 1e-300 .. 1e300 that
takes both the frexp-scaled branch and the direct FP32-range branch.  Bound: 2
units in the last place (the Newton steps square the 2^-23 estimate's error twice
and round once more)."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def test_fp64_helpers_within_two_ulps():
    torch = need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    rng = np.random.default_rng(31)
    x = np.concatenate([np.logspace(-300, 300, 60001), rng.uniform(0.5, 2.0, 4000),
                        np.array([1.0, 2.0, 0.5, 3.0, 1e-30, 1e30, 0.9999999999999999, 1.0000000000000002])])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(6 * x.size, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rhmc_selftest_fp64_helpers(ctypes.c_void_p(xd.data_ptr()), x.size, ctypes.c_void_p(out.data_ptr()),
                                          stream) == 0
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(6, x.size)
    rcp, sq, rcp_fast, rsq, ieee_rcp, ieee_sqrt = o
    # CUDA's IEEE results are the correctly rounded ones
    assert np.array_equal(ieee_rcp, 1.0 / x) and np.array_equal(ieee_sqrt, np.sqrt(x))
    worst = {"frcp": _ulps(rcp, ieee_rcp).max(), "fsqrt": _ulps(sq, ieee_sqrt).max(),
             "frcp_fast": _ulps(rcp_fast, ieee_rcp).max(), "frsqrt": _ulps(rsq, (1 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)).max()}
    print("\nmax ulp error:", {k: float(v) for k, v in worst.items()})
    for name, v in worst.items():
        assert v <= 2.0, (name, v)
