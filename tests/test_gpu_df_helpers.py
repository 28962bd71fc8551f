"""The double-float arithmetic of the mixed solve (a value is an unevaluated pair of
floats hi + lo; products by the FMA-based TwoProduct of Ogita, Rump and Oishi 2005, sums
by Knuth's TwoSum).  The FP64-accurate residuals and force and the base n x n steps run
on it, so it is pinned here directly:

- the split of a double is exact: hi = RN_float(x) and lo = RN_float(x - hi), bit for bit
  against numpy's float32 rounding, including ties to even and a mantissa that rounds up
  into the next binade;
- hi + lo recovers x to 2^-47 relative (lo keeps 24 of the 29 remaining bits);
- a + b within 2^-44 (|a| + |b|), a b within 2^-44 |a b|, the running sum a b + b b
  within 2^-44 (|a b| + b^2);
- 1 / a within 2^-43 (one Newton step on the correctly rounded FP32 reciprocal: 2^-46,
  plus the low parts) and 1 / sqrt(a) within 2^-42 (one Newton step on an FP32 estimate
  of relative error e <= 2^-22 leaves (3/2) e^2 < 2^-43.4, plus rounding).
References in numpy's extended precision.  Magnitudes 2^-30 .. 2^30, random signs."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(47)
    m = 100000
    x = np.exp2(rng.uniform(-30, 30, m)) * rng.choice([-1.0, 1.0], m)
    y = np.exp2(rng.uniform(-30, 30, m)) * rng.choice([-1.0, 1.0], m)
    u = 2.0 ** -24
    special = np.array([1.0, 0.5, 3.0, 0.1, 1 + u, 1 + 3 * u, -(1 + u), 1 + u + 2.0 ** -52, 1 - 2.0 ** -25,
                        2.0 ** 24 + 1, 2 - 2.0 ** -30, -(2 - 2.0 ** -30), 1.5 + u, 1.5 + 3 * u, 2.0 ** 29 - 1])
    x = np.concatenate([special, x, -y[:1000]])  # -y: sums that cancel
    y = np.concatenate([special[::-1], y, y[:1000] * (1 + 2.0 ** -40)])
    return x, y


def test_double_float_helpers_exact_split_and_bounds():
    torch = need_gpu()
    from paper_1808_01829_gb300 import _lib

    lib = _lib.load()
    x, y = _inputs()
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.empty(8 * x.size, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rhmc_selftest_df_helpers(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), x.size,
                                        ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    hi, lo, merged, add, mul, rcp, rsq, acc = out.cpu().numpy().reshape(8, x.size)
    # the split, bit for bit
    hi_ref = x.astype(np.float32).astype(np.float64)
    lo_ref = (x - hi_ref).astype(np.float32).astype(np.float64)  # x - hi_ref is exact in FP64
    assert np.array_equal(hi, hi_ref)
    assert np.array_equal(lo, lo_ref)
    X, Y = x.astype(np.longdouble), y.astype(np.longdouble)

    def rel(got, want, scale):
        return float(np.max(np.abs(got.astype(np.longdouble) - want) / scale))

    worst = {
        "merge": rel(merged, X, np.abs(X)) / 2.0 ** -47,
        "add": rel(add, X + Y, np.abs(X) + np.abs(Y)) / 2.0 ** -44,
        "mul": rel(mul, X * Y, np.abs(X * Y)) / 2.0 ** -44,
        "running sum": rel(acc, X * Y + Y * Y, np.abs(X * Y) + Y * Y) / 2.0 ** -44,
        "rcp": rel(rcp, 1 / X, np.abs(1 / X)) / 2.0 ** -43,
    }
    pos = x > 0
    worst["rsqrt"] = rel(rsq[pos], 1 / np.sqrt(X[pos]), 1 / np.sqrt(X[pos])) / 2.0 ** -42
    print("\nworst error / bound:", worst)
    for name, v in worst.items():
        assert v <= 1.0, (name, v)
    assert np.all(rsq[~pos] == 0.0)
