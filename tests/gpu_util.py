"""Helpers for the GPU parity tests (test infrastructure)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def colrel(a, b):
    """Per-column relative error of blocks (..., n): max over columns of ||a-b|| / ||b||."""
    a = np.asarray(a).reshape(-1, a.shape[-1])
    b = np.asarray(b).reshape(-1, b.shape[-1])
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def make_ctx(dims, mass, U, bc_t=-1):
    torch = need_gpu()
    from paper_1808_01829_gb300.api import RhmcContext

    ctx = RhmcContext(dims, mass, bc_t=bc_t, device=0)
    ctx.set_gauge(torch.from_numpy(np.ascontiguousarray(U)).cuda())
    return ctx


def to_gpu(a):
    torch = need_gpu()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_solution(dims, mass, U, B, shifts, Xg, tol, Xo=None):
    """Parity of shifted solutions (criteria of the solver tests).

    For every (shift, column): the FP64 true residual ||B e_j - (A + sigma_s) X e_j|| / ||B e_j||,
    with A applied by the oracle, is <= tol.  With the oracle's own solution Xo (solved to
    1e-13) also ||X_gpu - X_orc|| <= tol ||B e_j|| / (4m^2 + sigma_s) + 1e-10 ||X_orc e_j||,
    the error a residual tol allows since lambda_min(A) >= 4m^2.  Returns the largest ratios
    (residual / tol, error / bound) so that callers can report them."""
    import oracle

    bn = np.linalg.norm(B.reshape(-1, B.shape[-1]), axis=0)
    worst_r, worst_e = 0.0, 0.0
    for s, sig in enumerate(shifts):
        R = B - oracle.apply_A(dims, mass, U, Xg[s], sigma=sig)
        rn = np.linalg.norm(R.reshape(-1, B.shape[-1]), axis=0) / bn
        assert np.all(rn <= tol), (s, sig, rn)
        worst_r = max(worst_r, float(np.max(rn)) / tol)
        if Xo is not None:
            err = np.linalg.norm((Xg[s] - Xo[s]).reshape(-1, B.shape[-1]), axis=0)
            xn = np.linalg.norm(Xo[s].reshape(-1, B.shape[-1]), axis=0)
            bound = tol * bn / (4 * mass ** 2 + sig) + 1e-10 * xn
            assert np.all(err <= bound), (s, sig, err / bound)
            worst_e = max(worst_e, float(np.max(err / bound)))
    return worst_r, worst_e


def force_bound(mass, Phi, beta, Xo, tol):
    """Relative force error a solve to tol allows: 2 max_s tol ||Phi|| / ((4m^2 + beta_s) ||X^(s)||) + 1e-10."""
    bn = np.linalg.norm(Phi)
    return 2 * max(tol * bn / ((4 * mass ** 2 + b) * np.linalg.norm(Xo[s])) for s, b in enumerate(beta)) + 1e-10


def sample_links(dims, count, seed):
    """count (lex, mu) link indices: every direction, the t = Lt-1 -> 0 boundary links
    (antiperiodic sign), the x = Lx-1 wrap and random bulk links."""
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)

    def lex(x, y, z, t):
        return x + lx * (y + ly * (z + lz * t))

    out = []
    for mu in range(4):  # corners and boundary planes
        out.append((lex(lx - 1, ly - 1, lz - 1, lt - 1), mu))
        out.append((lex(0, 0, 0, 0), mu))
    for k in range(8):  # t boundary, both parities
        out.append((lex(k % lx, (3 * k) % ly, (5 * k) % lz, lt - 1), 3))
        out.append((lex((k + 1) % lx, (3 * k) % ly, (5 * k) % lz, 0), 3))
    for k in range(4):
        out.append((lex(lx - 1, k % ly, (2 * k) % lz, (3 * k) % lt), 0))
    V = lx * ly * lz * lt
    while len(out) < count:
        out.append((int(rng.integers(V)), int(rng.integers(4))))
    return np.asarray(out[:count], dtype=np.int64)
