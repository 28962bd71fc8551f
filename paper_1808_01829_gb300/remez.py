"""Rational approximation of x^r for the pseudofermion action, Eq. (RA).

    x^r  ~=  alpha_0 + sum_{j=1}^{N} alpha_j / (x + beta_j),   x in [a, b],

with alpha_j, beta_j > 0 (Sec. II).  The coefficients are those of the
minimax approximation of type (N, N) in the *relative* error |R(x)/x^r - 1|
(the paper bounds the relative error of its approximations, Sec. IV: below
1e-7 with about 15 shifts for the molecular-dynamics force, below 1e-15 with
about 30 for the heatbath and accept/reject steps).  It is found by a Remez
exchange in multiple precision (mpmath):

1. start from 2N+2 reference points spread like Chebyshev nodes in log x;
2. solve the levelled equations  p(x_i) - q(x_i) x_i^r (1 + (-1)^i E) = 0
   for the numerator p, the denominator q (normalised q_0 = 1) and the
   level E, by a fixed-point iteration on E (each step one linear solve);
3. locate the extrema of the relative error on a dense log grid, refine each
   by golden-section search, and take 2N+2 alternating ones as the new
   reference;
4. stop when the extrema's magnitudes agree to `equi_tol`;
5. turn p/q into partial fractions from the roots of q (poles -beta_j) and
   the residues alpha_j = p(-beta_j) / q'(-beta_j); alpha_0 is the ratio of
   leading coefficients.

This is host-side set-up; the solver receives (alpha_0, alpha_j, beta_j) as
plain numbers.  Results are cached in ``rational_coeffs.json`` next to this
file so that machines without mpmath can still look them up.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field
from typing import List

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rational_coeffs.json")


@dataclass
class RationalApprox:
    r: float
    a: float
    b: float
    alpha0: float
    alpha: List[float]
    beta: List[float]
    error: float  # max relative error on [a, b] (the levelled |E|)
    extrema: List[float] = field(default_factory=list)

    @property
    def nshift(self) -> int:
        return len(self.beta)

    def __call__(self, x):
        """Evaluate the partial-fraction form (float64)."""
        import numpy as np

        x = np.asarray(x, dtype=np.float64)
        out = np.full(x.shape, self.alpha0)
        for al, be in zip(self.alpha, self.beta):
            out = out + al / (x + be)
        return out

    def to_json(self):
        return {
            "r": self.r, "a": self.a, "b": self.b, "alpha0": self.alpha0, "alpha": self.alpha,
            "beta": self.beta, "error": self.error, "extrema": self.extrema,
        }


def _key(r, a, b, n):
    return f"r={float(r)!r};a={float(a)!r};b={float(b)!r};n={int(n)}"


def _load_cache():
    if os.path.exists(_CACHE):
        with open(_CACHE) as f:
            return json.load(f)
    return {}


def remez(r: float, a: float, b: float, n: int, equi_tol: float = 1e-4, max_iter: int = 60,
          dps: int | None = None, grid_per_interval: int = 64) -> RationalApprox:
    """Minimax relative-error rational approximation of type (n, n) to x^r on [a, b]."""
    import mpmath as mp

    if not (0 < a < b) or n < 1 or r == 0:
        raise ValueError("need 0 < a < b, n >= 1, r != 0")
    ctx = mp.mp.clone() if hasattr(mp.mp, "clone") else mp.mp
    ctx.dps = dps or (40 + 6 * n)
    mpf = ctx.mpf
    R_ = mpf(r)
    la, lb = ctx.log(mpf(a)), ctx.log(mpf(b))
    m = 2 * n + 2

    def f(x):
        return ctx.power(x, R_)

    # 1. Chebyshev-like start in log x
    xs = [ctx.exp(la + (lb - la) * (1 - ctx.cos(ctx.pi * i / (m - 1))) / 2) for i in range(m)]

    def solve_levelled(xs):
        E = mpf(0)
        q_old = [mpf(1)] + [mpf(0)] * n
        for _ in range(100):
            # unknowns: p_0..p_n, q_1..q_n, E    (q_0 = 1)
            A = ctx.matrix(m, m)
            rhs = ctx.matrix(m, 1)
            for i, x in enumerate(xs):
                fx = f(x)
                sgn = 1 if i % 2 == 0 else -1
                xp = mpf(1)
                for k in range(n + 1):
                    A[i, k] = xp
                    xp *= x
                xp = x
                for k in range(1, n + 1):
                    A[i, n + k] = -fx * xp
                    xp *= x
                qo = ctx.polyval(list(reversed(q_old)), x)
                A[i, 2 * n + 1] = -sgn * fx * qo
                rhs[i] = fx  # q_0 f term moved to the right
            sol = ctx.lu_solve(A, rhs)
            p = [sol[k] for k in range(n + 1)]
            q = [mpf(1)] + [sol[n + k] for k in range(1, n + 1)]
            E_new = sol[2 * n + 1]
            if abs(E_new - E) <= abs(E_new) * mpf(10) ** (-(ctx.dps // 2)):
                return p, q, E_new
            E, q_old = E_new, q
        return p, q, E_new

    def err(p, q, x):
        return ctx.polyval(list(reversed(p)), x) / (ctx.polyval(list(reversed(q)), x) * f(x)) - 1

    p = q = None
    E = mpf(0)
    ext = xs
    for it in range(max_iter):
        p, q, E = solve_levelled(xs)
        # 3. extrema of the relative error on a dense grid in log x, refined
        G = grid_per_interval * m
        lg = [la + (lb - la) * k / (G - 1) for k in range(G)]
        ev = [err(p, q, ctx.exp(t)) for t in lg]
        cand = []  # (t, value) local extrema including endpoints
        for k in range(G):
            left = ev[k - 1] if k > 0 else None
            right = ev[k + 1] if k < G - 1 else None
            v = ev[k]
            is_ext = True
            if left is not None and abs(left) > abs(v) and (left * v > 0):
                is_ext = False
            if right is not None and abs(right) > abs(v) and (right * v > 0):
                is_ext = False
            if is_ext:
                if 0 < k < G - 1:
                    # golden-section refinement of |err| on [lg[k-1], lg[k+1]]
                    lo, hi = lg[k - 1], lg[k + 1]
                    sgn = 1 if v > 0 else -1
                    gr = (ctx.sqrt(5) - 1) / 2
                    c1, c2 = hi - gr * (hi - lo), lo + gr * (hi - lo)
                    f1, f2 = sgn * err(p, q, ctx.exp(c1)), sgn * err(p, q, ctx.exp(c2))
                    for _ in range(60):
                        if f1 > f2:
                            hi, c2, f2 = c2, c1, f1
                            c1 = hi - gr * (hi - lo)
                            f1 = sgn * err(p, q, ctx.exp(c1))
                        else:
                            lo, c1, f1 = c1, c2, f2
                            c2 = lo + gr * (hi - lo)
                            f2 = sgn * err(p, q, ctx.exp(c2))
                    t = (lo + hi) / 2
                    cand.append((t, err(p, q, ctx.exp(t))))
                else:
                    cand.append((lg[k], v))
        # keep one extremum per sign run (the largest), in order
        runs = []
        for t, v in cand:
            if runs and (runs[-1][1] > 0) == (v > 0):
                if abs(v) > abs(runs[-1][1]):
                    runs[-1] = (t, v)
            else:
                runs.append((t, v))
        # trim to m points keeping alternation: drop the smaller end runs
        while len(runs) > m:
            if abs(runs[0][1]) < abs(runs[-1][1]):
                runs.pop(0)
            else:
                runs.pop()
        if len(runs) < m:
            raise RuntimeError(f"remez: found only {len(runs)} alternating extrema (need {m})")
        mags = [abs(v) for _, v in runs]
        ext = [ctx.exp(t) for t, _ in runs]
        spread = (max(mags) - min(mags)) / max(mags)
        xs = ext
        if spread < equi_tol:
            break
    else:
        raise RuntimeError("remez: no convergence")
    emax = max(mags)
    # 5. partial fractions
    qrev = list(reversed(q))  # highest degree first
    roots = ctx.polyroots(qrev, maxsteps=400, extraprec=4 * ctx.prec)
    betas, alphas = [], []
    dq = [qrev[k] * (n - k) for k in range(n)]  # derivative, highest first
    prev = list(reversed(p))
    for z in roots:
        if abs(ctx.im(z)) > abs(z) * mpf(10) ** (-(ctx.dps // 3)):
            raise RuntimeError("remez: complex pole")
        z = ctx.re(z)
        betas.append(-z)
        alphas.append(ctx.polyval(prev, z) / ctx.polyval(dq, z))
    order = sorted(range(n), key=lambda k: betas[k])
    betas = [betas[k] for k in order]
    alphas = [alphas[k] for k in order]
    alpha0 = p[n] / q[n]
    return RationalApprox(
        r=float(r), a=float(a), b=float(b), alpha0=float(alpha0),
        alpha=[float(v) for v in alphas], beta=[float(v) for v in betas], error=float(emax),
        extrema=[float(x) for x in ext],
    )


def rational_approx(r: float, a: float, b: float, n: int, write_cache: bool = False) -> RationalApprox:
    """Cached lookup of `remez(r, a, b, n)`; computes (needs mpmath) on a miss."""
    cache = _load_cache()
    k = _key(r, a, b, n)
    if k in cache:
        d = cache[k]
        return RationalApprox(**d)
    ra = remez(r, a, b, n)
    if write_cache:
        cache = _load_cache()
        cache[k] = ra.to_json()
        with open(_CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return ra


# Rational approximations used by the standard workloads: x^(-1/(4 n_pf)) on
# the stated spectral interval, with the stated number of shifts.
STANDARD = [
    (-1.0 / 8, 1e-3, 64.0, 8),     # 4^4,  n_pf = 2
    (-1.0 / 16, 2e-3, 64.0, 12),   # 8^4,  n_pf = 4
    (-1.0 / 32, 1e-3, 64.0, 14),   # 16^3 x 32, n_pf = 8
    (-1.0 / 64, 4e-4, 64.0, 16),   # 24^4, n_pf = 16
    (-1.0 / 8, 2e-3, 64.0, 12),    # batched ensemble, n_pf = 2
    (-1.0 / 32, 2e-3, 64.0, 12),   # batched ensemble, n_pf = 8
    (-1.0 / 48, 2e-3, 64.0, 12),   # batched ensemble, n_pf = 12
    (-1.0 / 64, 2e-3, 64.0, 12),   # batched ensemble, n_pf = 16
    (1.0 / 16, 1e-3, 64.0, 8),     # heatbath x^(+1/(8 n_pf)), 4^4, n_pf = 2
    (1.0 / 32, 2e-3, 64.0, 12),    # heatbath, 8^4, n_pf = 4
    # convergence study (studies.py): x^(-1/(4 n_pf)), n_pf = 1, 2, 4, 8, 16
    (-1.0 / 4, 2e-3, 64.0, 12),
    (-1.0 / 4, 4e-4, 64.0, 16),
    (-1.0 / 8, 4e-4, 64.0, 16),
    (-1.0 / 16, 4e-4, 64.0, 16),
    (-1.0 / 32, 4e-4, 64.0, 16),
    # force-norm study (studies.py): heatbath x^(+1/(8 n_pf)) on [2e-3, 64], n_pf = 1, 2, 8, 16
    (1.0 / 8, 2e-3, 64.0, 12),
    (1.0 / 16, 2e-3, 64.0, 12),
    (1.0 / 64, 2e-3, 64.0, 12),
    (1.0 / 128, 2e-3, 64.0, 12),
]


def main():  # pragma: no cover - cache writer
    import argparse

    ap = argparse.ArgumentParser(description="compute and cache the standard rational approximations")
    ap.add_argument("--write-cache", action="store_true")
    args = ap.parse_args()
    for r, a, b, n in STANDARD:
        ra = rational_approx(r, a, b, n, write_cache=args.write_cache)
        print(f"r={r:.6f} [{a},{b}] N={n}: error {ra.error:.3e}, beta_min {ra.beta[0]:.3e}, beta_max {ra.beta[-1]:.3e}")


if __name__ == "__main__":  # pragma: no cover
    main()
