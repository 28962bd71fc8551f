"""Convergence and force-norm studies on synthetic fields (analogues of the
paper's Figs. 1 and 2 and of its force-norm cost estimates, Sec. II).

    python -m paper_1808_01829_gb300.studies iterations [--dims 16 16 16 16] [--masses 0.01 0.02 0.05]
    python -m paper_1808_01829_gb300.studies residuals  [--dims 16 16 16 16] [--mass 0.01]
    python -m paper_1808_01829_gb300.studies force-norm [--dims 12 12 12 12] [--mass 0.05]

Every study prints a markdown table.

* ``iterations`` (Fig. 1): for n_pf = 1, 2, 4, 8, 16 Gaussian pseudofermions
  and the rational approximation of x^(-1/(4 n_pf)), it solves
  (A + beta_s) X = Phi to a relative residual of 1e-8 with the block
  multishift solve SBCGrQ (FP64) and with per-vector multishift CG (FP64).
  It reports:
  - the block iterations, and the per-vector iterations summed over the columns;
  - the ratio of operator applications per column, n_pf x block iterations
    against the per-vector sum;
  - the times.

  The block Krylov space of n_pf columns converges in fewer iterations as
  n_pf grows (Sec. III).
* ``residuals`` (Fig. 2): for n_pf = 1, 4, 16 it takes the FP64 true residual
  of every shifted system, max over the columns, against the shift sigma, at
  two stopping points:
  - after a fixed number of iterations;
  - at the iteration where the unshifted (smallest-shift) system reaches
    1e-7.

  No defect correction runs (RHMC_TUNE_NO_DEFECT_CORRECTION).  Larger n_pf
  lowers the small-shift residuals at a fixed k, and raises the large-shift
  ones at a fixed unshifted residual, because fewer iterations are run.
* ``force-norm`` (Sec. II, Eqs. (force_norm), (cost), (cost_clark)): on
  several synthetic gauge fields, and for each n_pf, it draws pseudofermions by
  the heatbath phi = A^(1/(8 n_pf)) eta, using the rational approximation of
  x^(+1/(8 n_pf)) through rhmc_rational_solve.  It then forms the force of the
  x^(-1/(4 n_pf)) action (rhmc_force) and its norm F^2 = sum_{x,mu,a}
  (F^a)^2 / 2 (rhmc_force_lie).  It reports:
  - the mean and variance of F^2;
  - the fit F^2 = c0 + c1 / n_pf;
  - the relative cost estimates n_pf var(F^2)^(1/4) and n_pf^2 kappa^(1/n_pf).

  kappa is taken as the spectral bound (4m^2 + 64) / 4m^2 of A.
"""
from __future__ import annotations

import argparse
import math
import time


def _ctx(dims, mass, seed):
    import torch

    from . import synthetic as syn
    from .api import RhmcContext

    ctx = RhmcContext(dims, mass)
    U = torch.from_numpy(syn.random_links(dims, 0.5, syn.seed_gauge(seed))).cuda()
    ctx.set_gauge(U)
    return ctx, U


def _phi(dims, n, seed):
    import torch

    from . import synthetic as syn

    return torch.from_numpy(syn.gaussian_pseudofermions(dims, n, syn.seed_phi(seed))).cuda()


def _force_approx(n, mass):
    from .remez import rational_approx

    if 4 * mass * mass >= 2e-3:
        return rational_approx(-1.0 / (4 * n), 2e-3, 64.0, 12)
    return rational_approx(-1.0 / (4 * n), 4e-4, 64.0, 16)


def iterations(a):
    import torch

    print(f"lattice {'x'.join(map(str, a.dims))}, links exp(i 0.5 H), tol {a.tol:g}, FP64")
    print("| m | n_pf | shifts | block iters | per-vector iters (sum) | per-column work ratio | block s | per-vector s |")
    print("|---|---|---|---|---|---|---|---|")
    for m in a.masses:
        ctx, _ = _ctx(a.dims, m, 20)
        for n in a.npf:
            ra = _force_approx(n, m)
            Phi = _phi(a.dims, n, 20 + n)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, ib = ctx.block_multishift_cg(Phi, ra.beta, a.tol, precision="fp64")
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, iv = ctx.multishift_cg_pervector(Phi, ra.beta, a.tol)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            ratio = n * ib.iters / max(iv.iters, 1)
            print(f"| {m:g} | {n} | {len(ra.beta)} | {ib.iters} | {iv.iters} | {ratio:.3f} | {t1 - t0:.2f} | "
                  f"{t2 - t1:.2f} |", flush=True)
        ctx.close()


def residuals(a):
    import numpy as np

    from . import _lib

    ctx, _ = _ctx(a.dims, a.mass, 21)
    ra = _force_approx(16, a.mass)  # the shifts of the 16-pseudofermion approximation, for every n_pf
    sig = list(ra.beta)
    ctx.tune_set(_lib.RHMC_TUNE_NO_DEFECT_CORRECTION, 1)
    cols = {}
    for n in a.npf:
        Phi = _phi(a.dims, n, 40 + n)
        # iteration at which the unshifted system alone reaches 1e-7
        _, ib = ctx.block_multishift_cg(Phi, [sig[0]], a.base_tol, precision="fp64", allow_not_converged=True)
        kb = ib.iters
        res = {}
        for label, k in (("k", a.k), ("base", kb)):
            _, info = ctx.block_multishift_cg(Phi, sig, 1e-15, max_iter=k, precision="fp64",
                                              allow_not_converged=True)
            r = np.asarray(info.per_shift_resid).reshape(len(sig), n)
            res[label] = (info.iters, r.max(axis=1))
        cols[n] = res
    ctx.tune_set(_lib.RHMC_TUNE_NO_DEFECT_CORRECTION, 0)
    ctx.close()
    print(f"lattice {'x'.join(map(str, a.dims))}, m {a.mass:g}, links exp(i 0.5 H), FP64, no defect correction; "
          f"max over columns of the true relative residual of (A + sigma) X = Phi")
    hdr = " | ".join(f"n_pf={n}, k={cols[n]['k'][0]}" for n in a.npf) + " | " + \
        " | ".join(f"n_pf={n}, base 1e-7 (k={cols[n]['base'][0]})" for n in a.npf)
    print(f"| sigma | {hdr} |")
    print("|---|" + "---|" * (2 * len(a.npf)))
    for s, sv in enumerate(sig):
        cells = [f"{cols[n]['k'][1][s]:.2e}" for n in a.npf] + [f"{cols[n]['base'][1][s]:.2e}" for n in a.npf]
        print(f"| {sv:.3e} | " + " | ".join(cells) + " |", flush=True)


def force_norm(a):
    import numpy as np
    import torch

    from .remez import rational_approx

    lo = 2e-3
    if 4 * a.mass * a.mass < lo:
        raise SystemExit("force-norm: 4 m^2 must be at least 2e-3 (the cached approximations' lower end)")
    V = math.prod(a.dims)
    kappa = (4 * a.mass ** 2 + 64.0) / (4 * a.mass ** 2)
    rows = []
    ctxs = [_ctx(a.dims, a.mass, 60 + c) for c in range(a.configs)]
    for n in a.npf:
        hb = rational_approx(1.0 / (8 * n), lo, 64.0, 12)      # phi = A^(1/(8 n)) eta
        fa = rational_approx(-1.0 / (4 * n), lo, 64.0, 12)     # S = phi^dagger A^(-1/(4 n)) phi
        vals = []
        for c, (ctx, U) in enumerate(ctxs):
            Uv = U.reshape(V, 4, 3, 3)
            for d in range(a.draws):
                eta = _phi(a.dims, n, 1000 * (c + 1) + 100 * d + n)
                phi, _ = ctx.rational_solve(eta, hb.alpha0, hb.alpha, hb.beta, a.tol)
                G, _, _ = ctx.force(phi, fa.alpha0, fa.alpha, fa.beta, a.tol, precision="mixed")
                _, f2 = ctx.force_lie(Uv, G, want_F=False)
                vals.append(f2 / (4 * V))  # per link
        v = np.asarray(vals)
        rows.append((n, v.mean(), v.var(ddof=1), v.std(ddof=1) / math.sqrt(len(v)), len(v)))
    for ctx, _ in ctxs:
        ctx.close()
    torch.cuda.synchronize()
    ns = np.array([r[0] for r in rows], dtype=float)
    mean = np.array([r[1] for r in rows])
    err = np.array([r[3] for r in rows])
    # weighted least squares F^2 = c0 + c1 / n_pf
    Amat = np.stack([np.ones_like(ns), 1.0 / ns], axis=1) / err[:, None]
    c0, c1 = np.linalg.lstsq(Amat, mean / err, rcond=None)[0]
    cost1 = ns * np.array([r[2] for r in rows]) ** 0.25
    cost2 = ns ** 2 * kappa ** (1.0 / ns)
    print(f"lattice {'x'.join(map(str, a.dims))}, m {a.mass:g}, {a.configs} gauge fields (links exp(i 0.5 H)) x "
          f"{a.draws} heatbath draws; F^2 per link; kappa = {kappa:.0f}")
    print("| n_pf | samples | mean F^2 | var F^2 | fit c0 + c1/n_pf | cost n_pf var^(1/4) (rel.) | "
          "cost n_pf^2 kappa^(1/n_pf) (rel.) |")
    print("|---|---|---|---|---|---|---|")
    for i, (n, m, var, e, cnt) in enumerate(rows):
        print(f"| {n} | {cnt} | {m:.6g} ± {e:.2g} | {var:.3e} | {c0 + c1 / n:.6g} | {cost1[i] / cost1[0]:.3f} | "
              f"{cost2[i] / cost2[0]:.4f} |", flush=True)
    print(f"fit: c0 = {c0:.6g}, c1 = {c1:.6g}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="study")
    p1 = sub.add_parser("iterations", help="Fig. 1: block vs per-vector iterations over n_pf and mass")
    p1.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 16])
    p1.add_argument("--masses", type=float, nargs="+", default=[0.01, 0.02, 0.05])
    p1.add_argument("--npf", type=int, nargs="+", default=[1, 2, 4, 8, 16])
    p1.add_argument("--tol", type=float, default=1e-8)
    p2 = sub.add_parser("residuals", help="Fig. 2: shifted residuals against sigma")
    p2.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 16])
    p2.add_argument("--mass", type=float, default=0.01)
    p2.add_argument("--npf", type=int, nargs="+", default=[1, 4, 16])
    p2.add_argument("--k", type=int, default=120, help="fixed iteration count (a multiple of 6)")
    p2.add_argument("--base-tol", type=float, default=1e-7)
    p3 = sub.add_parser("force-norm", help="force norm F^2 and cost estimates over n_pf")
    p3.add_argument("--dims", type=int, nargs=4, default=[12, 12, 12, 12])
    p3.add_argument("--mass", type=float, default=0.05)
    p3.add_argument("--npf", type=int, nargs="+", default=[1, 2, 4, 8, 16])
    p3.add_argument("--configs", type=int, default=4)
    p3.add_argument("--draws", type=int, default=8)
    p3.add_argument("--tol", type=float, default=1e-10)
    a = ap.parse_args(argv)
    if a.study is None:
        a = ap.parse_args(["iterations"] + (argv or []))
    {"iterations": iterations, "residuals": residuals, "force-norm": force_norm}[a.study](a)


if __name__ == "__main__":
    main()
