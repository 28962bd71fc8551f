"""A bounded solve for profiler captures.

    python -m paper_1808_01829_gb300.profile_case --dims 16 16 16 32 --n 16 --shifts 16 --iters 24

sets up one synthetic ensemble (links exp(i 0.5 H), Gaussian pseudofermions),
a rational approximation (16 shifts: x^(-1/64) on [4e-4, 64]; otherwise
x^(-1/(4n)) on [2e-3, 64], from the coefficient cache) and runs the block
multishift solve `--repeat` times with at most `--iters` iterations each, so
that a kernel profiler can capture launches of the solver's kernels on a
workload whose fields are larger than L2 but whose device footprint stays at
a few GB.  It prints the solver statistics of the last solve and times
nothing.
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--mass", type=float, default=0.01)
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--shifts", type=int, default=16)
    ap.add_argument("--iters", type=int, default=24)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                    help="rhmc_tune_set(KEY, VALUE) before the solves (repeatable)")
    a = ap.parse_args(argv)

    import torch

    from . import _lib
    from . import synthetic as syn
    from .api import RhmcContext
    from .remez import rational_approx

    ra = rational_approx(-1.0 / 64, 4e-4, 64.0, 16) if a.shifts == 16 else None
    if ra is None:
        ra = rational_approx(-1.0 / (4 * a.n), 2e-3, 64.0, a.shifts)
    for kv in a.tune:
        k, v = kv.split("=")
        _lib.check(_lib.load().rhmc_tune_set(int(k), int(v)), "rhmc_tune_set")
    ctx = RhmcContext(a.dims, a.mass)
    ctx.set_gauge(torch.from_numpy(syn.random_links(a.dims, 0.5, syn.seed_gauge(3))).cuda())
    B = torch.from_numpy(syn.gaussian_pseudofermions(a.dims, a.n, syn.seed_phi(3))).cuda()
    info = None
    for _ in range(a.repeat):
        _, info = ctx.block_multishift_cg(B, ra.beta, a.tol, max_iter=a.iters, precision=a.precision,
                                          allow_not_converged=True)
    torch.cuda.synchronize()
    print(f"dims {a.dims} n {a.n} shifts {len(ra.beta)} iters {info.iters} dirac_calls {info.dirac_calls} "
          f"true_rel_resid_max {info.true_rel_resid_max:.3e}")
    ctx.close()


if __name__ == "__main__":
    main()
