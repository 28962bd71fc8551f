#!/usr/bin/env python3
"""Benchmark: time per pseudofermion-force evaluation at 24^4, n_pf = 16.

One step = one full force evaluation through the C ABI: the staging of the
resident FP64 links into the operator's FP32 and double-float records
(rhmc_set_gauge), then rhmc_force: the block multishift solve SBCGrQ
(Algorithm 1) of (A + beta_s) X^(s) = Phi for all 16 pseudofermions and all 16
shifts to a true relative residual of 1e-8 (mixed precision: FP32 operator and
block updates in an FP64 reliable-update / defect-correction loop), then the
force G of Eq. (force) in FP64.  Phi and U are resident on the device when the
timed region starts.

Also reported on the same line:
* e2e: the same step from host (pinned) U and Phi to G in host memory, copies
  inside the timed region;
* roofline: the multi-RHS FP32 hop at 24^4, n = 16 against the measured HBM peak;
* baseline_fp64_scg: plain per-vector FP64 multishift CG + the same force on
  this GPU (the comparison of the metric), median of 3 after a warm-up;
* same_precision: the block algorithm's own gain (Sec. IV.B, Fig. 9 analogue):
  FP64 block against FP64 per-vector, and mixed block (the timed step)
  against mixed per-vector (the same solver with one right-hand side per
  solve: multishift CG in the same reliable-update / defect-correction scheme);
* alu_peaks and roofline_alu: the measured FP32 / FP64 CUDA-core peaks and the
  fractions of them reached by the double-float operator (FP32-ALU bound), the
  FP64 operator of the per-vector baseline and the n x n coefficient chain;
* trajectory: time per RHMC trajectory (Sec. II set-up, Sec. IV parameters) on the
  paper's 8^4 lattice, the FP64 gauge kernels at 24^4 against the measured FP64
  peak, and the trajectory oracle on a bounded sample;
* cpu_baseline: the FP64 CPU oracle on the host cores, on a bounded sample.

--impl reference times the oracle (the only reference available: the paper
ships no code) on the same workload, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "24^4 staggered, m=0.01, n_pf=16, 16 shifts of x^(-1/64) on [4e-4,64], eps=0.5, tol 1e-8",
    "dims": [24, 24, 24, 24],
    "mass": 0.01,
    "n_pf": 16,
    "n_shifts": 16,
    "r": -1.0 / 64,
    "interval": [4e-4, 64.0],
    "eps": 0.5,
    "tol": 1e-8,
    "precision": "mixed",
    "index": 3,
}
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic
# byte of a kernel, from one capture on a smaller case of the same kernel
# (profiles/); the per-launch traffic of the bench's launches is scaled from it
# by the units processed.  A kernel changed since its capture has no entry.
TRAFFIC_RATIO = {
    "update_shifts_fp32": (0.843, "profiles/k_base_step_24x24x24x24_n16.md (24^4, the fused base step; writes still in "
                                  "L2 when the launch ends are not counted; scaled by bytes moved)"),
    "hop_fp32": (0.942, "profiles/k_hop_pf_traffic_24x24x24x24_n16.md (24^4, both hop kinds; scaled by bytes moved)"),
}
# SBCGrQ iterations of the bench workload (24^4, 16 x 16, tol 1e-8) measured with
# the library's FP64 path; the oracle runs the same recursion
REF_ITERS = 276
METRIC = "time/force eval at 24^4,n_pf=16 (1e-8 res): block+mixed vs FP64 CG; Dslash GB/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--small", action="store_true", help="8^4 n_pf=4 quick check (not a bench line)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the FP64 per-vector SCG comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble measurement")
    ap.add_argument("--no-traj", action="store_true", help="skip the RHMC trajectory measurement")
    ap.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                    help="rhmc_tune_set(KEY, VALUE) before the run (repeatable; recorded in config)")
    return ap.parse_args()


def dist_env():
    from paper_1808_01829_gb300 import replicas

    return replicas.env()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def make_inputs(cfg, n_override=None):
    from paper_1808_01829_gb300 import synthetic as syn
    from paper_1808_01829_gb300.remez import rational_approx

    dims = cfg["dims"]
    n = n_override or cfg["n_pf"]
    U = syn.random_links(dims, cfg["eps"], syn.seed_gauge(cfg["index"]))
    Phi = syn.gaussian_pseudofermions(dims, n, syn.seed_phi(cfg["index"]))
    ra = rational_approx(cfg["r"], cfg["interval"][0], cfg["interval"][1], cfg["n_shifts"])
    return U, Phi, ra


# ------------------------------------------------------------------ CPU oracle
def cpu_sample(cfg, U, Phi, ra, budget_s=20.0):
    """Time the FP64 oracle's SBCGrQ per iteration at the full workload (a fixed
    number of iterations), plus its force; scale to one force evaluation with
    the GPU's iteration count."""
    import oracle

    oracle.build()
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    X = oracle.sbcgrq(cfg["dims"], cfg["mass"], U, Phi, ra.beta, fixed_iters=1)[0]
    t_iter = time.perf_counter() - t0
    t_force = 0.0
    if t_iter < budget_s:
        t0 = time.perf_counter()
        oracle.force(cfg["dims"], U, X, ra.alpha)
        t_force = time.perf_counter() - t0
    return t_iter, t_force, threads


# the smaller configurations of the measurement plan (4^4 n_pf=2, 8^4 n_pf=4, 16^3x32 n_pf=8)
SMALL_CONFIGS = [
    {"name": "4^4, m=0.1, n_pf=2, 8 shifts of x^(-1/8) on [1e-3,64], eps=0.3", "dims": (4, 4, 4, 4), "mass": 0.1,
     "n_pf": 2, "ra": (-1.0 / 8, 1e-3, 64.0, 8), "eps": 0.3, "index": 1, "tol": 1e-10, "full": True},
    {"name": "8^4, m=0.05, n_pf=4, 12 shifts of x^(-1/16) on [2e-3,64], eps=0.5", "dims": (8, 8, 8, 8), "mass": 0.05,
     "n_pf": 4, "ra": (-1.0 / 16, 2e-3, 64.0, 12), "eps": 0.5, "index": 2, "tol": 1e-10, "full": True},
    {"name": "16^3x32, m=0.02, n_pf=8, 14 shifts of x^(-1/32) on [1e-3,64], eps=0.5", "dims": (16, 16, 16, 32),
     "mass": 0.02, "n_pf": 8, "ra": (-1.0 / 32, 1e-3, 64.0, 14), "eps": 0.5, "index": 3, "tol": 1e-8, "full": False},
]


def oracle_configs(reps=3):
    """The oracle's SBCGrQ (block) and per-vector multishift CG at the smaller
    configurations, FP64 on all host cores: whole solves with their iteration counts
    (median of `reps`), the force, and both solves once more on one thread (the paper's
    setting) at 4^4 and 8^4; at 16^3 x 32, where whole solves take minutes, seconds per
    iteration from 8 fixed iterations of each (one right-hand side for the per-vector
    solver)."""
    import numpy as np

    import oracle
    from paper_1808_01829_gb300 import synthetic as syn
    from paper_1808_01829_gb300.remez import rational_approx

    oracle.build()
    out = []
    for c in SMALL_CONFIGS:
        ra = rational_approx(*c["ra"])
        U = syn.random_links(c["dims"], c["eps"], syn.seed_gauge(c["index"]))
        B = syn.gaussian_pseudofermions(c["dims"], c["n_pf"], syn.seed_phi(c["index"]))
        rec = {"config": c["name"], "tol": c["tol"], "cores": oracle.max_threads()}
        if c["full"]:
            tb, tp = [], []
            for _ in range(reps):
                t0 = time.perf_counter()
                X, it_b, _ = oracle.sbcgrq(c["dims"], c["mass"], U, B, ra.beta, tol=c["tol"], max_iter=50000)
                tb.append(time.perf_counter() - t0)
                t0 = time.perf_counter()
                it_p = 0
                for j in range(c["n_pf"]):
                    it_p += oracle.scg(c["dims"], c["mass"], U, np.ascontiguousarray(B[..., j]), ra.beta,
                                       tol=c["tol"], max_iter=50000)[1]
                tp.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            oracle.force(c["dims"], U, X, ra.alpha)
            t_f = time.perf_counter() - t0
            # the paper's setting: one thread (one run each)
            threads = oracle.max_threads()
            oracle.set_threads(1)
            try:
                t0 = time.perf_counter()
                oracle.sbcgrq(c["dims"], c["mass"], U, B, ra.beta, tol=c["tol"], max_iter=50000)
                t1b = time.perf_counter() - t0
                t0 = time.perf_counter()
                for j in range(c["n_pf"]):
                    oracle.scg(c["dims"], c["mass"], U, np.ascontiguousarray(B[..., j]), ra.beta, tol=c["tol"],
                               max_iter=50000)
                t1p = time.perf_counter() - t0
            finally:
                oracle.set_threads(threads)
            rec.update({"sbcgrq_ms": statistics.median(tb) * 1e3, "sbcgrq_iters": it_b,
                        "pervector_scg_ms": statistics.median(tp) * 1e3, "pervector_scg_iters_total": it_p,
                        "force_ms": t_f * 1e3, "timing": f"median of {reps}",
                        "one_thread": {"sbcgrq_ms": t1b * 1e3, "pervector_scg_ms": t1p * 1e3}})
        else:
            k = 8
            t0 = time.perf_counter()
            oracle.sbcgrq(c["dims"], c["mass"], U, B, ra.beta, fixed_iters=k)
            t_b = (time.perf_counter() - t0) / k
            t0 = time.perf_counter()
            oracle.scg(c["dims"], c["mass"], U, np.ascontiguousarray(B[..., 0]), ra.beta, fixed_iters=k)
            t_p = (time.perf_counter() - t0) / k
            rec.update({"sbcgrq_s_per_iter": t_b, "pervector_scg_s_per_iter_per_rhs": t_p,
                        "timing": f"{k} fixed iterations each, one right-hand side for the per-vector solver"})
        out.append(rec)
    return out


def cpu_one_thread(cfg, ra):
    """The paper's per-core setting: one oracle SBCGrQ iteration on one thread at a
    lattice of half the extents (1/16 of the volume, same n_pf and shifts), scaled
    to the full volume.  Returns (seconds per full-volume iteration, sample text)."""
    import oracle
    from paper_1808_01829_gb300 import synthetic as syn

    small = [max(2, d // 2) for d in cfg["dims"]]
    vol_ratio = 1.0
    for d, d2 in zip(cfg["dims"], small):
        vol_ratio *= d / d2
    U = syn.random_links(small, cfg["eps"], syn.seed_gauge(cfg["index"]))
    Phi = syn.gaussian_pseudofermions(small, cfg["n_pf"], syn.seed_phi(cfg["index"]))
    oracle.build()
    threads = oracle.max_threads()
    oracle.set_threads(1)
    try:
        oracle.sbcgrq(small, cfg["mass"], U, Phi, ra.beta, fixed_iters=1)  # warm
        t0 = time.perf_counter()
        oracle.sbcgrq(small, cfg["mass"], U, Phi, ra.beta, fixed_iters=1)
        t = time.perf_counter() - t0
    finally:
        oracle.set_threads(threads)
    sample = (f"one oracle SBCGrQ iteration on 1 thread at {'x'.join(map(str, small))} ({t:.3f} s), "
              f"scaled by the volume ratio {vol_ratio:.0f}")
    return t * vol_ratio, sample


def oracle_parity(ctx, cfg, U, Phi, ra, G, ws):
    """Errors of the timed step's results against the FP64 oracle, per result:
    every (shift, column) true relative residual of the solutions (oracle operator;
    it bounds the solution error by tol ||B|| / (4m^2 + sigma) since lambda_min >= 4m^2)
    over tol, and the force computed on the GPU from those solutions against the
    oracle's force on 64 sampled links (t-boundary links included)."""
    import numpy as np
    import torch

    import oracle

    tol, dims, mass = cfg["tol"], cfg["dims"], cfg["mass"]
    Pd = torch.from_numpy(Phi).to(ctx.device)
    Xd, _ = ctx.block_multishift_cg(Pd, ra.beta, tol, precision=cfg["precision"])
    Gx, _, _ = ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, tol, X=Xd, out=G, workspace=ws)
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(4242)
    V = lx * ly * lz * lt
    links = [((x % lx) + lx * (((3 * x) % ly) + ly * (((5 * x) % lz) + lz * (lt - 1))), 3) for x in range(8)]
    links += [(int(rng.integers(V)), int(rng.integers(4))) for _ in range(56)]
    links = np.asarray(links, dtype=np.int64)
    rows = torch.from_numpy(links[:, 0]).to(ctx.device)
    mus = torch.from_numpy(links[:, 1]).to(ctx.device)
    Gs = Gx[rows, mus].cpu().numpy()
    X = Xd.cpu().numpy()
    del Xd
    t0 = time.perf_counter()
    bn = np.linalg.norm(Phi.reshape(-1, Phi.shape[-1]), axis=0)
    worst = 0.0
    for q, sig in enumerate(ra.beta):
        R = Phi - oracle.apply_A(dims, mass, U, X[q], sigma=sig)
        worst = max(worst, float(np.max(np.linalg.norm(R.reshape(-1, Phi.shape[-1]), axis=0) / bn)))
    Go = oracle.force_at(dims, U, X, ra.alpha, links)
    ferr = float(np.linalg.norm(Gs - Go) / np.linalg.norm(Go))
    return {"max_true_resid_over_tol": worst / tol, "solution_err_bound_ratio_max": worst / tol,
            "force_kernel_rel_err_64_links": ferr, "oracle_seconds": time.perf_counter() - t0,
            "how": "oracle operator on every (shift, column) of the GPU's solutions (the residual bounds the "
                   "solution error by resid ||B|| / (4m^2 + sigma)); oracle force on 64 links "
                   "from the same solutions (kernel parity, FP64 bound 1e-12)"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = WORKLOAD
    U, Phi, ra = make_inputs(cfg)
    # SBCGrQ iterations of this workload to the 1e-8 residual: the recursion the
    # oracle runs, counted on the GPU (REF_ITERS)
    ref_iters = int(os.environ.get("RHMC_REF_ITERS", "0")) or REF_ITERS
    times = []
    for step in range(args.warmup + args.steps):
        t_iter, t_force, threads = cpu_sample(cfg, U, Phi, ra)
        if step >= args.warmup:
            times.append((t_iter, t_force))
    t_iter = statistics.median(t for t, _ in times)
    t_force = statistics.median(f for _, f in times)
    iters = ref_iters
    est_ms = (t_iter * iters + t_force) * 1e3
    t1, sample1 = cpu_one_thread(cfg, ra)
    line = {
        "metric": METRIC, "value": est_ms, "unit": "ms", "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": est_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["workload"], "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": est_ms, "unit": "ms", "cores": threads, "kind": "oracle",
                         "sample": f"one oracle SBCGrQ iteration ({t_iter:.2f} s) + oracle force ({t_force:.2f} s) "
                                   f"at the full 24^4 workload, scaled by the {iters} SBCGrQ iterations of this workload",
                         "one_thread": {"value": t1 * iters * 1e3, "unit": "ms",
                                        "sample": sample1 + f", times the {iters} iterations (solve only)"}},
        "e2e": {"value": est_ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ batched ensembles
BATCH = {
    "workload": "6 ensembles 8^4,12^4,16^4,16^3x32,20^4,24^4 (eps=0.5), n_pf 2,4,8,8,12,16, 12 shifts of "
                "x^(-1/(4 n_pf)) on [2e-3,64], m=0.025, tol 1e-8, mixed",
    "dims": [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (16, 16, 16, 32), (20, 20, 20, 20), (24, 24, 24, 24)],
    "n_pf": [2, 4, 8, 8, 12, 16],
    "mass": 0.025,
    "tol": 1e-8,
}


def run_batch(dev, reps=3):
    """One batched SBCGrQ over six uneven ensembles (rhmc_block_multishift_cg_batch)
    against the same six solves issued one after another on one stream."""
    import torch
    from paper_1808_01829_gb300 import synthetic as syn
    from paper_1808_01829_gb300.api import RhmcContext, block_multishift_cg_batch
    from paper_1808_01829_gb300.remez import rational_approx

    from paper_1808_01829_gb300 import autotune

    items, tuned = [], []
    cache = os.path.join(tempfile.mkdtemp(prefix="rhmc_tune_"), "tune.json")
    for k, (dims, n) in enumerate(zip(BATCH["dims"], BATCH["n_pf"])):
        ra = rational_approx(-1.0 / (4 * n), 2e-3, 64.0, 12)
        ctx = RhmcContext(dims, BATCH["mass"], device=dev.index or 0)
        ctx.set_gauge(torch.from_numpy(syn.random_links(dims, 0.5, syn.seed_gauge(10 + k))).to(dev))
        B = torch.from_numpy(syn.gaussian_pseudofermions(dims, n, syn.seed_phi(10 + k))).to(dev)
        # per-ensemble launch settings (hop RHS per thread, update tile shape), untimed
        tuned.append(autotune.tune(ctx, n, shifts=ra.beta, cache=cache))
        items.append((ctx, B, ra.beta))
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        out = []
        for it in range(reps + 1):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                out.append(a.elapsed_time(b))
        return statistics.median(out), r

    seq_ms, seq = timed(lambda: [c.block_multishift_cg(B, sh, BATCH["tol"], precision="mixed")[1]
                                 for c, B, sh in items])
    # each member alone (the sum is the sequential time; the largest bounds the batch from below)
    member_ms = [timed(lambda c=c, B=B, sh=sh: c.block_multishift_cg(B, sh, BATCH["tol"], precision="mixed"))[0]
                 for c, B, sh in items]
    bat_ms, bat = timed(lambda: [i for _, i in block_multishift_cg_batch(items, BATCH["tol"], precision="mixed")])
    sites_rhs = sum(int(torch.tensor(d).prod()) // 2 * n for d, n in zip(BATCH["dims"], BATCH["n_pf"]))
    res = {"workload": BATCH["workload"], "ms": bat_ms, "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / bat_ms,
           "member_ms": member_ms,
           "iters": [i.iters for i in bat], "true_rel_resid_max": max(i.true_rel_resid_max for i in bat),
           "autotuned": [{str(k): v for k, v in t.items()} for t in tuned],
           "site_rhs_shifts_per_s": sites_rhs * 12 / (bat_ms * 1e-3)}
    for c, _, _ in items:
        c.close()
    return res


# ------------------------------------------------------------------ RHMC trajectory
TRAJ = {
    "workload": "RHMC trajectory on 8^4 (the paper's lattice, Sec. IV), beta=5.12, m=0.025, n_pf=4, eps=0.5 links; "
                "MD/action x^(-1/16), heatbath x^(+1/32), 12 shifts on [2e-3,64]; tau=1, n_steps=10, n_gauge=3, "
                "lambda=1/6 (two-level OMF2); MD solves mixed 1e-7, heatbath/action FP64 1e-14",
    "dims": (8, 8, 8, 8), "mass": 0.025, "n_pf": 4, "beta": 5.12, "tau": 1.0, "n_steps": 10, "n_gauge": 3,
    "lam": 1.0 / 6, "tol_md": 1e-7, "tol_action": 1e-14,
}
# real flops per link of the FP64 trajectory kernels (3 x 3 complex product = 27 complex MACs
# = 216 flops): gauge kick 13 products (six staples of two products each, then U V); link
# update 17 (degree-16 Taylor polynomial in Horner form, then E U; no squaring at these steps)
TRAJ_FLOPS = {"gauge_kick": 13 * 216, "link_update": 17 * 216}


def run_trajectory(dev, fp64_peak, with_oracle, reps=3):
    """Time per RHMC trajectory (rhmc_hmc_trajectory) on the 8^4 workload above, the FP64
    gauge kernels at 24^4 against the measured FP64 peak, and the oracle on a bounded
    sample (one outer OMF2 step with its gauge drifts, plus the heatbath and the two
    actions, scaled to n_steps outer steps)."""
    import torch

    from paper_1808_01829_gb300 import hmc
    from paper_1808_01829_gb300 import synthetic as syn
    from paper_1808_01829_gb300.api import RhmcContext
    from paper_1808_01829_gb300.remez import rational_approx

    T = TRAJ
    dims, n = T["dims"], T["n_pf"]
    ra = rational_approx(-1.0 / (4 * n), 2e-3, 64.0, 12)
    hb = rational_approx(1.0 / (8 * n), 2e-3, 64.0, 12)
    U0 = syn.random_links(dims, 0.5, syn.seed_gauge(20))
    p = torch.from_numpy(syn.momentum_normals(dims, 21)).to(dev)
    eta = torch.from_numpy(syn.gaussian_pseudofermions(dims, n, 22)).to(dev)
    ctx = RhmcContext(dims, T["mass"], device=dev.index or 0)
    ctx.set_gauge(torch.from_numpy(U0).to(dev))
    prm = hmc.MdParams(beta=T["beta"], tau=T["tau"], n_steps=T["n_steps"], n_gauge=T["n_gauge"], lam=T["lam"],
                       tol_md=T["tol_md"], precision="mixed")
    stream = torch.cuda.current_stream(dev)
    times, rec = [], None
    for it in range(reps + 1):
        U = torch.from_numpy(U0).to(dev)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rec = hmc.trajectory(ctx, U, p, eta, hb, ra, ra, prm, tol_action=T["tol_action"], u=0.5)
        b.record(stream)
        torch.cuda.synchronize()
        if it > 0:
            times.append(a.elapsed_time(b))
    ctx.close()
    out = {"workload": T["workload"], "ms_per_trajectory": statistics.median(times),
           "timing": f"median of {reps} after one warm-up, CUDA events", "dH": rec["dH"],
           "accepted_at_u_0.5": rec["accepted"], "force_evals": rec["md"]["force_evals"],
           "gauge_kicks": rec["md"]["gauge_force_evals"], "md_solver_iters": rec["md"]["solver_iters"],
           "md_max_rel_resid": rec["md"]["max_rel_resid"]}

    # FP64 gauge kernels at 24^4 (FP64-ALU bound): events around 10 launches each
    d24 = (24, 24, 24, 24)
    c24 = RhmcContext(d24, 0.01, device=dev.index or 0)
    U24 = torch.from_numpy(syn.random_links(d24, 0.5, syn.seed_gauge(3))).to(dev)
    P24 = hmc.momenta(c24, torch.from_numpy(syn.momentum_normals(d24, 23)).to(dev))
    links = 4 * c24.V
    kern = {}
    for name, fn in (("gauge_kick", lambda: hmc.gauge_kick(c24, U24, P24, T["beta"], 1e-3)),
                     ("link_update", lambda: hmc.link_update(c24, U24, P24, 1e-3))):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(10):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        us = a.elapsed_time(b) * 100.0
        tf = TRAJ_FLOPS[name] * links / (us * 1e-6) / 1e12
        kern[name] = {"us_per_launch": us, "bound": "fp64", "achieved": tf, "peak": fp64_peak,
                      "unit": "TFLOP/s (FP64)", "frac": tf / fp64_peak if fp64_peak else None,
                      "count": f"{TRAJ_FLOPS[name]} flops per link, {links} links (24^4)"}
    c24.close()
    out["kernels_24x24x24x24"] = kern

    # oracle (the trajectory's CPU baseline): one outer OMF2 step (three pseudofermion forces, two
    # gauge drifts) + heatbath + two actions
    if not with_oracle:
        return out
    try:
        from oracle import trajectory as tr

        Uc = U0
        Pc = tr.momenta_from_normals(syn.momentum_normals(dims, 21))
        etac = syn.gaussian_pseudofermions(dims, n, 22)
        t0 = time.perf_counter()
        Phi = tr.heatbath(dims, T["mass"], Uc, etac, hb, T["tol_action"])
        tr.fermion_action(dims, T["mass"], Uc, Phi, ra, T["tol_action"])
        t1 = time.perf_counter()
        tr.trajectory(dims, T["mass"], Uc, Pc, Phi, T["beta"], ra, T["tau"] / T["n_steps"], 1, T["n_gauge"],
                      T["lam"], T["tol_md"])
        t2 = time.perf_counter()
        est = (2 * (t1 - t0) - 0.0) + (t2 - t1) * T["n_steps"]
        out["cpu_oracle"] = {"value": est * 1e3, "unit": "ms per trajectory", "kind": "oracle",
                             "cores": os.cpu_count(),
                             "sample": f"heatbath + one action ({t1 - t0:.2f} s, counted twice for the two "
                                       f"actions) and one outer OMF2 step ({t2 - t1:.2f} s) x {T['n_steps']}"}
    except Exception as e:  # a measurement beside the bench line: it never fails the line
        out["cpu_oracle"] = {"error": f"{type(e).__name__}: {e}"[:200]}
    return out


# ------------------------------------------------------------------ hop widths
def dslash_widths(ctx, dev, widths=(1, 2, 4, 8, 16), reps=10):
    """FP32 hop at several right-hand-side widths on the bench lattice (the width-1
    against width-n comparison of Sec. IV.B, Fig. 8): microseconds and algorithmic
    GB/s per launch from the library's event profiler.  The launches alternate
    between the two parities, so the two link sets (2 x 96 MB at 24^4) exceed L2."""
    import torch

    from paper_1808_01829_gb300 import roofline

    out = []
    for n in widths:
        X = torch.randn(ctx.Vh, 3, n, dtype=torch.complex128, device=dev)
        ctx.hop(X, 1, precision="fp32")
        stats = roofline.profile(lambda: [ctx.hop(X, r & 1, precision="fp32") for r in range(reps)])
        e = roofline.entry(stats, "hop_fp32")
        out.append({"n_rhs": n, "us_per_launch": round(e["us_per_launch"], 2), "GB/s": round(e["achieved"], 1),
                    "frac": round(e["frac"], 3)})
        del X
    return out


# ------------------------------------------------------------------ ALU fractions
DF_OPS_PER_SITE_RHS = 8 * 9 * 4 * 12  # double-float hop: 8 links x 9 entries x 4 real products x 12 FP32 instructions


def alu_fractions(ctx, stats, cfg, lib):
    """Measured CUDA-core peaks (rhmc_probe_alu_peaks) and the fractions reached by
    the FP32-ALU-bound double-float hop (FP32 instruction rate), and by the FP64
    parts: the n x n coefficient chain (estimated flops) and the FP64 hop of the
    per-vector baseline (570 flops per site and right-hand side)."""
    import ctypes

    from paper_1808_01829_gb300 import roofline

    f32, f32x2, f64 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.rhmc_probe_alu_peaks(ctx.device.index or 0, ctypes.byref(f32), ctypes.byref(f32x2), ctypes.byref(f64),
                                  None)
    if rc != 0:
        return None
    peaks = {"fp32_tflops": f32.value, "fp32x2_tflops": f32x2.value, "fp64_tflops": f64.value,
             "how": "best of 5 launches of independent FMA chains on every SM, CUDA events (2 flops per FMA lane)"}
    n, ns = cfg["n_pf"], cfg["n_shifts"]
    vh = ctx.Vh
    out = {}
    if "hop_df" in stats:
        e = stats["hop_df"]
        ops = e["launches"] * vh * n * DF_OPS_PER_SITE_RHS
        achieved = ops / (e["ms"] * 1e-3) / 1e12  # T FP32 instructions / s
        peak = f32.value / 2
        out["hop_df"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 instr/s",
                         "frac": achieved / peak, "peak_source": "of measured (rhmc_probe_alu_peaks)",
                         "count": "8 x 9 x 4 real products x 12 FP32 instructions per site and right-hand side"}
    if "nxn" in stats:
        e = stats["nxn"]
        # per iteration, alpha (LDL^dagger inverse, ~4 n^3/3 complex MACs) and rho (LDL^dagger, triangular
        # inverse, delta update, ~2 n^3 complex MACs), 8 flops per complex MAC; two launches per iteration
        flops = e["launches"] / 2 * 8 * (4 / 3 + 2) * n ** 3
        achieved = flops / (e["ms"] * 1e-3) / 1e12
        out["nxn"] = {"bound": "latency", "achieved": achieved, "peak": f64.value, "unit": "TFLOP/s (FP64)",
                      "frac": achieved / f64.value, "peak_source": "of measured (rhmc_probe_alu_peaks)",
                      "count": "estimated: (4/3 + 2) n^3 complex MACs per iteration; one SM per problem"}
    if "nxn_shifts" in stats:
        e = stats["nxn_shifts"]
        flops = e["launches"] * (ns - 1) * 8 * 10 * n ** 3  # nine products and one inverse per shift
        achieved = flops / (e["ms"] * 1e-3) / 1e12
        out["nxn_shifts"] = {"bound": "latency", "achieved": achieved, "peak": f64.value, "unit": "TFLOP/s (FP64)",
                             "frac": achieved / f64.value, "peak_source": "of measured (rhmc_probe_alu_peaks)",
                             "count": "estimated: 10 n^3 complex MACs per shift and iteration"}
    try:  # the FP64 hop of the per-vector baseline (width 1)
        import torch

        X = torch.randn(ctx.Vh, 3, 1, dtype=torch.complex128, device=ctx.device)
        ctx.hop(X, 1, precision="fp64")
        st = roofline.profile(lambda: [ctx.hop(X, r & 1, precision="fp64") for r in range(10)])
        e = st["hop_fp64"]
        flops = e["launches"] * vh * 570
        achieved = flops / (e["ms"] * 1e-3) / 1e12
        gbs = e["bytes"] / (e["ms"] * 1e-3) / 1e9
        out["hop_fp64_width1"] = {"bound": "fp64", "achieved": achieved, "peak": f64.value,
                                  "unit": "TFLOP/s (FP64)", "frac": achieved / f64.value,
                                  "hbm_GB/s": gbs, "hbm_frac": gbs / roofline.peaks()["hbm_gbs"],
                                  "peak_source": "of measured (rhmc_probe_alu_peaks)",
                                  "count": "570 flops per site per right-hand side"}
    except Exception as ex:  # a measurement beside the bench line: it never fails the line
        out["hop_fp64_width1"] = {"error": f"{type(ex).__name__}: {ex}"[:200]}
    return {"peaks": peaks, "fractions": out}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    from paper_1808_01829_gb300 import replicas

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    replicas.init("nccl")
    dev = torch.device("cuda", local)
    from paper_1808_01829_gb300 import _build
    from paper_1808_01829_gb300.api import RhmcContext

    _build.build()
    from paper_1808_01829_gb300 import _lib as _l

    for kv in args.tune:
        k, v = kv.split("=")
        _l.check(_l.load().rhmc_tune_set(int(k), int(v)), "rhmc_tune_set")
    cfg = dict(WORKLOAD)
    if args.small:
        cfg.update(dims=[8, 8, 8, 8], mass=0.05, n_pf=4, n_shifts=12, r=-1.0 / 16, interval=[2e-3, 64.0], index=1,
                   workload="8^4 quick check")
    U, Phi, ra = make_inputs(cfg)
    ctx = RhmcContext(cfg["dims"], cfg["mass"], device=local)
    Ud = torch.from_numpy(U).to(dev)
    ctx.set_gauge(Ud)
    Pd = torch.from_numpy(Phi).to(dev)
    n, ns = cfg["n_pf"], cfg["n_shifts"]
    ws = torch.empty(ctx.workspace_bytes(n, ns, cfg["precision"]), dtype=torch.uint8, device=dev)
    G = torch.empty((ctx.V, 4, 3, 3), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        # one force evaluation: FP32 (and double-float) link staging from the resident FP64
        # links, the solve, the force
        ctx.set_gauge(Ud)
        return ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, cfg["tol"], precision=cfg["precision"], out=G,
                         workspace=ws)

    infos = []
    for _ in range(args.warmup):
        infos.append(step()[2])
    replicas.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    lib = ctx.lib
    l0 = lib.rhmc_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, S, info = step()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = int(lib.rhmc_kernel_launches() - l0)
    replicas.barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    last = infos[-1]

    # ---- end to end: pinned host U and Phi -> device, staging, force, G -> pinned host
    Uh = torch.from_numpy(U).pin_memory()
    Ph = torch.from_numpy(Phi).pin_memory()
    Gh = torch.empty((ctx.V, 4, 3, 3), dtype=torch.complex128).pin_memory()
    Ud2 = torch.empty_like(Ud)
    Pd2 = torch.empty_like(Pd)
    e2e = []
    for it in range(max(2, min(3, args.steps)) + 1):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Ud2.copy_(Uh, non_blocking=True)
        Pd2.copy_(Ph, non_blocking=True)
        ctx.set_gauge(Ud2)
        ctx.force(Pd2, ra.alpha0, ra.alpha, ra.beta, cfg["tol"], precision=cfg["precision"], out=G, workspace=ws)
        Gh.copy_(G, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if it > 0:
            e2e.append(a.elapsed_time(b))
    e2e_ms = statistics.median(e2e)

    # ---- per-kernel times: one more step with the library's event profiler
    from paper_1808_01829_gb300 import roofline

    stats = roofline.profile(step)
    kt = roofline.table(stats)
    hbm_kernels = [r["kernel"] for r in kt if r["GB/s"]]
    dominant = hbm_kernels[0] if hbm_kernels else None
    roof = roofline.entry(stats, dominant) if dominant else None
    if roof and dominant in TRAFFIC_RATIO:
        ratio, src = TRAFFIC_RATIO[dominant]
        roof["traffic"] = ratio * roof["algorithmic_bytes_per_launch"]
        roof["traffic_source"] = src
    roof_dslash = roofline.entry(stats, "hop_fp32") if "hop_fp32" in stats else None
    roof_tensor = roofline.tensor_entry(stats, "basis_tc") if stats.get("basis_tc", {}).get("flops") else None
    if roof_dslash and "hop_fp32" in TRAFFIC_RATIO:
        ratio, src = TRAFFIC_RATIO["hop_fp32"]
        roof_dslash["traffic"] = ratio * roof_dslash["algorithmic_bytes_per_launch"]
        roof_dslash["traffic_source"] = src

    # ---- comparisons (Fig. 9 analogue): per-vector FP64 multishift CG + force (the metric's
    # baseline), and the same-precision pairs that isolate the block algorithm's gain.  Each is
    # warmed up once (workspace sized outside the timed calls), then the median of `reps`.
    base, same = None, None
    if not args.no_baseline and rank == 0:
        def timed_median(fn, reps=3):
            fn()
            out = []
            for _ in range(reps):
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = fn()
                b.record(stream)
                torch.cuda.synchronize()
                out.append(a.elapsed_time(b))
            return statistics.median(out), r

        def pervector_fp64():
            Xs, binfo = ctx.multishift_cg_pervector(Pd, ra.beta, cfg["tol"])
            ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, cfg["tol"], X=Xs, out=G, workspace=ws)
            return binfo

        def block_fp64():
            _, _, info = ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, cfg["tol"], precision="fp64", out=G,
                                   workspace=ws64)
            return info

        def pervector_mixed():
            Xs = torch.empty((ns,) + tuple(Pd.shape), dtype=Pd.dtype, device=dev)
            its = 0
            for j in range(n):
                col = Pd[..., j:j + 1].contiguous()
                Xj, info = ctx.block_multishift_cg(col, ra.beta, cfg["tol"], precision="mixed", workspace=ws1)
                Xs[..., j:j + 1] = Xj
                its += info.iters
            ctx.force(Pd, ra.alpha0, ra.alpha, ra.beta, cfg["tol"], X=Xs, out=G, workspace=ws)
            return its

        ms_pv, binfo = timed_median(pervector_fp64)
        base = {"ms": ms_pv, "iters_total": binfo.iters, "dirac_calls_width1": binfo.dirac_calls,
                "speedup": ms_pv / ms, "timing": "median of 3 after one warm-up"}
        ws64 = torch.empty(ctx.workspace_bytes(n, ns, "fp64"), dtype=torch.uint8, device=dev)
        ms_b64, b64info = timed_median(block_fp64)
        del ws64
        ws1 = torch.empty(ctx.workspace_bytes(1, ns, "mixed"), dtype=torch.uint8, device=dev)
        ms_pvm, pvm_iters = timed_median(pervector_mixed)
        del ws1
        same = {"fp64": {"block_ms": ms_b64, "pervector_ms": ms_pv, "block_speedup": ms_pv / ms_b64,
                         "block_iters": b64info.iters, "pervector_iters_total": binfo.iters},
                "mixed": {"block_ms": ms, "pervector_ms": ms_pvm, "block_speedup": ms_pvm / ms,
                          "block_iters": last.iters, "pervector_iters_total": pvm_iters},
                "note": "per-vector mixed = the block solver with one right-hand side per solve (multishift CG "
                        "with the same FP32 operator, FP64-accurate reliable updates and defect corrections), "
                        "16 solves in turn, then the same force"}
        torch.cuda.empty_cache()

    # ---- CUDA-core peaks and the FP32 / FP64 fractions
    alu = None
    if rank == 0 and not args.small:
        alu = alu_fractions(ctx, stats, cfg, lib)

    batch = None
    if not args.no_batch and not args.small:
        batch = run_batch(dev)

    traj = None
    if not args.no_traj and not args.small and rank == 0:
        try:
            traj = run_trajectory(dev, alu["peaks"]["fp64_tflops"] if alu else None,
                                  with_oracle=not args.no_cpu and world == 1)
        except Exception as e:  # a measurement beside the bench line: it never fails the line
            traj = {"error": f"{type(e).__name__}: {e}"[:300]}

    widths = None
    if rank == 0 and not args.small:
        try:
            widths = dslash_widths(ctx, dev)
        except Exception as e:  # a measurement beside the bench line: it never fails the line
            widths = {"error": f"{type(e).__name__}: {e}"[:300]}

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        t_iter, t_force, threads = cpu_sample(cfg, U, Phi, ra)
        est = (t_iter * last.iters + t_force) * 1e3
        cpu = {"value": est, "unit": "ms", "cores": threads, "kind": "oracle",
               "sample": f"one oracle SBCGrQ iteration ({t_iter:.2f} s) + oracle force ({t_force:.2f} s) at the "
                         f"full workload, scaled by the GPU's {last.iters} iterations"}
        try:  # per-result error of the timed step's solutions and force against the oracle
            cpu["parity_vs_oracle"] = oracle_parity(ctx, cfg, U, Phi, ra, G, ws)
        except Exception as e:  # never fails the line
            cpu["parity_vs_oracle"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        try:  # the oracle's per-vector multishift CG at the full workload: one iteration on one
            # right-hand side, scaled by the per-vector iteration total of the GPU's FP64 baseline
            import numpy as np

            import oracle

            if base is None:
                raise RuntimeError("no per-vector baseline was run")
            k = 4
            t0 = time.perf_counter()
            oracle.scg(cfg["dims"], cfg["mass"], U, np.ascontiguousarray(Phi[..., 0]), ra.beta, fixed_iters=k)
            t_pv = (time.perf_counter() - t0) / k
            pv_iters = base["iters_total"]
            cpu["pervector_scg_estimate"] = {
                "value": t_pv * pv_iters * 1e3, "unit": "ms",
                "sample": f"{k} oracle SCG iterations on one right-hand side at the full workload ({t_pv:.3f} s "
                          f"each), times {pv_iters} per-vector iterations (16 right-hand sides, the GPU baseline's "
                          f"count), solve only"}
        except Exception as e:  # never fails the line
            cpu["pervector_scg_estimate"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        try:  # the oracle's block and per-vector solvers at the smaller configurations
            cpu["oracle_configs"] = oracle_configs()
        except Exception as e:  # never fails the line
            cpu["oracle_configs"] = {"error": f"{type(e).__name__}: {e}"[:200]}
        try:  # the paper's per-core setting, beside the all-cores figure
            t1, sample1 = cpu_one_thread(cfg, ra)
            cpu["one_thread"] = {"value": t1 * last.iters * 1e3, "unit": "ms",
                                 "sample": sample1 + f", times the GPU's {last.iters} iterations (solve only)"}
        except Exception as e:  # never fails the line
            cpu["one_thread"] = {"error": f"{type(e).__name__}: {e}"[:200]}

    if rank == 0:
        len_b = Phi.nbytes + U.nbytes
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "force_evals_per_s": world * 1000.0 / ms,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": cfg["workload"], "precision": cfg["precision"],
                       "step": "link staging (FP64 links resident) + solve to tol for every (shift, column) + force",
                       "l2": "inputs larger than L2 (U 191 MB, fields 64-127 MB each)",
                       "parallelism": f"replicas x{world}", **({"tune": args.tune} if args.tune else {})},
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": len_b, "d2h_bytes_per_step": G.numel() * 16},
            "gpu_launches": launches,
            "roofline": roof,
            "roofline_dslash": roof_dslash,
            "roofline_tensor": roof_tensor,
            "dslash_widths": widths,
            "kernel_table": kt,
            "clocks": clk,
            "solver": {"iters": last.iters, "dirac_calls": last.dirac_calls, "reliable_updates": last.reliable_updates,
                       "refinements": last.refinements, "refine_iters": last.refine_iters,
                       "phase1_rel_resid_max": last.phase1_rel_resid_max,
                       "phase1_ms": last.phase1_ms, "refine_ms": last.refine_ms,
                       "true_rel_resid_max": last.true_rel_resid_max},
            "baseline_fp64_scg": base,
            "same_precision": same,
            "alu_peaks": alu["peaks"] if alu else None,
            "roofline_alu": alu["fractions"] if alu else None,
            "batched_ensemble": batch,
            "trajectory": traj,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close()
    replicas.finalize()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
