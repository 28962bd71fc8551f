"""Autotuner for the library's launch parameters (rhmc_tune_set).

For a given workload (lattice, n_rhs) it times the candidates of each tunable
with the library's own event profiler and keeps the fastest:

* hop right-hand sides per thread (1, 2, 4 dividing n): FP32 and FP64 operator;
* threads per CTA of the fused shift update (64, 128, 256): a short solve.

Results are cached in a JSON file keyed by GPU name, lattice extents and width,
so later runs only apply them.  Tuning only changes how kernels are launched,
never what they compute.
"""
from __future__ import annotations

import json
import os
from typing import Optional

import torch

from . import _lib, roofline

KEY_HOP_R = 0
KEY_UPDATE_THREADS = 1
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rhmc_gb300_autotune.json")


def _key(dims, n):
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    return f"{name}|{'x'.join(str(d) for d in dims)}|n={n}"


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def apply(settings: dict):
    lib = _lib.load()
    for k, v in settings.items():
        _lib.check(lib.rhmc_tune_set(int(k), int(v)), "rhmc_tune_set")


def reset():
    lib = _lib.load()
    for k in range(8):
        lib.rhmc_tune_set(k, 0)


def tune(rctx, n: int, shifts=None, cache: Optional[str] = DEFAULT_CACHE, force: bool = False, reps: int = 5):
    """Tune for context rctx and width n; returns {key: value} (applied)."""
    db = _load(cache)
    key = _key(rctx.dims, n)
    if key in db and not force:
        settings = {int(k): v for k, v in db[key].items()}
        apply(settings)
        return settings
    lib = _lib.load()
    from . import synthetic as syn

    X = torch.from_numpy(syn.gaussian_pseudofermions(rctx.dims, n, 99)).to(rctx.device)
    settings = {}
    # hop: right-hand sides per thread, timed on the FP32 operator
    best = None
    for R in (1, 2, 4):
        if n % R:
            continue
        lib.rhmc_tune_set(KEY_HOP_R, R)
        try:
            rctx.apply_mdagm_mrhs(X, 0.0, "fp32")
            st = roofline.profile(lambda: [rctx.apply_mdagm_mrhs(X, 0.0, "fp32") for _ in range(reps)])
        except _lib.RhmcError:
            continue
        t = st["hop_fp32"]["ms"] / st["hop_fp32"]["launches"]
        if best is None or t < best[0]:
            best = (t, R)
    settings[KEY_HOP_R] = best[1]
    lib.rhmc_tune_set(KEY_HOP_R, best[1])
    # fused shift update: threads per CTA, timed inside a short solve
    if shifts:
        best = None
        for thr in (64, 128, 256):
            lib.rhmc_tune_set(KEY_UPDATE_THREADS, thr)
            try:
                st = roofline.profile(lambda: rctx.block_multishift_cg(X, shifts, 1e-3, max_iter=12,
                                                                       precision="mixed", allow_not_converged=True))
            except _lib.RhmcError:
                continue
            if "update_fp32" not in st:
                continue
            t = st["update_fp32"]["ms"] / max(st["update_fp32"]["bytes"], 1.0)
            if best is None or t < best[0]:
                best = (t, thr)
        if best:
            settings[KEY_UPDATE_THREADS] = best[1]
            lib.rhmc_tune_set(KEY_UPDATE_THREADS, best[1])
    if cache:
        db = _load(cache)
        db[key] = {str(k): v for k, v in settings.items()}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(db, f, indent=1)
    return settings
