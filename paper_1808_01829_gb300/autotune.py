"""Autotuner for the library's launch parameters (rhmc_tune_set).

For a given workload (lattice, n_rhs) it times, with the library's own event
profiler, the candidates of

* the FP32 hop: one or two right-hand sides per thread (RHMC_TUNE_HOP_STAGED
  3 / 4), on the FP32 operator;
* at 16 right-hand sides, the row tiles of the packed Gram (RHMC_TUNE_GRAM_TILE)
  and of the fused base step (RHMC_TUNE_BASE_TILE), in a short mixed-precision
  solve with the given shifts;

and keeps the fastest.  The settings are applied to the context
(rhmc_ctx_tune_set), so ensembles solved together by
rhmc_block_multishift_cg_batch each run their own.  Results are cached in a
JSON file keyed by GPU name, lattice extents and width, so later runs only
apply them.  Tuning changes how kernels are launched, never what they compute.
"""
from __future__ import annotations

import json
import os
from typing import Optional

import torch

from . import _lib, roofline

KEY_HOP = 8          # RHMC_TUNE_HOP_STAGED
KEY_BASE_TILE = 19   # RHMC_TUNE_BASE_TILE
KEY_GRAM_TILE = 20   # RHMC_TUNE_GRAM_TILE
HOP_CANDIDATES = (3, 4)
TILE_CANDIDATES = (0, 1, 2, 3)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rhmc_gb300_autotune.json")


def _key(dims, n):
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    return f"{name}|{'x'.join(str(d) for d in dims)}|n={n}"


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def apply(rctx, settings: dict):
    for k, v in settings.items():
        rctx.tune_set(int(k), int(v))


def reset(rctx):
    for k in (KEY_HOP, KEY_BASE_TILE, KEY_GRAM_TILE):
        rctx.tune_set(k, 0)


def _per_launch(stats, name, per_byte=False):
    s = stats.get(name)
    if not s or not s["launches"]:
        return None
    return s["ms"] / (max(s["bytes"], 1.0) if per_byte else s["launches"])


def tune(rctx, n: int, shifts=None, cache: Optional[str] = DEFAULT_CACHE, force: bool = False, reps: int = 5):
    """Tune for context rctx and width n; returns {key: value} (applied to rctx)."""
    db = _load(cache)
    key = _key(rctx.dims, n)
    if key in db and not force:
        settings = {int(k): v for k, v in db[key].items()}
        apply(rctx, settings)
        return settings
    from . import synthetic as syn

    X = torch.from_numpy(syn.gaussian_pseudofermions(rctx.dims, n, 99)).to(rctx.device)
    settings = {}
    best = None
    for mode in HOP_CANDIDATES:
        if mode == 4 and n % 2:
            continue
        rctx.tune_set(KEY_HOP, mode)
        try:
            rctx.apply_mdagm_mrhs(X, 0.0, "fp32")
            st = roofline.profile(lambda: [rctx.apply_mdagm_mrhs(X, 0.0, "fp32") for _ in range(reps)])
        except _lib.RhmcError:
            continue
        t = _per_launch(st, "hop_fp32")
        if t is not None and (best is None or t < best[0]):
            best = (t, mode)
    if best:
        settings[KEY_HOP] = best[1]
        rctx.tune_set(KEY_HOP, best[1])
    if shifts and n == 16:
        for tkey, cat in ((KEY_GRAM_TILE, "gram_fp32"), (KEY_BASE_TILE, "update_shifts_fp32")):
            best = None
            for v in TILE_CANDIDATES:
                rctx.tune_set(tkey, v)
                try:
                    st = roofline.profile(lambda: rctx.block_multishift_cg(X, shifts, 1e-3, max_iter=12,
                                                                           precision="mixed",
                                                                           allow_not_converged=True))
                except _lib.RhmcError:
                    continue
                t = _per_launch(st, cat)
                if t is not None and (best is None or t < best[0]):
                    best = (t, v)
            rctx.tune_set(tkey, best[1] if best else 0)
            if best:
                settings[tkey] = best[1]
    if cache:
        db = _load(cache)
        db[key] = {str(k): v for k, v in settings.items()}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(db, f, indent=1)
    return settings
