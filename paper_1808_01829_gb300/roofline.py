"""Per-kernel timing through the library's profiler, and roofline entries.

The library records CUDA events on the launching stream around each of its
kernel launches (rhmc_profile_enable) together with the launch's algorithmic
bytes: every input read once, every output written once.  Achieved bandwidth
is those bytes divided by the event-timed duration; the peak is the measured
HBM copy bandwidth of this GPU model (MEASURED_PEAKS.json at the repository
root), or a fallback figure when that file is absent.
"""
from __future__ import annotations

import ctypes
import json
import os

from . import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FALLBACK_HBM_GBS = 6800.0
FALLBACK_FP32_TFLOPS = 73.0  # FP32 FMA throughput measured with a probe on this GPU model


FALLBACK_BF16_TFLOPS = 1900.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d.get("bf16_tflops", FALLBACK_BF16_TFLOPS)),
                "source": "of measured"}
    return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS, "source": "of fallback"}


def tensor_entry(stats: dict, name: str, peak=None):
    """Roofline object for a tensor-core kernel: issued FP16 MMA flops per launch over its
    event-timed duration, against the measured dense BF16 peak (FP16 runs at the same rate)."""
    p = peak or peaks()
    s = stats[name]
    per_launch_s = s["ms"] / s["launches"] * 1e-3
    achieved = s["flops"] / s["launches"] / per_launch_s / 1e12
    return {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": p["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / p["bf16_tflops"], "peak_source": p["source"] + " (dense BF16; FP16 same rate)",
            "flops_per_launch": s["flops"] / s["launches"], "us_per_launch": per_launch_s * 1e6,
            "launches": s["launches"], "traffic": None}


def profile(fn):
    """Run fn() with the library profiler on; return {category: {launches, ms, bytes}}."""
    lib = _lib.load()
    _lib.check(lib.rhmc_profile_enable(1), "rhmc_profile_enable")
    try:
        fn()
    finally:
        out = {}
        for k, name in enumerate(_lib.PROF_CATEGORIES):
            n = ctypes.c_longlong(0)
            ms = ctypes.c_double(0)
            by = ctypes.c_double(0)
            _lib.check(lib.rhmc_profile_read(k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)),
                       "rhmc_profile_read")
            if n.value:
                fl = ctypes.c_double(0)
                _lib.check(lib.rhmc_profile_read_flops(k, ctypes.byref(fl)), "rhmc_profile_read_flops")
                out[name] = {"launches": int(n.value), "ms": ms.value, "bytes": by.value, "flops": fl.value}
        lib.rhmc_profile_enable(0)
    return out


def entry(stats: dict, name: str, peak=None, traffic=None):
    """Roofline object for one kernel category (HBM bound)."""
    p = peak or peaks()
    s = stats[name]
    per_launch_bytes = s["bytes"] / s["launches"]
    per_launch_s = s["ms"] / s["launches"] * 1e-3
    achieved = per_launch_bytes / per_launch_s / 1e9
    return {
        "kernel": name, "bound": "hbm", "achieved": achieved, "peak": p["hbm_gbs"], "unit": "GB/s",
        "frac": achieved / p["hbm_gbs"], "peak_source": p["source"], "traffic": traffic,
        "algorithmic_bytes_per_launch": per_launch_bytes, "us_per_launch": per_launch_s * 1e6,
        "launches": s["launches"],
    }


def table(stats: dict):
    total = sum(v["ms"] for v in stats.values()) or 1.0
    rows = []
    for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"]):
        gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 and v["bytes"] > 0 else None
        rows.append({"kernel": k, "launches": v["launches"], "ms": round(v["ms"], 3),
                     "share": round(v["ms"] / total, 4), "GB/s": round(gbs, 1) if gbs else None})
    return rows
