"""Host logic of the measurement and tuning helpers (no GPU): the roofline
arithmetic the bench reports, and the autotuner's choice, application and JSON
cache with a stand-in context and stand-in profiler timings."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_1808_01829_gb300 import autotune, roofline


def test_roofline_entry_and_table():
    stats = {"hop_fp32": {"launches": 4, "ms": 0.4, "bytes": 4 * 250e6},
             "nxn": {"launches": 10, "ms": 0.1, "bytes": 0.0}}
    peak = {"hbm_gbs": 5000.0, "source": "of test"}
    e = roofline.entry(stats, "hop_fp32", peak=peak)
    assert e["us_per_launch"] == pytest.approx(100.0)
    assert e["algorithmic_bytes_per_launch"] == pytest.approx(250e6)
    assert e["achieved"] == pytest.approx(2500.0)          # 250 MB in 100 us
    assert e["frac"] == pytest.approx(0.5) and e["peak_source"] == "of test"
    rows = roofline.table(stats)
    assert [r["kernel"] for r in rows] == ["hop_fp32", "nxn"]
    assert rows[0]["share"] == pytest.approx(0.8) and rows[0]["GB/s"] == pytest.approx(2500.0)
    assert rows[1]["GB/s"] is None


class FakeCtx:
    def __init__(self):
        self.dims = (4, 4, 4, 4)
        self.device = torch.device("cpu")
        self.tune = {}
        self.solves = 0

    def tune_set(self, k, v):
        self.tune[int(k)] = int(v)

    def apply_mdagm_mrhs(self, X, sigma, precision):
        return X

    def block_multishift_cg(self, X, shifts, tol, max_iter=0, precision="mixed", allow_not_converged=False):
        self.solves += 1
        return X, None


def test_autotune_picks_applies_and_caches(tmp_path, monkeypatch):
    ctx = FakeCtx()
    hop_us = {3: 70.0, 4: 60.0}                  # RHMC_TUNE_HOP_STAGED candidates
    gram_us = {0: 37.0, 1: 38.0, 2: 41.0, 3: 36.0}  # RHMC_TUNE_GRAM_TILE candidates
    base_us = {0: 90.0, 1: 99.0, 2: 95.0, 3: 97.0}  # RHMC_TUNE_BASE_TILE candidates
    calls = []
    cur = {"ctx": ctx}  # the context being tuned

    def fake_profile(fn):
        c = cur["ctx"]
        solves = c.solves
        fn()
        calls.append(dict(c.tune))
        if c.solves > solves:  # a short solve ran: Gram and base-step timings
            g, b = c.tune.get(autotune.KEY_GRAM_TILE, 0), c.tune.get(autotune.KEY_BASE_TILE, 0)
            return {"gram_fp32": {"launches": 2, "ms": 2 * gram_us[g] * 1e-3, "bytes": 1e6},
                    "update_shifts_fp32": {"launches": 2, "ms": 2 * base_us[b] * 1e-3, "bytes": 1e6}}
        m = c.tune[autotune.KEY_HOP]
        return {"hop_fp32": {"launches": 5, "ms": 5 * hop_us[m] * 1e-3, "bytes": 5e8}}

    monkeypatch.setattr(autotune.roofline, "profile", fake_profile)
    cache = str(tmp_path / "sub" / "tune.json")
    want = {autotune.KEY_HOP: 4, autotune.KEY_GRAM_TILE: 3, autotune.KEY_BASE_TILE: 0}
    s = autotune.tune(ctx, 16, shifts=[0.1, 0.2], cache=cache)
    assert s == want
    assert all(ctx.tune[k] == v for k, v in want.items())
    with open(cache) as f:
        db = json.load(f)
    assert list(db.values()) == [{str(k): v for k, v in want.items()}]
    # a second call reads the cache: no timing, same settings applied to a new context
    n_calls = len(calls)
    ctx2 = FakeCtx()
    cur["ctx"] = ctx2
    assert autotune.tune(ctx2, 16, shifts=[0.1, 0.2], cache=cache) == s
    assert len(calls) == n_calls and ctx2.tune == want
    autotune.reset(ctx2)
    assert ctx2.tune == {k: 0 for k in want}
    # odd width: the two-RHS-per-thread hop is not a candidate
    ctx3 = FakeCtx()
    cur["ctx"] = ctx3
    s3 = autotune.tune(ctx3, 5, cache=None)
    assert s3 == {autotune.KEY_HOP: 3}
