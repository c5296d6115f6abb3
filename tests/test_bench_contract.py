"""The benchmark's JSON line carries every key of its contract, with the
right types, computed from synthetic timings (host only: no GPU work)."""
import argparse
import io
import json
from contextlib import redirect_stdout

import pytest

import bench


def _prof(ms, calls, kernels):
    return dict(ms=ms, launches=calls, kernels=kernels)


def _fake_out(steps):
    prof = {"locate": _prof(0.0, 0, 0), "field": _prof(0.037 * steps, steps, steps),
            "push": _prof(0.51 * steps, steps, 2 * steps), "finalize": _prof(0.033 * steps, steps, steps),
            "charge": _prof(0.0, 0, 0), "sort": _prof(0.082 * steps, steps // 4, 5 * (steps // 4)),
            "cross": _prof(0.15 * steps, steps, steps), "adjoint": _prof(0.0, 0, 0)}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 20}
    mixed = dict(ms=0.67 * steps, prof=prof, stats=dict(crossings=10, frozen=0, steps=steps, wait_timeouts=0),
                 counts=(117649, 795024, 1340928, 663552), clocks=clocks, e2e_s=0.8e-3 * steps,
                 h2d=17087616, d2h=6360192, levels3=None)
    fp64 = dict(ms=3.0 * steps, prof=prof, counts=mixed["counts"], clocks=clocks)
    return {"mixed": mixed, "fp64": fp64}


def test_bench_line_has_the_contract_keys(monkeypatch):
    monkeypatch.setattr(bench, "issue_roofline", lambda *a: {"kernel": "k_push_mixed_tma", "bound": "issue",
                                                             "achieved": 1.0, "peak": 2.0, "unit": "x", "frac": 0.5})
    args = argparse.Namespace(steps=100, warmup=10, workload="cube48", sort_every=4)
    cpu = {"value": 1.4e6, "unit": "particle-steps/s", "cores": 1, "kind": "oracle", "sample": "s"}
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.report(args, 1, 10_000_000, _fake_out(100), cpu, None)
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict), ("roofline", dict), ("e2e", dict),
                 ("gpu_launches", int), ("clocks", dict), ("cpu_baseline", dict)):
        assert isinstance(d[k], t), k
    assert d["vs_baseline"] is None and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["value"] == pytest.approx(10_000_000 * 100 / (0.067))
    assert "workload" in d["config"]
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    e = d["e2e"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in e, k
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
    assert d["gpu_launches"] == sum(v["kernels"] for v in _fake_out(100)["mixed"]["prof"].values())


def test_downshift_object_is_carried_when_measured(monkeypatch):
    monkeypatch.setattr(bench, "issue_roofline", lambda *a: {"frac": 0.5})
    args = argparse.Namespace(steps=10, warmup=3, workload="cube48", sort_every=4)
    out = _fake_out(10)
    out["downshift"] = {"value": 1.5e9, "unit": "particle-steps/s", "ms_per_step": 6.5}
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.report(args, 1, 10_000_000, out, None, None)
    d = json.loads(buf.getvalue().strip())
    assert d["downshift"] == out["downshift"] and "cpu_baseline" not in d


def test_downshift_algorithmic_bytes():
    counts = (117649, 795024, 1340928, 663552)
    nn, ne, nf, nt = counts
    b = bench.bytes_alg_per_step_downshift(10_000_000, counts)
    # FP64 state (52 B) plus the history the rule needs: 3 past velocities
    # (72 B) and 2 past complex E~, B~ samples (192 B), each read and written
    assert b == 10_000_000 * 2 * (52 + 3 * 24 + 2 * 12 * 8) + 72 * nt + 24 * nn + 24 * ne + 16 * nf
    # mixed forms: FP32 velocities (state 40 B), the same history in FP32
    # (132 B), complex64 DoFs
    bm = bench.bytes_alg_per_step_downshift(10_000_000, counts, "mixed")
    assert bm == 10_000_000 * 2 * (40 + 3 * 12 + 2 * 12 * 4) + 72 * nt + 24 * nn + 16 * ne + 8 * nf
    assert bm / 10_000_000 == pytest.approx(351.4, abs=0.05)


def test_algorithmic_bytes_per_step_match_the_stated_formula():
    counts = (117649, 795024, 1340928, 663552)
    nn, ne, nf, nt = counts
    b = bench.bytes_alg_per_step(10_000_000, counts, "mixed")
    assert b == 10_000_000 * 2 * 40 + 72 * nt + 24 * nn + (8 + 8) * ne + 8 * nf
    assert b / 10_000_000 == pytest.approx(87.4, abs=0.05)
    assert bench.bytes_alg_per_step(10_000_000, counts, "fp64") / 10_000_000 == pytest.approx(113.1, abs=0.05)


def test_step_fraction_variant_and_reports_are_carried(monkeypatch):
    """roofline.frac_step (whole step on the algorithmic bytes), the 24-bit
    variant's object, the per-quantity error report, the large-load legs,
    the adjoint window's HBM fractions and the FP64 rate are in the line."""
    monkeypatch.setattr(bench, "issue_roofline", lambda *a: None)
    args = argparse.Namespace(steps=100, warmup=10, workload="cube48", sort_every=4)
    out = _fake_out(100)
    out["mixed_q24"] = dict(out["mixed"], ms=0.72 * 100)
    out["errors"] = {"mixed": {"tet_agreement": 1.0}}
    out["large"] = {"jittered64": {"value": 7e9}, "large96": {"value": 1.4e10}}
    out["fp64_rate"] = 5.3e11
    out["large_adjoint"] = {"memory_plan": {"every": 5, "stash": True}}
    adj = {"particles": 4_000_000, "counts": (117649, 795024, 1340928, 663552), "steps": 50, "every": 10,
           "mixed": {"forward_particle_steps_per_s": 1.5e10, "reverse_particle_steps_per_s": 6e9}}
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.report(args, 1, 10_000_000, out, None, adj)
    d = json.loads(buf.getvalue().strip())
    b_alg = bench.bytes_alg_per_step(10_000_000, out["mixed"]["counts"], "mixed")
    assert d["roofline"]["frac_step"] == pytest.approx(b_alg / 0.67e-3 / 1e9 / d["roofline"]["peak"])
    assert d["mixed_q24"]["ms_per_step"] == pytest.approx(0.72)
    assert d["mixed_error_vs_oracle"] == out["errors"] and d["large_forward"] == out["large"]
    assert d["fp64_rate_lane_ops_per_s"] == 5.3e11
    a = d["adjoint"]["mixed"]
    assert a["hbm_frac_reverse"] == pytest.approx(6e9 * a["bytes_per_particle_step_reverse"] / 1e9 /
                                                  d["roofline"]["peak"])
    assert a["bytes_per_particle_step_reverse"] > 232
    assert d["large_adjoint"] == out["large_adjoint"]


def test_reverse_window_bytes_count_each_pass():
    """bytes_reverse_window: a stash-mode sweep is the recomputed steps plus
    one state copy per step plus the adjoint-step and segment terms; the
    recompute mode swaps the stash copies for two copies per step and adds
    the extra recomputed steps."""
    counts = (117649, 795024, 1340928, 663552)
    n, K = 4_000_000, 20
    fwd = bench.bytes_alg_per_step(n, counts, "mixed")
    st = bench.bytes_reverse_window(n, counts, "mixed", K, 5, True, K)
    rc = bench.bytes_reverse_window(n, counts, "mixed", K, 5, False, 60)
    assert rc - st == pytest.approx(40 * fwd + K * n * 2 * 41)
    adj_step = n * (40 + 13 + 72)
    per_step_mesh = 72 * 663552 + 320 * 663552 + 32 * (795024 + 1340928)
    assert st == K * fwd + K * n * 82 + K * (adj_step + per_step_mesh) + 4 * n * (82 + 72 + 4)
