"""bench.py's reference arm on the CPU: the oracle baseline sample runs on one host core, and
`--impl reference` prints one JSON line with the keys the contract fixes (impl, metric, value,
unit, steps, warmup, ms_per_step, higher_is_better, cpu_baseline of kind "oracle", e2e without
host copies).  Under several ranks only rank 0 prints."""
from __future__ import annotations

import argparse
import io
import json
from contextlib import redirect_stdout

import bench


def test_cpu_baseline_sample_runs_the_oracle_on_one_core():
    d = bench.cpu_baseline(1.0)
    assert d["kind"] == "oracle" and d["cores"] == 1 and d["unit"] == bench.UNIT
    assert d["value"] is not None and d["value"] > 0
    assert "fine primal + adjoint slices" in d["sample"] and "BLAS threads = 1" in d["sample"]


def _args(steps=2, warmup=3):
    return argparse.Namespace(steps=steps, warmup=warmup, gpus=1, impl="reference")


def test_reference_arm_prints_one_contract_line(monkeypatch):
    calls = []

    def fake(budget):
        calls.append(budget)
        return {"value": 1.0e6 + len(calls), "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "s"}

    monkeypatch.setattr(bench, "cpu_baseline", fake)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(_args())
    lines = [ln for ln in out.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert len(calls) == 5                                   # 3 warm-up samples, then 2 timed ones
    assert 2.0 <= calls[0] <= 20.0                           # a bounded sample per step
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["value"] == (1.0e6 + 4 + 1.0e6 + 5) / 2      # the mean of the timed samples
    assert line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith(bench.WORKLOAD)


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    monkeypatch.setattr(bench, "cpu_baseline", lambda budget: (_ for _ in ()).throw(AssertionError("ran")))
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(_args())
    assert out.getvalue().strip() == ""


def _fake_counters():
    kinds = ("fine_primal", "coarse_primal", "correct_primal", "fine_adjoint", "coarse_adjoint", "correct_adjoint")
    stats = {"by_kind": {k: {"solves": 32.0, "cg_iters": 320.0, "refinements": 32.0} for k in kinds}}
    kind_ms = {k: 1.0 + i for i, k in enumerate(kinds)}          # correct_adjoint dominates
    return kind_ms, stats


def test_roofline_bytes_follow_the_per_dof_rule(monkeypatch):
    monkeypatch.setattr(bench, "stepper_sources_sha16", lambda: bench.NCU_TRAFFIC["sources_sha16"])
    kind_ms, stats = _fake_counters()
    r = bench.roofline(kind_ms, stats, 1000, 2, "fp32_refine")
    assert r["kernel"] == "correct_adjoint" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    per_launch = 1000 * ((16 + 8) * 32 + 36 * 320 + 28 * 32) / 2   # adjoint solves read T_j too
    assert r["algorithmic_bytes_per_launch"] == per_launch
    assert abs(r["achieved"] - per_launch / 6e-3 / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert r["per_kernel"]["fine_primal"]["algorithmic_bytes"] == 1000 * (16 * 32 + 36 * 320 + 28 * 32) / 2
    assert r["traffic"] == bench.NCU_TRAFFIC["bytes"]["correct_adjoint"]


def test_stored_traffic_is_reported_only_for_its_workload_and_precision(monkeypatch):
    monkeypatch.setattr(bench, "stepper_sources_sha16", lambda: bench.NCU_TRAFFIC["sources_sha16"])
    kind_ms, stats = _fake_counters()
    for workload, precision in (("diff256", "fp32_refine"), ("loop512", "fp32_refine"), (bench.WORKLOAD, "fp64")):
        r = bench.roofline(kind_ms, stats, 1000, 1, precision, workload)
        assert r["traffic"] is None and "no ncu capture of this workload" in r["traffic_source"]
    monkeypatch.setattr(bench, "stepper_sources_sha16", lambda: "0000000000000000")
    r = bench.roofline(kind_ms, stats, 1000, 1, "fp32_refine")
    assert r["traffic"] is None and "current stepper sources" in r["traffic_source"]
