"""The benchmark's reference arm (`bench.py --impl reference`) runs on host
cores only: its one JSON line carries the contract's keys, times whole
measured oracle solves (nothing extrapolated) and declares no host-device
traffic.  Run in-process on an 8^4 lattice so that the CPU suite stays short;
the 32^4 workload runs the same code."""

import json
import types

import pytest


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    import bench
    monkeypatch.setattr(bench, "DIMS", (8, 8, 8, 8))
    monkeypatch.setattr(bench, "KAPPA", 0.12)
    args = types.SimpleNamespace(steps=3, warmup=3, gpus=1)
    assert bench.run_reference(args, 0) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["higher_is_better"] is False and r["unit"] == "s"
    for k in ("metric", "value", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "vs_baseline", "dtype",
              "data", "config"):
        assert k in r, k
    assert r["value"] > 0 and r["steps"] == 3 and r["n_gpus"] == 1 and r["all_timed_solves_converged"]
    assert abs(r["ms_per_step"] - 1e3 * r["value"]) <= 1.0   # value is rounded to 1 ms
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"]
    assert "3 whole plain FP64 BiCGStab solves" in cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_stops_at_its_time_budget(monkeypatch, capsys):
    """Timed solves stop once their sum reaches the budget; the line reports
    the steps actually timed next to the steps requested."""
    import bench
    monkeypatch.setattr(bench, "DIMS", (8, 8, 8, 8))
    monkeypatch.setattr(bench, "KAPPA", 0.12)
    args = types.SimpleNamespace(steps=20, warmup=1, gpus=1)
    assert bench.run_reference(args, 0, budget_s=1e-9) == 0
    r = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert r["steps"] == 1 and r["steps_requested"] == 20


def test_reference_arm_other_ranks_do_nothing(capsys):
    import bench
    assert bench.run_reference(types.SimpleNamespace(steps=1, warmup=1, gpus=2), 1) == 0
    assert capsys.readouterr().out == ""
