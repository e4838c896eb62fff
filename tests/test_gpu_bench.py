"""bench.py on the GPU: a run whose clocks rule it out is measured once
more, with the first run's clocks kept in the line."""
import json
import sys

import pytest

import bench

pytestmark = pytest.mark.gpu


def test_disqualified_run_is_measured_again(monkeypatch, capsys):
    calls = []

    def first_run_only(clocks):
        calls.append(clocks)
        return len(calls) == 1

    monkeypatch.setattr(bench, "clocks_disqualify", first_run_only)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--n", "64", "--steps", "2", "--warmup", "1", "--no-extras"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert len(calls) == 1   # decided once, after the first timed run
    assert line["value"] > 0 and line["steps"] == 2
    # the line's contract: every key present, whatever its value at this size
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks", "e2e"):
        assert k in line, k
    assert "workload" in line["config"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    assert line["gpu_launches"] == 2 * 2 and line["higher_is_better"] is True
    if line["clocks"] is not None:   # nvidia-smi present
        assert "remeasured_after" in line["clocks"]
