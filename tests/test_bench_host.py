"""Host-side logic of bench.py that needs no GPU: the clock summary (which
decides whether a run's clocks disqualify it), the comment-insensitive
kernel-source digest and the traffic lookup keyed by it."""
import datetime
import os

import pytest

import bench


def _row(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    # timestamp, index, clocks.sm, clocks.max.sm, power.draw, reasons.active, 4 named reasons
    return ", ".join([ts, "0", str(sm), "2070", "900.0", "0x0000000000000000", *reasons])


def _sampler(tmp_path, rows, t0, t1):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.proc = object()   # stands for the nvidia-smi process
    s.t0, s.t1 = t0, t1
    return s


def test_clock_summary_keeps_the_timed_region(tmp_path):
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 1.0, 1000)]                                   # warm-up, outside the window
    rows += [_row(t0 + 0.05 * i, 2070 if i % 2 else 2055) for i in range(10)]
    rows.append(_row(t0 + 0.2, 1980, ("Not Active", "Not Active", "Not Active", "Active")))
    s = _sampler(tmp_path, rows, t0, t0 + 0.5)
    out = s.summary()
    assert out["samples"] == 11 and out["window"] == "timed region"
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_widens_into_the_warm_up(tmp_path):
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 0.25, 2070, ("Active", "Not Active", "Not Active", "Not Active")),
            _row(t0 - 0.15, 2070), _row(t0 + 0.01, 2070)]
    s = _sampler(tmp_path, rows, t0, t0 + 0.02)
    out = s.summary()
    assert out["samples"] == 3 and "warm-up" in out["window"]
    assert out["reasons"] == ["hw_slowdown"]


def test_clock_summary_without_samples_is_none(tmp_path):
    s = _sampler(tmp_path, ["garbage line"], 1.0, 2.0)
    assert s.summary() is None
    s.proc = None   # nvidia-smi did not start
    assert s.summary() is None


def test_source_digest_ignores_comments(tmp_path, monkeypatch):
    from paper_2606_12753_gb300 import _build
    a = tmp_path / "a.cu"
    a.write_text("int f() { return 1; }  // one\n")
    monkeypatch.setattr(_build, "_deps", lambda: [str(a)])
    d0 = bench.kernel_source_digest()
    a.write_text("/* a comment */\nint f()   {\n  return 1;\n}\n")
    assert bench.kernel_source_digest() == d0
    a.write_text("int f() { return 2; }\n")
    assert bench.kernel_source_digest() != d0
    a.write_text("int f() { return 1; }\n")
    assert bench.kernel_source_digest() == d0
    monkeypatch.setattr(_build, "FAST_FP32_FLAGS", [])     # the same source compiled differently
    assert bench.kernel_source_digest() != d0
    monkeypatch.setattr(_build, "FAST_FP32_FLAGS", ["-prec-div=false", "-prec-sqrt=false"])
    monkeypatch.setattr(_build, "NVCC_FLAGS", [x if x != _build.CSRC else "/elsewhere/csrc" for x in _build.NVCC_FLAGS])
    assert bench.kernel_source_digest() == d0                # machine paths do not count


def test_traffic_lookup_follows_the_current_sources():
    """A capture stamped with the current digest is reported; any other
    stamp reads as no traffic figure (null in the bench line)."""
    tag = "stage_kernel<mixed,2>@turbulence_3d_256"
    value, digest = bench.traffic_from_profiles(tag)
    assert digest == bench.kernel_source_digest()
    lines = open(os.path.join(bench.ROOT, "profiles", "traffic.txt")).read().splitlines()
    stamped = [ln for ln in lines if f"kernel={tag} " in ln and f"src={digest} " in ln]
    if stamped:
        assert value is not None and value > 0
    else:
        assert value is None


def test_clocks_disqualify():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_disqualify(ok)
    assert not bench.clocks_disqualify(None)
    assert not bench.clocks_disqualify({**ok, "sm_mhz": 1700.0, "reasons": ["sw_power_cap"]})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_disqualify({**ok, "reasons": [r]})
    assert bench.clocks_disqualify({**ok, "sm_mhz": 1400.0})   # well below maximum, no reason: a clock lock


def test_profile_record_carries_the_instruction_count():
    rec, digest = bench.profile_record("stage_kernel<mixed,2>@turbulence_3d_256")
    if rec is not None:   # captured for the current sources
        assert float(rec["warp_inst_per_launch"]) > 0 and float(rec["dram_bytes_per_launch"]) > 0
    assert bench.ISSUE_PEAK_WARP_INST_PER_S == pytest.approx(152 * 4 * 2.07e9)


def test_minimum_bytes_are_the_conserved_states():
    """The roofline's bytes per cell-update: the conserved states read and
    written once per stage (FP64 8-value states; the mixed form's U* and the
    FP32 form in 4-byte values), halos from cache."""
    for prec, total in (("fp64", 320), ("mixed", 256), ("fp32", 160)):
        assert sum(bench.MIN_STAGE_BYTES[prec]) == total
    s1, s2 = bench.MIN_STAGE_BYTES["mixed"]
    assert s1 == 8 * 8 + 8 * 4 and s2 == 8 * 4 + 8 * 8 + 8 * 8
    # the design's stored primitives only add bytes
    for prec in ("fp64", "mixed", "fp32"):
        assert all(d > m for d, m in zip(bench.STAGE_BYTES[prec], bench.MIN_STAGE_BYTES[prec]))


def test_oracle_throughput_counts_every_process():
    rate, cells, el = bench.oracle_throughput(8, 2, 1, 2)
    assert cells == 2 * 2 * 8 ** 3 and el > 0
    assert rate == pytest.approx(cells / el / 1e6)
