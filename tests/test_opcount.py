"""The operation-counting build of the oracle (oracle/opcount.cpp), which
gives the algorithmic flops per cell-update the benchmark's arithmetic
rooflines use.  Pins: it computes bit-identical results to the oracle; the
cubic fit over tiled periodic patterns recovers exact per-cell counts where
the definition fixes them (primitive recovery of Sec. 2.2, the RK2 Heun
accumulation); the benchmark's constants equal the committed table."""
import json
import os
import re

import numpy as np
import pytest

import oracle as O
from oracle import opcount as OC
from paper_2606_12753_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _small(integrator="rk2"):
    b = I.turbulence_3d(8, seed=2606)
    cfg = O.Config(8, 8, 8, b.dx, b.dy, b.dz, gamma=b.gamma, integrator=integrator)
    return b, cfg, O.cfl_dt(cfg, b.cell, b.face)


def test_counting_build_is_bit_identical():
    b, cfg, dt = _small()
    c1, f1 = O.step_dts(cfg, b.cell, b.face, [dt])
    d1 = O.rhs(cfg, b.cell, b.face)
    with OC.counting() as read:
        c2, f2 = O.step_dts(cfg, b.cell, b.face, [dt])
        d2 = O.rhs(cfg, b.cell, b.face)
        n = read()
    assert np.array_equal(c1, c2) and all(np.array_equal(x, y) for x, y in zip(f1, f2))
    assert np.array_equal(d1[0], d2[0]) and all(np.array_equal(x, y) for x, y in zip(d1[1], d2[1]))
    assert n["add"] > 0 and n["mul"] > 0 and n["div"] > 0 and n["sqrt"] > 0
    # an outflow box with every HLLD region as well
    rb = I.random_state((6, 5, 4), seed=3, bc=(1, 0, 1))
    rcfg = O.Config(6, 5, 4, rb.dx, rb.dy, rb.dz, gamma=rb.gamma, bc=(1, 0, 1))
    a1 = O.step_dts(rcfg, rb.cell, rb.face, [1e-3])
    with OC.counting():
        a2 = O.step_dts(rcfg, rb.cell, rb.face, [1e-3])
    assert np.array_equal(a1[0], a2[0]) and all(np.array_equal(x, y) for x, y in zip(a1[1], a2[1]))


def test_primitive_recovery_count_per_cell():
    """Sec. 2.2's recovery, per cell: B_c = (B_lo + B_hi)/2 on 3 axes, formed
    once for the pressure and once for the primitive array (6 add, 6 mul);
    p = (gamma-1)(E - |m|^2/(2 rho) - |B_c|^2/2) (7 add incl. gamma-1, 9 mul,
    1 div); v = m/rho (3 div); the rho and p floors (2 compares)."""
    b, cfg, dt = _small()
    pc = OC.per_cell(cfg, b.cell, b.face, dt)
    # two operator evaluations per RK2 step
    assert pc["prims"] == pytest.approx({"add": 26, "mul": 30, "div": 8, "sqrt": 0, "cmp": 4, "misc": 0},
                                        abs=1e-6)


@pytest.mark.parametrize("integrator,expect", [("rk2", 48.0), ("rk3", 96.0)])
def test_rk_accumulation_count_per_cell(integrator, expect):
    """Heun: U* = U + dt L (2 flops), U^{n+1} = (U + U* + dt L)/2 (4 flops);
    Shu-Osher SSP-RK3: 2 + 5 + 5 flops; for 5 cell values and 3 faces per cell."""
    b, cfg, dt = _small(integrator)
    sp = OC.split(OC.per_cell(cfg, b.cell, b.face, dt))
    assert sp["rk_accumulate"] == pytest.approx(expect, abs=1e-6)
    assert sp["total"] == pytest.approx(sp["operators"] + sp["rk_accumulate"] + sp["cfl"])


def test_bench_constants_match_the_table():
    with open(os.path.join(ROOT, "oracle", "opcount_table.json")) as f:
        tab = json.load(f)["workloads"]
    src = open(os.path.join(ROOT, "bench.py")).read()
    block = src[src.index("FLOPS = {"):src.index("}\n", src.index("FLOPS = {")) + 1]
    rows = re.findall(r'\("(\w+)", "(\w+)", "(\w+)"\): \{"total": ([\d.]+), "fp64_in_mixed": ([\d.]+)\}', block)
    assert len(rows) == 4
    names = {("turbulence", "primitive", "rk2"): "turbulence_3d (RK2, PLM-MC primitive, HLLD, upwind CT)",
             ("turbulence", "characteristic", "rk2"): "turbulence_3d (RK2, PLM-MC characteristic, HLLD, upwind CT)",
             ("orszag_tang", "primitive", "rk2"): "orszag_tang_3d (RK2, PLM-MC primitive, HLLD, upwind CT)",
             ("orszag_tang", "primitive", "rk3"): "orszag_tang_3d (SSP-RK3, PLM-MC primitive, HLLD, upwind CT)"}
    for kind, recon, integ, total, f64 in rows:
        ref = tab[names[(kind, recon, integ)]]["flops"]
        assert float(total) == pytest.approx(ref["total"], abs=1e-3)
        assert float(f64) == pytest.approx(ref["fp64_in_mixed"], abs=1e-3)
