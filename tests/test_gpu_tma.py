"""Planes by TMA in the FP32-bulk stage kernels (mixed and FP32 state).

Interior tiles of a box whose rows are a multiple of 16 bytes take their
ring planes as two tensor-copy boxes (8 primitives, 3 lower-face fields)
instead of the per-element gather.  The copy moves the same values into the
same places, so a step must give the same state bit for bit with the planes
copied either way (MHD_COPY_AUTO against MHD_COPY_GATHER), and the handle's
counter shows that TMA planes were used.  Parity with the oracle on such a
box is checked at the FP32-bulk bar, with the oracle's FP32-form thresholds.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, state_errors

pytestmark = pytest.mark.gpu


def _steps(box, precision, copy, dts, integrator="rk2"):
    from paper_2606_12753_gb300 import mhd
    with mhd.Solver(box, precision=precision, plane_copy=copy, integrator=integrator) as s:
        s.set_state(box.cell, box.face)
        for dt in dts:
            s.step(dt, 1)
        c, f = s.get_state()
        st = s.stats()
    assert st["status"] == 0, st
    return c, f, st


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("bc", [(0, 0, 0), (0, 0, 1), (1, 1, 1)])
def test_tma_planes_equal_the_gather_bitwise(precision, bc):
    # 64 x 40 x 21: with 16 x 8 tiles, the x tiles at 16 and 32 and the y
    # tiles at 8, 16, 24 are interior; 21 planes leave a ragged z chunk
    box = I.random_state((64, 40, 21), seed=71, bc=bc)
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    dts = [dt, 0.9 * dt]
    c0, f0, st0 = _steps(box, precision, "gather", dts)
    c1, f1, st1 = _steps(box, precision, "auto", dts)
    assert st0["tma_planes"] == 0
    assert st1["tma_planes"] > 0
    np.testing.assert_array_equal(c1, c0)
    for d in range(3):
        np.testing.assert_array_equal(f1[d], f0[d])


def test_tma_planes_equal_the_gather_bitwise_rk3():
    box = I.random_state((48, 32, 18), seed=72)
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    c0, f0, _ = _steps(box, "mixed", "gather", [dt], integrator="rk3")
    c1, f1, st = _steps(box, "mixed", "auto", [dt], integrator="rk3")
    assert st["tma_planes"] > 0
    np.testing.assert_array_equal(c1, c0)
    for d in range(3):
        np.testing.assert_array_equal(f1[d], f0[d])


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_tma_box_matches_the_oracle(precision):
    box = I.random_state((48, 40, 20), seed=73)
    cfg = ocfg(box, precision)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    dts = [dt, 0.95 * dt, 0.9 * dt]
    rc, rf = O.step_dts(cfg, box.cell, box.face, dts)
    c, f, st = _steps(box, precision, "auto", dts)
    assert st["tma_planes"] > 0
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-5, errs


def test_no_tma_where_rows_break_the_16_byte_rule():
    # 37 cells per row: 148-byte rows are not a multiple of 16 bytes
    box = I.random_state((37, 24, 12), seed=74)
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    _, _, st = _steps(box, "mixed", "auto", [dt])
    assert st["tma_planes"] == 0
