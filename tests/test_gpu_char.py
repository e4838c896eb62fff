"""Characteristic reconstruction (MHD_RECON_CHARACTERISTIC) on the GPU
against the oracle's characteristic mode: FP64 at 1e-12 over several steps
(periodic and outflow axes, ragged tiles) and for the operator alone, mixed
and FP32 at 1e-5, and a state whose field lies along x (B_t = 0 in the x
sweeps, B_n = 0 in the y and z sweeps: the degenerate eigenvector
branches)."""
import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, state_errors

pytestmark = pytest.mark.gpu


def _gpu_steps(box, precision, dts):
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, recon="characteristic", tile=(16, 8, 5))
    s.set_state(box.cell, box.face)
    for h in dts:
        s.step(float(h), 1)
    out = s.get_state()
    st = s.stats()
    s.close()
    assert st["status"] == 0
    return out


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (0, 1, 0)])
def test_char_fp64_matches_oracle(bc):
    box = I.random_state((37, 21, 13), seed=41, bc=bc)
    cfg = ocfg(box, recon=1)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    dts = [dt, 0.9 * dt, 0.8 * dt]
    c, f = _gpu_steps(box, "fp64", dts)
    rc, rf = O.step_dts(cfg, box.cell, box.face, dts)
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_char_reduced_precision_matches_oracle(precision):
    box = I.random_state((37, 21, 13), seed=42, bc=(0, 0, 0))
    cfg = ocfg(box, precision, recon=1)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    c, f = _gpu_steps(box, precision, [dt, dt])
    rc, rf = O.step_dts(cfg, box.cell, box.face, [dt, dt])
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-5, errs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_char_operator_matches_oracle(precision):
    from paper_2606_12753_gb300 import mhd
    box = I.random_state((29, 21, 13), seed=43, bc=(0, 0, 0), noise=0.0)
    du, db = O.rhs(ocfg(box, precision, recon=1), box.cell, box.face)
    s = mhd.Solver(box, precision=precision, recon="characteristic", tile=(16, 8, 6))
    s.set_state(box.cell, box.face)
    gc, gf = s.rhs()
    s.close()
    errs = state_errors(gc, gf, du, db)
    assert max(errs.values()) <= (1e-12 if precision == "fp64" else 1e-5), errs


def test_char_degenerate_field_along_x():
    box = I.random_state((33, 17, 12), seed=44, bc=(0, 0, 0), bamp=0.0, b0=(0.6, 0.0, 0.0))
    assert np.all(box.face[1] == 0) and np.all(box.face[2] == 0)
    cfg = ocfg(box, recon=1)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    c, f = _gpu_steps(box, "fp64", [dt, dt])
    rc, rf = O.step_dts(cfg, box.cell, box.face, [dt, dt])
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs
    # and the characteristic step differs from the primitive one there
    r0, _ = O.step_dts(ocfg(box), box.cell, box.face, [dt, dt])
    assert not np.array_equal(rc, r0)
