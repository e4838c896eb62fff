"""SSP-RK3 (Shu & Osher) on the GPU against the oracle's RK3 step: FP64 at
1e-12 over several steps (several tiles and z-chunks, ragged tails,
periodic and outflow axes), mixed and FP32 at 1e-5, the CFL dt taken on the
device each step, and a uniform state."""
import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, state_errors

pytestmark = pytest.mark.gpu


def _gpu(box, precision, dts=None, nsteps=None, tile=(16, 8, 6)):
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, tile=tile, integrator="rk3")
    s.set_state(box.cell, box.face)
    used = []
    if dts is not None:
        for h in dts:
            s.step(float(h), 1)
    else:
        for _ in range(nsteps):
            used.append(s.cfl_dt())
            s.step(-1.0, 1)
    out = s.get_state()
    st = s.stats()
    s.close()
    assert st["status"] == 0
    return out, used


def _oracle(box, dts, precision=None):
    cfg = ocfg(box, precision, integrator="rk3")
    return O.step_dts(cfg, box.cell, box.face, dts)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (1, 0, 1)])
def test_rk3_fp64_matches_oracle(bc):
    box = I.random_state((37, 21, 13), seed=31, bc=bc)
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    dts = [dt, 0.9 * dt, 0.8 * dt]
    (c, f), _ = _gpu(box, "fp64", dts)
    rc, rf = _oracle(box, dts)
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_rk3_reduced_precision_matches_oracle(precision):
    box = I.random_state((37, 21, 13), seed=32, bc=(0, 0, 0))
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    dts = [dt, dt]
    (c, f), _ = _gpu(box, precision, dts)
    rc, rf = _oracle(box, dts, precision)
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-5, errs


def test_rk3_self_computed_dt_matches_oracle():
    box = I.random_state((24, 17, 19), seed=33, bc=(0, 0, 0))
    (c, f), used = _gpu(box, "fp64", nsteps=3)
    cfg = ocfg(box, integrator="rk3")
    rc, rf, odts = O.step(cfg, box.cell, box.face, -1.0, nsteps=3)
    np.testing.assert_allclose(used, odts, rtol=1e-13)
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs


def test_rk3_uniform_state():
    box = I.uniform_state((19, 10, 9))
    (c, f), _ = _gpu(box, "fp64", [1e-3] * 3)
    np.testing.assert_allclose(c, box.cell, rtol=1e-15, atol=1e-16)
    for d in range(3):
        np.testing.assert_allclose(f[d], box.face[d], rtol=1e-15, atol=1e-16)


def test_rk3_and_rk2_differ_and_rk3_profile_has_three_stages():
    from paper_2606_12753_gb300 import mhd
    box = I.random_state((32, 16, 16), seed=34, bc=(0, 0, 0))
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    s = mhd.Solver(box, precision="mixed", integrator="rk3")
    s.set_state(box.cell, box.face)
    s.set_profiling(True)
    s.step(dt, 2)
    ms, n = s.profile()
    c3, _ = s.get_state()
    s.close()
    assert n == [2, 2, 2] and all(t > 0 for t in ms)
    s = mhd.Solver(box, precision="mixed")
    s.set_state(box.cell, box.face)
    s.set_profiling(True)
    s.step(dt, 2)
    ms, n = s.profile()
    c2, _ = s.get_state()
    s.close()
    assert n == [2, 2, 0]
    assert not np.array_equal(c2, c3)
