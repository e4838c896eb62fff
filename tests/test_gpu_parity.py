"""GPU parity: the CUDA stage kernels through the C ABI against the FP64 oracle.

Tolerances (relative L1 per variable, both sides given the same dt sequence):
1e-12 for the FP64 path, 1e-5 for the mixed FP32/FP64 and FP32 paths.
Sizes span several tiles in x, y and z and leave ragged tails.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, state_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 1e-5}


def run_gpu(box, dts, precision="fp64", **kw):
    from paper_2606_12753_gb300 import mhd
    with mhd.Solver(box, precision=precision, **kw) as s:
        s.set_state(box.cell, box.face)
        for dt in dts:
            s.step(dt, 1)
        c, f = s.get_state()
        st = s.stats()
    assert s.h is None   # the handle is destroyed on leaving the block
    return c, f, st


def check(box, nsteps, precision, tol=None, emf=0, **kw):
    cfg = ocfg(box, precision, emf_mean=emf)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    dts = [dt * (1.0 - 0.05 * s) for s in range(nsteps)]
    rc, rf = O.step_dts(cfg, box.cell, box.face, dts)
    c, f, st = run_gpu(box, dts, precision, emf="mean" if emf else "upwind", **kw)
    errs = state_errors(c, f, rc, rf)
    t = tol if tol is not None else TOL[precision]
    bad = {k: v for k, v in errs.items() if not v <= t}
    assert not bad, f"{precision} {box.name}: errors above {t}: {bad} (all: {errs})"
    assert st["status"] == 0
    return errs


@pytest.mark.parametrize("tile", [(16, 8, 32), (8, 8, 5), (24, 8, 7)])
def test_fp64_periodic_3d_one_step(tile):
    box = I.random_state((37, 29, 19), seed=11)
    check(box, 1, "fp64", tile=tile)


def test_fp64_periodic_3d_multi_step():
    box = I.random_state((34, 21, 18), seed=12)
    check(box, 6, "fp64", tile=(16, 8, 8))


@pytest.mark.parametrize("bc", [(1, 1, 1), (1, 0, 1), (0, 1, 0)])
def test_fp64_outflow(bc):
    box = I.random_state((26, 19, 13), seed=13, bc=bc)
    check(box, 3, "fp64", tile=(16, 8, 6))


def test_fp64_mean_emf():
    box = I.random_state((20, 17, 11), seed=14)
    check(box, 2, "fp64", emf=1, tile=(16, 8, 4))


def test_fp64_hll():
    box = I.random_state((20, 17, 11), seed=15)
    cfg = ocfg(box, riemann=O.HLL)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    rc, rf = O.step_dts(cfg, box.cell, box.face, [dt, dt])
    c, f, _ = run_gpu(box, [dt, dt], "fp64", riemann="hll")
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs


def test_fp64_orszag_tang_2d():
    box = I.orszag_tang_2d(64)
    check(box, 20, "fp64")


def test_fp64_degenerate_axes():
    # 1D along each axis, 2D, and boxes smaller than one tile
    for dims in [(40, 1, 1), (1, 33, 1), (1, 1, 30), (5, 3, 2), (3, 40, 1)]:
        box = I.random_state(dims, seed=sum(dims))
        check(box, 2, "fp64")


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_reduced_precision_parity(precision):
    box = I.random_state((37, 29, 19), seed=21)
    check(box, 3, precision)


def test_mixed_outflow_and_2d():
    check(I.random_state((26, 19, 13), seed=22, bc=(1, 1, 1)), 2, "mixed")
    check(I.orszag_tang_2d(64), 10, "mixed")


def test_cfl_and_divb_reductions():
    from paper_2606_12753_gb300 import mhd
    for bc in [(0, 0, 0), (1, 1, 1)]:
        box = I.random_state((23, 17, 9), seed=31, bc=bc)
        cfg = ocfg(box)
        s = mhd.Solver(box, precision="fp64")
        s.set_state(box.cell, box.face)
        assert s.cfl_dt() == pytest.approx(O.cfl_dt(cfg, box.cell, box.face), rel=1e-13)
        assert s.divb_max() == pytest.approx(O.divb_max(cfg, box.face), rel=1e-6, abs=1e-12)
        s.step(-1.0, 5)
        c, f = s.get_state()
        scale = max(np.abs(x).max() for x in f) / box.dx
        assert s.divb_max() < 1e-13 * scale
        s.close()


def test_self_computed_dt_matches_oracle():
    from paper_2606_12753_gb300 import mhd
    box = I.random_state((24, 20, 10), seed=41)
    cfg = ocfg(box)
    rc, rf, dts = O.step(cfg, box.cell, box.face, -1.0, nsteps=4)
    s = mhd.Solver(box, precision="fp64")
    s.set_state(box.cell, box.face)
    s.step(-1.0, 4)
    c, f = s.get_state()
    st = s.stats()
    s.close()
    assert st["last_dt"] == pytest.approx(dts[-1], rel=1e-12)
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs


def test_uniform_state_bitwise_on_gpu():
    from paper_2606_12753_gb300 import mhd
    for prec in ("fp64", "mixed", "fp32"):
        box = I.uniform_state((19, 13, 7), bc=(1, 0, 1))
        s = mhd.Solver(box, precision=prec)
        s.set_state(box.cell, box.face)
        s.step(1e-3, 3)
        c, f = s.get_state()
        s.close()
        if prec == "fp32":
            np.testing.assert_array_equal(c, box.cell.astype(np.float32))
        else:
            np.testing.assert_array_equal(c, box.cell)
        for d in range(3):
            np.testing.assert_array_equal(f[d], box.face[d].astype(c.dtype))


def test_nonfinite_is_reported():
    from paper_2606_12753_gb300 import mhd
    box = I.random_state((16, 12, 8), seed=51)
    cell = box.cell.copy()
    cell[4, 3, 4, 5] = np.nan
    s = mhd.Solver(box, precision="fp64")
    s.set_state(cell, box.face)
    with pytest.raises(mhd.MHDError) as ei:
        s.step(1e-3, 1)
    assert ei.value.code == mhd.MHD_ERR_NONFINITE
    s.close()


def test_floor_hits_are_counted():
    """Floors are counted wherever primitives are recovered.  The oracle
    recovers U^n and U* in each step; the GPU recovers the state set from the
    host (U^0) once, then U* and U^{n+1} at the end of each stage, so over one
    step GPU = oracle + hits(U^1)."""
    from paper_2606_12753_gb300 import mhd
    box = I.random_state((16, 12, 8), seed=52)
    cell = box.cell.copy()
    # two cells with total energy below the magnetic + kinetic energy
    cell[4, 2, 3, 4] = 0.0
    cell[4, 5, 6, 7] = 0.0
    cfg = ocfg(box)
    st_step, st0, st1 = O.Stats(), O.Stats(), O.Stats()
    c1, f1, _ = O.step(cfg, cell, box.face, 1e-4, stats=st_step)
    O.rhs(cfg, cell, box.face, stats=st0)
    O.rhs(cfg, c1, f1, stats=st1)
    s = mhd.Solver(box, precision="fp64")
    s.set_state(cell, box.face)
    s.step(1e-4, 1)
    st = s.stats()
    s.close()
    assert st_step.p_floor_hits >= 2
    assert st0.p_floor_hits >= 2
    assert st["p_floor_hits"] == st_step.p_floor_hits + st1.p_floor_hits


RHS_TOL = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (1, 0, 1)])
def test_spatial_operator_parity(precision, bc):
    """L(U) alone -- reconstruction, Riemann fluxes, divergence, edge EMFs,
    -curl E -- element by element against the oracle's operator."""
    from paper_2606_12753_gb300 import mhd
    box = I.random_state((29, 21, 13), seed=61, bc=bc, noise=0.0)
    cfg = ocfg(box, precision)
    du, db = O.rhs(cfg, box.cell, box.face)
    s = mhd.Solver(box, precision=precision, tile=(16, 8, 6))
    s.set_state(box.cell, box.face)
    gc, gf = s.rhs()
    c, f = s.get_state()
    s.close()
    np.testing.assert_array_equal(c, box.cell.astype(c.dtype))      # state untouched
    errs = state_errors(gc, gf, du, db)
    tol = RHS_TOL[precision]
    assert max(errs.values()) <= tol, errs
