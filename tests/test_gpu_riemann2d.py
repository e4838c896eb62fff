"""The HLL 2D Riemann workload (a seeded four-quadrant MHD stand-in, outflow
in x and y, one periodic z cell) against the oracle: FP64 at 1e-12 and mixed
at 1e-5 on a ragged grid over several steps, and at full size (3200^2) on
sampled cells.  On an outflow domain a sample's sub-box is clamped to the
domain, so a side that meets the domain edge is the domain's own boundary."""
import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, state_errors, thresholds

pytestmark = pytest.mark.gpu


def _run(box, precision, dts):
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, riemann="hll")
    s.set_state(box.cell, box.face)
    for h in dts:
        s.step(float(h), 1)
    out = s.get_state()
    s.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_riemann2d_hll_matches_oracle(precision):
    box = I.riemann_2d(97, seed=8)
    cfg = ocfg(box, precision, riemann=O.HLL)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    dts = [dt] * 4
    c, f = _run(box, precision, dts)
    rc, rf = O.step_dts(cfg, box.cell, box.face, dts)
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= (1e-12 if precision == "fp64" else 1e-5), errs


def _subbox2d(box, centre, h, precision=None):
    i, j = centre
    n = box.nx
    lo_x, hi_x = max(0, i - h), min(n, i + h + 1)
    lo_y, hi_y = max(0, j - h), min(n, j + h + 1)
    cell = np.ascontiguousarray(box.cell[:, :, lo_y:hi_y, lo_x:hi_x])
    bx = np.ascontiguousarray(box.face[0][:, lo_y:hi_y, lo_x:hi_x + 1])
    by = np.ascontiguousarray(box.face[1][:, lo_y:hi_y + 1, lo_x:hi_x])
    bz = np.ascontiguousarray(box.face[2][:, lo_y:hi_y, lo_x:hi_x])
    cfg = O.Config(hi_x - lo_x, hi_y - lo_y, 1, box.dx, box.dy, box.dz, box.gamma, 0.4,
                   (O.OUTFLOW, O.OUTFLOW, O.PERIODIC), riemann=O.HLL, thresholds=thresholds(precision))
    return cfg, cell, [bx, by, bz], (i - lo_x, j - lo_y)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_riemann2d_hll_at_3200_sampled(precision):
    n = 3200
    box = I.riemann_2d(n, seed=3200)
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, riemann="hll")
    s.set_state(box.cell, box.face)
    dt = s.cfl_dt()
    s.step(dt, 1)
    c, f = s.get_state()
    s.close()
    rng = np.random.default_rng(3200)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n // 2 - 1, n // 2), (n // 2, n // 2 - 1), (15, 16), (16, 7),
           (1, n // 2), (n // 2, 2)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(12)]
    got_c, ref_c, got_f, ref_f = [], [], [], []
    for (i, j) in pts:
        cfg, cell, face, (ci, cj) = _subbox2d(box, (i, j), 7, precision)
        rc, rf = O.step_dts(cfg, cell, face, [dt])
        ref_c.append(rc[:, 0, cj, ci])
        got_c.append(c[:, 0, j, i])
        ref_f.append([rf[0][0, cj, ci], rf[1][0, cj, ci], rf[2][0, cj, ci]])
        got_f.append([f[0][0, j, i], f[1][0, j, i], f[2][0, j, i]])
    got_c, ref_c, got_f, ref_f = map(np.array, (got_c, ref_c, got_f, ref_f))
    errs = {v: float(np.abs(got_c[:, v] - ref_c[:, v]).sum() / np.abs(ref_c[:, v]).sum()) for v in range(5)}
    errs.update({5 + d: float(np.abs(got_f[:, d] - ref_f[:, d]).sum() / np.abs(ref_f[:, d]).sum()) for d in range(3)})
    assert max(errs.values()) <= (1e-12 if precision == "fp64" else 1e-5), errs
