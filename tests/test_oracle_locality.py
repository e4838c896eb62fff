"""Locality of the oracle's operator and step, which the full-size GPU parity
test relies on: L(U) at a cell (its conserved values and its lower faces)
depends only on the state within 2 cells of it -- PLM reaches 2 cells along
the normal, the edge EMFs one row across, which the neighbouring faces' PLM
stencils already cover -- and one RK2 step within 4.  An outflow sub-box cut
from a periodic state around the cell reproduces the full periodic result at
its centre exactly from those radii on, and not below them."""
import numpy as np

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, subbox


def _box():
    return I.random_state((17, 16, 18), seed=77, bc=(0, 0, 0), noise=0.3)


def _centres(b, seed=5, n=10):
    rng = np.random.default_rng(seed)
    return [(0, 0, 0), (b.nx - 1, b.ny - 1, b.nz - 1)] + \
        [(int(rng.integers(b.nx)), int(rng.integers(b.ny)), int(rng.integers(b.nz))) for _ in range(n)]


def _matches(b, fn, ref_c, ref_f, centre, h):
    i, j, k = centre
    cfg, c, f = subbox(b.cell, b.face, (b.nx, b.ny, b.nz), centre, h, (b.dx, b.dy, b.dz), b.gamma)
    sc, sf = fn(cfg, c, f)
    return np.array_equal(sc[:, h, h, h], ref_c[:, k, j, i]) and all(sf[d][h, h, h] == ref_f[d][k, j, i]
                                                                     for d in range(3))


def test_operator_is_local_to_radius_2():
    b = _box()
    du, db = O.rhs(ocfg(b), b.cell, b.face)
    for c in _centres(b):
        for h in (2, 4):
            assert _matches(b, O.rhs, du, db, c, h), (c, h)
    assert not all(_matches(b, O.rhs, du, db, c, 1) for c in _centres(b))


def test_step_is_local_to_radius_4():
    b = _box()
    dt = O.cfl_dt(ocfg(b), b.cell, b.face)
    rc, rf = O.step_dts(ocfg(b), b.cell, b.face, [dt])
    step = lambda cfg, c, f: O.step_dts(cfg, c, f, [dt])  # noqa: E731
    cs = _centres(b, n=4)
    for c in cs:
        for h in (4, 7):
            assert _matches(b, step, rc, rf, c, h), (c, h)
    assert not all(_matches(b, step, rc, rf, c, 3) for c in cs)


def test_rk3_step_is_local_to_radius_6():
    b = _box()
    cfg = ocfg(b, integrator="rk3")
    dt = O.cfl_dt(cfg, b.cell, b.face)
    rc, rf = O.step_dts(cfg, b.cell, b.face, [dt])

    def step(cfg_s, c, f):
        cfg_s.integrator = "rk3"
        return O.step_dts(cfg_s, c, f, [dt])

    cs = _centres(b, n=3)
    for c in cs:
        assert _matches(b, step, rc, rf, c, 6), c
    assert not all(_matches(b, step, rc, rf, c, 5) for c in cs)


def test_clamped_subbox_on_an_outflow_domain():
    # 2D outflow domain: a sub-box clamped to the domain (its sides that meet
    # the domain edge are the domain's boundary) reproduces the full step at
    # its sample, near the edges and the corners too
    b = I.riemann_2d(40, seed=9)
    cfg = ocfg(b, riemann=O.HLL)
    dt = O.cfl_dt(cfg, b.cell, b.face)
    rc, rf = O.step_dts(cfg, b.cell, b.face, [dt])
    n, h = b.nx, 7
    for (i, j) in [(0, 0), (1, 38), (39, 39), (20, 19), (5, 33)]:
        lx, hx, ly, hy = max(0, i - h), min(n, i + h + 1), max(0, j - h), min(n, j + h + 1)
        sub = O.Config(hx - lx, hy - ly, 1, b.dx, b.dy, b.dz, b.gamma, 0.4, (O.OUTFLOW, O.OUTFLOW, O.PERIODIC),
                       riemann=O.HLL)
        c = np.ascontiguousarray(b.cell[:, :, ly:hy, lx:hx])
        f = [np.ascontiguousarray(b.face[0][:, ly:hy, lx:hx + 1]), np.ascontiguousarray(b.face[1][:, ly:hy + 1, lx:hx]),
             np.ascontiguousarray(b.face[2][:, ly:hy, lx:hx])]
        sc, sf = O.step_dts(sub, c, f, [dt])
        assert np.array_equal(sc[:, 0, j - ly, i - lx], rc[:, 0, j, i]), (i, j)
        for d in range(3):
            assert sf[d][0, j - ly, i - lx] == rf[d][0, j, i], (i, j, d)
