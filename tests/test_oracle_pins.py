"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an exact solution of the
ideal-MHD equations, a conservation law, a symmetry of the equations, or a
convergence rate -- never against a retyped copy of the oracle's own formula.
The paper (Sec. 2.2) names the method's stages but prints no solution values,
so these are the pins: a dropped term, a wrong sign, a transposed operand or a
wrong index in any stage fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I

G = 5.0 / 3.0


def cfg_of(b, **kw):
    return O.Config(b.nx, b.ny, b.nz, b.dx, b.dy, b.dz, b.gamma, b.cfl, tuple(b.bc), **kw)


# ----------------------------------------------------------------- limiter

def test_mc_slope_closed_forms():
    # linear data: the MC slope is the exact gradient
    for a, s in [(0.3, 1.7), (-2.0, 0.25), (5.0, -3.0)]:
        assert O.mc_slope(a - s, a, a + s) == pytest.approx(s, rel=0, abs=1e-15)
    # extremum or flat: zero slope
    assert O.mc_slope(1.0, 2.0, 1.5) == 0.0
    assert O.mc_slope(3.0, 2.0, 2.5) == 0.0
    assert O.mc_slope(1.0, 1.0, 4.0) == 0.0
    # strongly one-sided data: limited by twice the smaller one-sided difference
    assert O.mc_slope(0.0, 0.1, 10.0) == pytest.approx(0.2, abs=1e-15)
    assert O.mc_slope(10.0, 9.9, 0.0) == pytest.approx(-0.2, abs=1e-15)
    # moderately uneven data: the central difference (dm+dp)/2 is smallest
    assert O.mc_slope(0.0, 1.0, 2.5) == pytest.approx(1.25, abs=1e-15)


# ----------------------------------------------------------------- speeds

def test_fast_speed_special_cases():
    rho, p = 1.7, 0.9
    a = math.sqrt(G * p / rho)
    # no field: sound speed
    assert O.fast_speed([rho, 0, 0, 0, p, 0, 0], 0.0, G) == pytest.approx(a, rel=1e-15)
    # field purely transverse: sqrt(a^2 + b^2)
    bt = (0.6, -0.8)
    b2 = (bt[0] ** 2 + bt[1] ** 2) / rho
    assert O.fast_speed([rho, 0.3, 0, 0, p, bt[0], bt[1]], 0.0, G) == pytest.approx(math.sqrt(a * a + b2), rel=1e-14)
    # field purely normal: max(a, Alfven speed)
    for bn in (0.3, 2.5):
        ca = abs(bn) / math.sqrt(rho)
        assert O.fast_speed([rho, 0, 0, 0, p, 0, 0], bn, G) == pytest.approx(max(a, ca), rel=1e-14)


# ----------------------------------------------------------------- fluxes

def _rotational_discontinuity(s_zero=True):
    rho, p, bn = 1.3, 0.7, 0.9
    ca = bn / math.sqrt(rho)
    bt, th = 0.8, 1.1
    byl, bzl = bt, 0.0
    byr, bzr = bt * math.cos(th), bt * math.sin(th)
    u = -ca if s_zero else 0.35
    vl, wl = 0.2, -0.1
    # Alfven jump relations: [v_t] = -[B_t]/sqrt(rho) for a wave moving at u + c_A
    vr = vl - (byr - byl) / math.sqrt(rho)
    wr = wl - (bzr - bzl) / math.sqrt(rho)
    WL = np.array([rho, u, vl, wl, p, byl, bzl])
    WR = np.array([rho, u, vr, wr, p, byr, bzr])
    return WL, WR, bn, u + ca


def _cons7(w, bn, g):
    rho, u, v, ww, p, by, bz = w
    return np.array([rho, rho * u, rho * v, rho * ww,
                     p / (g - 1) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * (bn * bn + by * by + bz * bz),
                     by, bz])


def test_physical_flux_rankine_hugoniot_hydro_shock():
    # textbook normal-shock relations (no field), in the shock frame the flux is continuous
    for M in (1.5, 3.0, 8.0):
        rho1, p1 = 1.0, 1.0
        c1 = math.sqrt(G * p1 / rho1)
        u1 = M * c1
        rho2 = rho1 * (G + 1) * M * M / ((G - 1) * M * M + 2)
        p2 = p1 * (2 * G * M * M - (G - 1)) / (G + 1)
        u2 = u1 * rho1 / rho2
        f1 = O.phys_flux([rho1, u1, 0.2, -0.3, p1, 0, 0], 0.0, G)
        f2 = O.phys_flux([rho2, u2, 0.2, -0.3, p2, 0, 0], 0.0, G)
        np.testing.assert_allclose(f1, f2, rtol=1e-13, atol=1e-13)


def test_physical_flux_rankine_hugoniot_alfven_discontinuity():
    # a moving rotational discontinuity satisfies F(UR) - F(UL) = s (UR - UL)
    WL, WR, bn, s = _rotational_discontinuity(s_zero=False)
    dF = O.phys_flux(WR, bn, G) - O.phys_flux(WL, bn, G)
    dU = _cons7(WR, bn, G) - _cons7(WL, bn, G)
    np.testing.assert_allclose(dF, s * dU, rtol=0, atol=1e-14)


@pytest.mark.parametrize("solver", ["hlld", "hll"])
def test_riemann_consistency(solver):
    fn = getattr(O, solver)
    rng = np.random.default_rng(7)
    for _ in range(200):
        w = np.array([rng.uniform(0.2, 2), rng.normal(0, 2), rng.normal(), rng.normal(),
                      rng.uniform(0.1, 2), rng.normal(), rng.normal()])
        bn = rng.normal()
        np.testing.assert_allclose(fn(w, w, bn, G), O.phys_flux(w, bn, G), rtol=1e-13, atol=1e-13)


def test_hlld_resolves_stationary_contact_and_tangential_discontinuity():
    # contact: only rho jumps, u = 0, B_n != 0 -> the exact flux is F(UL) = F(UR)
    WL = np.array([1.0, 0.0, 0.3, -0.2, 0.8, 0.5, 0.4])
    WR = WL.copy(); WR[0] = 0.2
    f = O.hlld(WL, WR, 0.7, G)
    np.testing.assert_allclose(f, O.phys_flux(WL, 0.7, G), rtol=0, atol=1e-14)
    np.testing.assert_allclose(f, O.phys_flux(WR, 0.7, G), rtol=0, atol=1e-14)
    # tangential discontinuity: B_n = 0, u = 0, total pressure balanced
    WL = np.array([1.0, 0.0, 0.5, -0.3, 1.0, 0.6, -0.2])
    WR = np.array([0.4, 0.0, -0.7, 0.9, 0.0, 1.1, 0.35])
    WR[4] = WL[4] + 0.5 * (WL[5] ** 2 + WL[6] ** 2) - 0.5 * (WR[5] ** 2 + WR[6] ** 2)
    assert WR[4] > 0
    f = O.hlld(WL, WR, 0.0, G)
    np.testing.assert_allclose(f, O.phys_flux(WL, 0.0, G), rtol=0, atol=1e-14)
    np.testing.assert_allclose(f, O.phys_flux(WR, 0.0, G), rtol=0, atol=1e-14)


def test_hlld_resolves_stationary_alfven_discontinuity():
    # Miyoshi & Kusano: isolated Alfven discontinuities are captured exactly
    WL, WR, bn, s = _rotational_discontinuity(s_zero=True)
    assert abs(s) < 1e-15
    f = O.hlld(WL, WR, bn, G)
    np.testing.assert_allclose(f, O.phys_flux(WL, bn, G), rtol=0, atol=1e-14)
    # HLL smears it: the pin is specific to the HLLD star states
    assert np.abs(O.hll(WL, WR, bn, G) - O.phys_flux(WL, bn, G)).max() > 1e-2


@pytest.mark.parametrize("solver", ["hlld", "hll"])
def test_riemann_mirror_symmetry(solver):
    # x -> -x with B -> -B: u and B_n flip, L and R swap; every flux component
    # flips sign except the normal momentum flux.
    fn = getattr(O, solver)
    rng = np.random.default_rng(11)
    S = np.array([-1, 1, -1, -1, -1, -1, -1.0])
    for _ in range(300):
        wl = np.array([rng.uniform(0.2, 2), rng.normal(0, 1.5), rng.normal(), rng.normal(),
                       rng.uniform(0.1, 2), rng.normal(), rng.normal()])
        wr = np.array([rng.uniform(0.2, 2), rng.normal(0, 1.5), rng.normal(), rng.normal(),
                       rng.uniform(0.1, 2), rng.normal(), rng.normal()])
        bn = rng.normal() if rng.uniform() < 0.9 else 0.0
        m = lambda w: np.array([w[0], -w[1], w[2], w[3], w[4], w[5], w[6]])
        f = fn(wl, wr, bn, G)
        g = fn(m(wr), m(wl), -bn, G)
        np.testing.assert_allclose(g, S * f, rtol=1e-12, atol=1e-12)


def test_hlld_supersonic_upwinding():
    # all waves moving right: the flux is the left physical flux, and vice versa
    w = np.array([1.0, 9.0, 0.1, 0.2, 0.5, 0.3, 0.1])
    w2 = np.array([0.8, 9.5, -0.1, 0.0, 0.6, 0.2, 0.4])
    np.testing.assert_array_equal(O.hlld(w, w2, 0.4, G), O.phys_flux(w, 0.4, G))
    w[1], w2[1] = -9.0, -9.5
    np.testing.assert_array_equal(O.hlld(w, w2, 0.4, G), O.phys_flux(w2, 0.4, G))


# ----------------------------------------------------------------- whole scheme

@pytest.mark.parametrize("integ", ["rk2", "rk3"])
def test_uniform_state_is_preserved_bitwise(integ):
    # RK2's combination is exact on a stationary state; RK3's weights 3/4,
    # 1/4, 1/3, 2/3 round, so it keeps a uniform state to a few ulps
    for bc in [(0, 0, 0), (1, 1, 1), (1, 0, 1)]:
        b = I.uniform_state((6, 5, 4), bc=bc)
        cfg = cfg_of(b)
        cfg.integrator = integ
        c, f, _ = O.step(cfg, b.cell, b.face, 1e-3, nsteps=3)
        if integ == "rk2":
            np.testing.assert_array_equal(c, b.cell)
            for d in range(3):
                np.testing.assert_array_equal(f[d], b.face[d])
        else:
            np.testing.assert_allclose(c, b.cell, rtol=1e-15, atol=1e-16)
            for d in range(3):
                np.testing.assert_allclose(f[d], b.face[d], rtol=1e-15, atol=1e-16)


def test_cfl_closed_form_uniform():
    b = I.uniform_state((8, 6, 4), rho=1.3, v=(0.3, -0.2, 0.1), p=0.7, B=(0.4, -0.5, 0.6))
    cfg = cfg_of(b)
    rho, p, v, B = 1.3, 0.7, (0.3, -0.2, 0.1), (0.4, -0.5, 0.6)
    a2 = G * p / rho
    b2 = sum(x * x for x in B) / rho
    tot = 0.0
    for d in range(3):
        # textbook fast speed for a field at angle theta to direction d
        cf = math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * B[d] ** 2 / rho)))
        tot += (abs(v[d]) + cf) / b.dx
    assert O.cfl_dt(cfg, b.cell, b.face) == pytest.approx(0.4 / tot, rel=1e-14)
    # a 2D box ignores the z term
    b2d = I.uniform_state((8, 6, 1), rho=1.3, v=v, p=p, B=B)
    tot2 = tot - (abs(v[2]) + math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * B[2] ** 2 / rho)))) / b.dx
    assert O.cfl_dt(cfg_of(b2d), b2d.cell, b2d.face) == pytest.approx(0.4 / tot2, rel=1e-14)


@pytest.mark.parametrize("integ", ["rk2", "rk3"])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (1, 0, 0)])
def test_divb_stays_at_roundoff(bc, integ):
    b = I.random_state((10, 9, 8), seed=3, bc=bc)
    cfg = cfg_of(b)
    cfg.integrator = integ
    assert O.divb_max(cfg, b.face) < 1e-12
    c, f, _ = O.step(cfg, b.cell, b.face, -1, nsteps=10)
    scale = max(np.abs(x).max() for x in f) / b.dx
    assert O.divb_max(cfg, f) < 1e-13 * scale


@pytest.mark.parametrize("integ", ["rk2", "rk3"])
def test_periodic_conservation(integ):
    b = I.random_state((10, 8, 6), seed=5)
    cfg = cfg_of(b)
    cfg.integrator = integ
    c, f, _ = O.step(cfg, b.cell, b.face, -1, nsteps=8)
    for v in range(5):
        s0, s1 = b.cell[v].sum(), c[v].sum()
        ref = np.abs(b.cell[v]).sum()
        assert abs(s1 - s0) <= 1e-13 * ref, (v, s0, s1)
    for d in range(3):
        s0, s1 = b.face[d].sum(), f[d].sum()
        assert abs(s1 - s0) <= 1e-13 * np.abs(b.face[d]).sum() + 1e-13


def _cyc(a):
    # old axes (z, y, x) -> new axes (z', y', x') = (y, x, z): new x' = old z, y' = old x, z' = old y
    return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))


def test_cyclic_axis_permutation():
    b = I.random_state((7, 6, 5), seed=9)
    cfg = cfg_of(b)
    c1, f1, _ = O.step(cfg, b.cell, b.face, 2e-3, nsteps=3)
    # relabel: x' = z, y' = x, z' = y  (cyclic).  Momentum (mx, my, mz) -> (mx', my', mz') = (mz, mx, my)
    cell = np.stack([_cyc(b.cell[0]), _cyc(b.cell[3]), _cyc(b.cell[1]), _cyc(b.cell[2]), _cyc(b.cell[4])])
    face = [_cyc(b.face[2]), _cyc(b.face[0]), _cyc(b.face[1])]
    cfg2 = O.Config(b.nz, b.nx, b.ny, b.dz, b.dx, b.dy, b.gamma, b.cfl, (0, 0, 0))
    c2, f2, _ = O.step(cfg2, cell, face, 2e-3, nsteps=3)
    exp_c = np.stack([_cyc(c1[0]), _cyc(c1[3]), _cyc(c1[1]), _cyc(c1[2]), _cyc(c1[4])])
    np.testing.assert_allclose(c2, exp_c, rtol=0, atol=1e-13)
    for d, e in zip(range(3), (2, 0, 1)):
        np.testing.assert_allclose(f2[d], _cyc(f1[e]), rtol=0, atol=1e-13)


def test_one_dimensional_reduction():
    """Along a 1D grid the CT edge EMF reduces to the face EMF, so the whole
    operator equals the plain 1D finite-volume update built from the oracle's
    single-face pieces (MC slopes + HLLD)."""
    n = 24
    b = I.random_state((n, 1, 1), seed=21)
    cfg = cfg_of(b)
    du, db = O.rhs(cfg, b.cell, b.face)
    rho = b.cell[0, 0, 0]
    v = b.cell[1:4, 0, 0] / rho
    Bx = b.face[0][0, 0]                     # face i at i-1/2 (uniform in 1D)
    By = b.face[1][0, 0]                     # ny = 1: cell value
    Bz = b.face[2][0, 0]
    bcx = 0.5 * (Bx + np.roll(Bx, -1))
    p = (G - 1) * (b.cell[4, 0, 0] - 0.5 * rho * (v ** 2).sum(0) - 0.5 * (bcx ** 2 + By ** 2 + Bz ** 2))
    W = np.stack([rho, v[0], v[1], v[2], p, By, Bz])          # rotated order for x-sweep
    F = np.zeros((7, n))
    for i in range(n):                                        # face i at i-1/2
        im2, im1, ip1 = (i - 2) % n, (i - 1) % n, (i + 1) % n
        sl = np.array([O.mc_slope(W[q, im2], W[q, im1], W[q, i]) for q in range(7)])
        sr = np.array([O.mc_slope(W[q, im1], W[q, i], W[q, ip1]) for q in range(7)])
        F[:, i] = O.hlld(W[:, im1] + 0.5 * sl, W[:, i] - 0.5 * sr, Bx[i], G)
    dF = (np.roll(F, -1, axis=1) - F) / b.dx
    np.testing.assert_allclose(du[:, 0, 0, :], -dF[:5], rtol=0, atol=1e-12)
    np.testing.assert_allclose(db[1][0, 0], -dF[5], rtol=0, atol=1e-12)
    np.testing.assert_allclose(db[2][0, 0], -dF[6], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(db[0], 0.0)


def test_orszag_tang_point_symmetry():
    """q(1-x, 1-y) = +q(x, y) for rho, p, E and -q for v, B: a symmetry of the
    equations that the discrete scheme must keep to rounding."""
    b = I.orszag_tang_2d(48)
    cfg = cfg_of(b)
    c, f, _ = O.step(cfg, b.cell, b.face, -1, nsteps=60)
    flip = lambda a: a[:, ::-1, ::-1]
    for v, sgn in zip(range(5), (1, -1, -1, -1, 1)):
        np.testing.assert_allclose(c[v], sgn * flip(c[v]), rtol=0, atol=1e-12 * max(np.abs(c[v]).max(), 1.0))
    # a face at i-1/2 maps to the face at (n-i)-1/2
    fx = np.roll(f[0][:, ::-1, ::-1], 1, axis=2)
    fy = np.roll(f[1][:, ::-1, ::-1], 1, axis=1)
    np.testing.assert_allclose(f[0], -fx, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f[1], -fy, rtol=0, atol=1e-12)


def test_checkpoint_resume_bitwise():
    b = I.random_state((8, 7, 6), seed=2)
    cfg = cfg_of(b)
    c1, f1, dts = O.step(cfg, b.cell, b.face, -1, nsteps=6)
    ca, fa, d1 = O.step(cfg, b.cell, b.face, -1, nsteps=3)
    cb, fb, d2 = O.step(cfg, ca, fa, -1, nsteps=3)
    np.testing.assert_array_equal(c1, cb)
    for d in range(3):
        np.testing.assert_array_equal(f1[d], fb[d])


def test_step_is_well_conditioned_on_a_low_beta_blast():
    """A 1e-15 relative perturbation of the state moves one RK2 step of a
    low-beta blast by rounding only.  Without the deadband on the mass-flux
    sign that orients the upwind EMF average, rounding-level mass fluxes flip
    the upwind side and the face field jumps by O(v B)."""
    box = I.blast_batch(1, seed=3, nmin=24, nmax=32)[0]
    cfg = cfg_of(box)
    rng = np.random.default_rng(0)
    c0, f0, _ = O.step(cfg, box.cell, box.face, 5e-4, nsteps=2)
    cell = box.cell * (1 + 1e-15 * rng.standard_normal(box.cell.shape))
    c1, f1, _ = O.step(cfg, cell, box.face, 5e-4, nsteps=2)
    from helpers import state_errors
    errs = state_errors(c1, f1, c0, f0)
    assert max(errs.values()) < 1e-11, errs
