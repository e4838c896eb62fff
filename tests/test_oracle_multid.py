"""Multi-dimensional and single-face pins of the oracle that 1D tests cannot see.

* Oblique linear waves (Gardiner & Stone 2008): fast, Alfven and slow modes
  along (1, 2, 0) on a 2n x n x 1 box and along (1, 1, 2) on a 2m x 2m x m
  box converge at second order, with the upwind and with the mean EMF.  A
  wave that is not aligned with the grid makes every edge EMF combine faces of
  two sweeps with nonzero transverse fluxes, which a grid-aligned 1D wave
  never does.
* Field-loop advection (Gardiner & Stone 2005, Sec. 5.1): the upwind side of
  the "contact" EMF average.  Carried obliquely, the loop's magnetic energy
  decays monotonically and slowly; taking the downwind side instead makes the
  scheme unstable (the energy grows, then overflows).
* HLL's dissipation sign: a stationary contact with rho_L > rho_R gives the
  mass flux c (rho_L - rho_R)/2 > 0 (c = the larger sound speed), the closed
  form of HLL with S_R = -S_L = c; HLL linear waves converge at second order.
* HLLD's degenerate star state (|den| ~ 0, reached when B_t -> 0 with the
  Alfven speed above the sound speed): the flux of the degenerate branch is
  the limit of the non-degenerate fluxes of nearby states B_t = delta b.

The runs are independent, so each test maps them over a pool of worker
processes (spawned, so no worker inherits a GPU context or a loaded library).
"""
from __future__ import annotations

import concurrent.futures as cf
import contextlib
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from multid_problems import G, field_loop_box, magnetic_energy, oblique_wave_box

# ------------------------------------------------------------------ workers


def _cfg(b, **kw):
    return O.Config(b.nx, b.ny, b.nz, b.dx, b.dy, b.dz, b.gamma, 0.4, tuple(b.bc), **kw)


def _ctx(subs):
    if not subs:
        return contextlib.nullcontext()
    from mutants import mutant
    return mutant(subs)


def oblique_error(dims, wave, emf_mean=0, riemann=O.HLLD, subs=None):
    """L1 error (sum over variables of the mean |error|) after half a wave
    period against the exact state, which is the initial profile with its
    sign flipped (the phase advanced by pi)."""
    with _ctx(subs):
        b, speed, kn = oblique_wave_box(dims, wave)
        ref, _, _ = oblique_wave_box(dims, wave, sign=-1.0)
        cfg = _cfg(b, emf_mean=emf_mean, riemann=riemann)
        half = math.pi / (kn * speed)
        dt = O.cfl_dt(cfg, b.cell, b.face)
        ns = int(math.ceil(half / dt))
        c, f = O.step_dts(cfg, b.cell, b.face, [half / ns] * ns)
    e = np.abs(c - ref.cell).mean(axis=(1, 2, 3)).sum()
    return float(e + sum(np.abs(f[d] - ref.face[d]).mean() for d in range(3)))


def field_loop_energy(n, emf_mean=0, t_end=0.5, samples=8, direction=1.0, subs=None):
    """Magnetic energy of the advected field loop at `samples` equally spaced
    times up to t_end, relative to the initial energy (stops at the first
    non-finite or growing value)."""
    with _ctx(subs):
        b = field_loop_box(n, direction=direction)
        cfg = _cfg(b, emf_mean=emf_mean)
        dims = (b.nx, b.ny, b.nz)
        e0 = magnetic_energy(b.face, dims, b.dx)
        c, f, t, out = b.cell, b.face, 0.0, [1.0]
        for s in range(1, samples + 1):
            te = t_end * s / samples
            while t < te - 1e-12:
                dt = O.cfl_dt(cfg, c, f)
                if not np.isfinite(dt) or dt <= 0:
                    return out + [float("nan")]
                dt = min(dt, te - t)
                c, f, _ = O.step(cfg, c, f, dt)
                t += dt
            e = magnetic_energy(f, dims, b.dx) / e0
            out.append(float(e))
            if not np.isfinite(e) or e > out[-2]:
                break
    return out


def _call(job):
    fn, args, kw = job
    return fn(*args, **kw)


def pool_map(jobs):
    """Run (fn, args, kwargs) jobs in spawned worker processes."""
    workers = max(1, min(len(jobs), os.cpu_count() or 2))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                initializer=_init_worker) as ex:
        return list(ex.map(_call, jobs))


def _init_worker():
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    for p in (here, os.path.dirname(here)):
        if p not in sys.path:
            sys.path.insert(0, p)


# ------------------------------------------------------------------ checks
# Each check returns (ok, detail) so that the planted-mistake test below can
# run the same check on a mutated oracle and require it to fail.

SIZES_2D = [(32, 16, 1), (64, 32, 1)]
SIZES_3D = [(16, 16, 8), (32, 32, 16)]
WAVES = ("fast", "alfven", "slow")


def check_oblique(emfs=(0, 1), waves=WAVES, subs=None, riemann=O.HLLD):
    jobs, keys = [], []
    for emf in emfs:
        for wave in waves:
            for sizes in (SIZES_2D, SIZES_3D):
                for dims in sizes:
                    jobs.append((oblique_error, (dims, wave), {"emf_mean": emf, "subs": subs, "riemann": riemann}))
                    keys.append((emf, wave, dims[2] > 1, dims))
    errs = dict(zip(keys, pool_map(jobs)))
    bad = {}
    for emf in emfs:
        for wave in waves:
            for three_d, sizes in ((False, SIZES_2D), (True, SIZES_3D)):
                e = [errs[(emf, wave, three_d, d)] for d in sizes]
                order = math.log2(e[0] / e[1]) if e[1] > 0 and np.isfinite(e).all() else float("nan")
                # measured 1.73-2.21 at these sizes (MC clips the extrema,
                # so the coarse pair sits below 2); the finer error stays
                # below 0.2 amp (measured 0.01-0.06 amp)
                if not (order >= 1.6 and e[1] <= 0.2e-6):
                    bad[(emf, wave, "3d" if three_d else "2d")] = (e, order)
    return not bad, bad


def check_field_loop(emfs=(0, 1), n=32, subs=None):
    """The loop carried along +(2, 1) and along -(2, 1): every mass flux is
    positive in one run and negative in the other, so both sides of the
    upwind choice are taken."""
    cases = [(emf, s) for emf in emfs for s in (1.0, -1.0)]
    res = pool_map([(field_loop_energy, (n,), {"emf_mean": emf, "direction": s, "subs": subs})
                    for emf, s in cases])
    bad = {}
    for case, e in zip(cases, res):
        e = np.array(e)
        # measured at t = 0.5: 0.82 (upwind), 0.87 (mean)
        ok = (len(e) == 9 and np.isfinite(e).all() and np.all(np.diff(e) < 0) and 0.6 < e[-1] < 0.97)
        if not ok:
            bad[case] = e.tolist()
    return not bad, bad


def _contact_case():
    rl, rr, p = 1.0, 0.25, 0.6
    vt = (0.3, -0.2)
    WL = np.array([rl, 0.0, vt[0], vt[1], p, 0.0, 0.0])
    WR = np.array([rr, 0.0, vt[0], vt[1], p, 0.0, 0.0])
    c = max(math.sqrt(G * p / rl), math.sqrt(G * p / rr))
    return WL, WR, c


def _cons7(w, bn):
    rho, u, v, ww, p, by, bz = w
    return np.array([rho, rho * u, rho * v, rho * ww,
                     p / (G - 1) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * (bn * bn + by * by + bz * bz),
                     by, bz])


def check_hll_contact(subs=None):
    """HLL across a stationary contact (B = 0, u = 0, equal p): S_R = -S_L = c,
    so F = (F_L + F_R)/2 - c (U_R - U_L)/2 with F_L = F_R = (0, p, 0, ...)."""
    with _ctx(subs):
        WL, WR, c = _contact_case()
        f = O.hll(WL, WR, 0.0, G)
    p = WL[4]
    fphys = np.array([0.0, p, 0, 0, 0, 0, 0])
    expect = fphys - 0.5 * c * (_cons7(WR, 0.0) - _cons7(WL, 0.0))
    ok = f[0] > 0 and np.allclose(f, expect, rtol=1e-14, atol=1e-14)
    return ok, (f.tolist(), expect.tolist())


def check_hll_linear_wave(subs=None):
    """1D HLL linear waves (grid-aligned, the 1D Gardiner-Stone setup) at
    second order; HLL smears the Alfven and slow waves more than HLLD but
    keeps the order."""
    jobs, keys = [], []
    for wave in ("fast", "alfven"):
        for n in (64, 128):
            jobs.append((oblique_error, ((n, 1, 1), wave), {"riemann": O.HLL, "subs": subs}))
            keys.append((wave, n))
    errs = dict(zip(keys, pool_map(jobs)))
    bad = {}
    for wave in ("fast", "alfven"):
        e = [errs[(wave, n)] for n in (64, 128)]
        order = math.log2(e[0] / e[1]) if np.isfinite(e).all() and e[1] > 0 else float("nan")
        if not order >= 1.8:
            bad[wave] = (e, order)
    return not bad, bad


def _degenerate_pair(delta):
    """Equal rho, p and u on both sides, B_n = 1 above the sound speed
    (c_A = 1, a = 0.41), tangential velocities jumping, B_t = delta (bL, bR)."""
    bL, bR = np.array([1.0, 0.5]), np.array([-0.5, 1.2])
    WL = np.array([1.0, 0.0, 0.3, -0.2, 0.1, delta * bL[0], delta * bL[1]])
    WR = np.array([1.0, 0.0, -0.1, 0.4, 0.1, delta * bR[0], delta * bR[1]])
    return WL, WR, 1.0


def check_hlld_degenerate(subs=None):
    with _ctx(subs):
        out = {}
        for d in (1e-3, 1e-4, 1e-5, 1e-7, 1e-9, 0.0):
            WL, WR, bn = _degenerate_pair(d)
            out[d] = O.hlld_region(WL, WR, bn, G)
    # the branch is taken where it should be (den/B_n^2 ~ delta^2 a^2/(c_A^2 - a^2))
    taken = {d: out[d][2] for d in out}
    ok = all(taken[d] == 0 for d in (1e-3, 1e-4, 1e-5)) and all(taken[d] == 2 for d in (1e-7, 1e-9, 0.0))
    f0 = out[0.0][0]
    # the non-degenerate fluxes approach the degenerate one linearly in delta
    dev = {d: float(np.abs(out[d][0] - f0).max()) for d in (1e-3, 1e-4, 1e-5)}
    ok = ok and all(dev[d] <= 5.0 * d for d in dev) and dev[1e-5] < dev[1e-4] < dev[1e-3]
    # below the threshold the flux stays on the same curve
    ok = ok and float(np.abs(out[1e-9][0] - f0).max()) <= 1e-8 and float(np.abs(out[1e-7][0] - f0).max()) <= 1e-6
    return ok, {"taken": taken, "dev": dev, "f0": f0.tolist(), "regions": {d: out[d][1] for d in out}}


# ------------------------------------------------------------------ tests


def test_oblique_linear_waves_second_order():
    ok, bad = check_oblique()
    assert ok, bad


def test_field_loop_energy_decays_monotonically():
    ok, bad = check_field_loop()
    assert ok, bad


def test_hll_dissipation_sign_at_a_stationary_contact():
    ok, detail = check_hll_contact()
    assert ok, detail


def test_hll_linear_waves_second_order():
    ok, bad = check_hll_linear_wave()
    assert ok, bad


def test_hlld_degenerate_branch_is_the_limit_of_nearby_states():
    ok, detail = check_hlld_degenerate()
    assert ok, detail
