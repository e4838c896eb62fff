"""Operation counts of the oracle's step -- TEST INFRASTRUCTURE.

``opcount.cpp`` compiles ``mhd_oracle.c`` unchanged with every double replaced
by a counting value type, so the counts are those of the method exactly as the
oracle computes it (Sec. 2.2: primitive recovery, PLM-MC, HLLD, CT EMFs, flux
divergence, the RK stages, the CFL maximum).  ``counting()`` swaps that build
in under the oracle's ordinary Python wrappers.

Per-cell figures: the oracle also works on its ghost layers, whose cost grows
like the box's surface.  A seeded periodic pattern is tiled 1..4 times per
axis (every tile is an exact copy, so each interior cell repeats the same
branches) and each count is fitted by a cubic in the edge length n; the n^3
coefficient is the count per interior cell.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

from . import _BUILD, _HERE, PERIODIC, Config, _Cfg, _state_ptrs, bind, copy_state

_SRC = os.path.join(_HERE, "opcount.cpp")
_ORC = os.path.join(_HERE, "mhd_oracle.c")
_LIB_PATH = os.path.join(_BUILD, "libopcount.so")
CATEGORIES = ("add", "mul", "div", "sqrt", "cmp", "misc")   # misc: abs, min, max, copysign
FLOP_CATEGORIES = ("add", "mul", "div", "sqrt")

_lib = None


def build(force: bool = False) -> str:
    """Compile the counting build (g++, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    t = max(os.path.getmtime(_SRC), os.path.getmtime(_ORC))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < t:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        # -fpermissive: the oracle is C and converts malloc's void* implicitly
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fpermissive", "-w",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = bind(C.CDLL(build()))
        L.orc_opcount_reset.restype = None
        L.orc_opcount_reset.argtypes = []
        L.orc_opcount_get.restype = None
        L.orc_opcount_get.argtypes = [C.POINTER(C.c_ulonglong)]
        P = C.POINTER(C.c_double)
        L.orc_opcount_prims.restype = None
        L.orc_opcount_prims.argtypes = [C.POINTER(_Cfg), P * 5, P * 3]
        _lib = L
    return _lib


@contextlib.contextmanager
def counting():
    """Run the oracle's Python wrappers on the counting build; yields a
    function that returns the counts accumulated since entry."""
    import oracle as O
    L = lib()
    old = O._lib
    O._lib = L
    L.orc_opcount_reset()

    def read():
        out = (C.c_ulonglong * 6)()
        L.orc_opcount_get(out)
        return dict(zip(CATEGORIES, (int(v) for v in out)))

    try:
        yield read
    finally:
        O._lib = old


def flops(counts: dict) -> float:
    return float(sum(counts[k] for k in FLOP_CATEGORIES))


def prims_counts(cfg: Config, cell, face) -> dict:
    """Counts of one primitive-recovery pass (the operator's first stage)."""
    cell, face = copy_state(cell, face)
    c = cfg.c()
    cp, fp = _state_ptrs(cfg, cell, face)
    with counting() as read:
        lib().orc_opcount_prims(C.byref(c), cp, fp)
        return read()


def _tile(cell, face, m):
    return (np.ascontiguousarray(np.tile(cell, (1, m, m, m))),
            [np.ascontiguousarray(np.tile(f, (m, m, m))) for f in face])


def _stage_states(cfg: Config, cell, face, dt: float):
    """The states the operator is evaluated on within one step (plain oracle):
    RK2 U^n, U* = U^n + dt L(U^n); SSP-RK3 U^n, U1, U2."""
    import oracle as O
    du, db = O.rhs(cfg, cell, face)
    s1 = (cell + dt * du, [f + dt * d for f, d in zip(face, db)])
    if cfg.integrator == "rk2":
        return [(cell, face), s1]
    du, db = O.rhs(cfg, *s1)
    s2 = (0.75 * cell + 0.25 * (s1[0] + dt * du),
          [0.75 * f + 0.25 * (g + dt * d) for f, g, d in zip(face, s1[1], db)])
    return [(cell, face), s1, s2]


def per_cell(cfg0: Config, cell0, face0, dt: float, tiles=(1, 2, 3, 4)) -> dict:
    """Per-interior-cell counts of the parts of one step, for the periodic
    pattern (cfg0, cell0, face0) with a fixed dt: 'step' (one step of
    cfg0.integrator), 'operator' (its operator evaluations, each on its own
    stage state), 'prims' (their primitive recoveries), 'cfl' (one CFL
    maximum).  Each value is a dict over CATEGORIES (floats: the n^3
    coefficients of cubic fits)."""
    import oracle as O
    assert tuple(cfg0.bc) == (PERIODIC,) * 3 and cfg0.nx == cfg0.ny == cfg0.nz
    n0 = cfg0.nx
    ns, raw = [], {"step": [], "operator": [], "prims": [], "cfl": []}
    for m in tiles:
        n = n0 * m
        cfg = Config(n, n, n, cfg0.dx, cfg0.dy, cfg0.dz, gamma=cfg0.gamma, cfl=cfg0.cfl, bc=cfg0.bc,
                     rho_floor=cfg0.rho_floor, p_floor=cfg0.p_floor, emf_mean=cfg0.emf_mean,
                     riemann=cfg0.riemann, integrator=cfg0.integrator, recon=cfg0.recon)
        cell, face = _tile(cell0, face0, m)
        with counting() as read:
            O.step_dts(cfg, cell, face, [dt])
            raw["step"].append(read())
        stages = _stage_states(cfg, cell, face, dt)
        with counting() as read:
            for c, f in stages:
                O.rhs(cfg, c, f)
            raw["operator"].append(read())
        tot = dict.fromkeys(CATEGORIES, 0)
        for c, f in stages:
            for k, v in prims_counts(cfg, c, f).items():
                tot[k] += v
        raw["prims"].append(tot)
        with counting() as read:
            O.cfl_dt(cfg, cell, face)
            raw["cfl"].append(read())
        ns.append(n)
    ns = np.array(ns, dtype=np.float64)
    V = np.vander(ns, 4)        # n^3, n^2, n, 1
    out = {}
    for part, rows in raw.items():
        out[part] = {}
        for k in CATEGORIES:
            y = np.array([r[k] for r in rows], dtype=np.float64)
            coef = np.linalg.solve(V, y) if len(ns) == 4 else np.linalg.lstsq(V, y, rcond=None)[0]
            out[part][k] = float(coef[0])
    return out


def split(pc: dict) -> dict:
    """Flops per cell-update of one step with its fused CFL maximum, and their
    split in the mixed form: FP64 for the primitive recoveries and the RK
    accumulation of the conserved state and faces; FP32 for reconstruction,
    Riemann solver, EMFs, divergence and the CFL maximum."""
    step, op, pr, cfl = (flops(pc[k]) for k in ("step", "operator", "prims", "cfl"))
    rk = step - op
    return {"total": step + cfl, "fp64_in_mixed": pr + rk, "fp32_in_mixed": (op - pr) + cfl,
            "operators": op, "prims": pr, "rk_accumulate": rk, "cfl": cfl}
