"""FP64 CPU oracle of the ideal-MHD Godunov step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never does, and this package never imports the product: the two share
no code.  The arithmetic lives in ``mhd_oracle.c`` (plain loops, FP64, built
without FMA contraction); this module only builds it and marshals numpy
arrays through ctypes.  ``mlp.py`` holds the FP64 reference of the face-switch
network.

State convention (shared with the seeded input generators, not with the GPU
code): ``cell`` is a float64 array of shape (5, nz, ny, nx) holding
(rho, mx, my, mz, E); ``face`` is a list of three float64 arrays holding Bx on
x-faces (shape (nz, ny, nx+o)), By on y-faces (nz, ny+o, nx) and Bz on z-faces
(nz+o, ny, nx), where o = 1 on an outflow axis and 0 on a periodic one.  Face
index i along the normal is the face at i-1/2.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

PERIODIC, OUTFLOW = 0, 1
HLLD, HLL, LEARNED, MASK = 0, 1, 2, 3
# rounding thresholds of the branch decisions (HLLD degeneracy, mass-flux
# deadband, characteristic degeneracies): those of the FP64 form, or those of
# the FP32-bulk forms (mixed and FP32), which take the decisions in FP32
THRESH_FP64, THRESH_FP32 = 0, 1


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, no FMA contraction) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("bc", C.c_int * 3),
                ("rho_floor", C.c_double), ("p_floor", C.c_double),
                ("emf_mean", C.c_int), ("riemann", C.c_int),
                ("mlp", C.POINTER(C.c_double)), ("mlp_zt", C.c_double),
                ("choice", C.POINTER(C.c_ubyte)), ("recon", C.c_int), ("thresholds", C.c_int),
                ("thresh_scale", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("rho_floor_hits", C.c_longlong), ("p_floor_hits", C.c_longlong),
                ("faces_hll", C.c_longlong), ("faces_hlld", C.c_longlong),
                ("hlld_region", C.c_longlong * 6), ("hlld_degenerate", C.c_longlong)]


# HLLD regions, in the order of the region census (Stats.hlld_region)
HLLD_REGIONS = ("L", "L*", "L**", "R**", "R*", "R")


@dataclass
class Config:
    """Grid and method parameters of one box."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    gamma: float = 5.0 / 3.0
    cfl: float = 0.4
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    rho_floor: float = 1e-10
    p_floor: float = 1e-10
    emf_mean: int = 0
    riemann: int = HLLD
    # LEARNED: the 1633 network parameters (oracle/mlp.py order) and the logit
    # threshold (HLLD when logit >= mlp_zt); MASK: per-face choices (uint8,
    # 1 = HLLD) indexed d * nx*ny*nz + cell
    mlp: np.ndarray | None = None
    mlp_zt: float = 0.0
    choice: np.ndarray | None = None
    # time integrator of step / step_dts: "rk2" (Heun) or "rk3" (Shu-Osher SSP)
    integrator: str = "rk2"
    # reconstruction: 0 = MC on the primitives, 1 = MC on the characteristic variables
    recon: int = 0
    # THRESH_FP64 or THRESH_FP32: the branch thresholds of the form under test
    thresholds: int = THRESH_FP64
    # every branch threshold times this factor (sensitivity of the decisions)
    thresh_scale: float = 1.0

    def c(self) -> _Cfg:
        mp = None
        if self.mlp is not None:
            self.mlp = np.ascontiguousarray(self.mlp, dtype=np.float64)
            assert self.mlp.size == 1633
            mp = self.mlp.ctypes.data_as(C.POINTER(C.c_double))
        cp = None
        if self.choice is not None:
            self.choice = np.ascontiguousarray(self.choice, dtype=np.uint8)
            assert self.choice.size == 3 * self.nx * self.ny * self.nz
            cp = self.choice.ctypes.data_as(C.POINTER(C.c_ubyte))
        if self.riemann == LEARNED:
            assert mp is not None, "LEARNED needs the network parameters"
        if self.riemann == MASK:
            assert cp is not None, "MASK needs the per-face choices"
        return _Cfg(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.gamma, self.cfl,
                    (C.c_int * 3)(*self.bc), self.rho_floor, self.p_floor, self.emf_mean,
                    self.riemann, mp, self.mlp_zt, cp, self.recon, self.thresholds, self.thresh_scale)

    def face_shapes(self):
        o = [1 if b == OUTFLOW else 0 for b in self.bc]
        return [(self.nz, self.ny, self.nx + o[0]),
                (self.nz, self.ny + o[1], self.nx),
                (self.nz + o[2], self.ny, self.nx)]


_lib = None
_P = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = bind(C.CDLL(build()))
    return _lib


def bind(L):
    """Declare the oracle's C signatures on a loaded library (the oracle, or
    its operation-counting build, which exports the same functions)."""
    L.orc_mc_slope.restype = C.c_double
    L.orc_mc_slope.argtypes = [C.c_double] * 3
    L.orc_fast_speed.restype = C.c_double
    L.orc_fast_speed.argtypes = [_P, C.c_double, C.c_double]
    for name in ("orc_phys_flux", "orc_hll", "orc_hlld"):
        fn = getattr(L, name)
        fn.restype = None
    L.orc_phys_flux.argtypes = [_P, C.c_double, C.c_double, _P]
    L.orc_hll.argtypes = [_P, _P, C.c_double, C.c_double, _P]
    L.orc_hlld.argtypes = [_P, _P, C.c_double, C.c_double, _P]
    L.orc_hlld_region.restype = None
    L.orc_hlld_region.argtypes = [_P, _P, C.c_double, C.c_double, _P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    PP = _P * 5
    PF = _P * 3
    L.orc_step.restype = None
    L.orc_step.argtypes = [C.POINTER(_Cfg), PP, PF, C.c_double, C.POINTER(_Stats)]
    L.orc_step_rk3.restype = None
    L.orc_step_rk3.argtypes = [C.POINTER(_Cfg), PP, PF, C.c_double, C.POINTER(_Stats)]
    L.orc_rhs.restype = None
    L.orc_rhs.argtypes = [C.POINTER(_Cfg), PP, PF, PP, PF, C.POINTER(_Stats)]
    L.orc_cfl_dt.restype = C.c_double
    L.orc_cfl_dt.argtypes = [C.POINTER(_Cfg), PP, PF]
    L.orc_divb_max.restype = C.c_double
    L.orc_divb_max.argtypes = [C.POINTER(_Cfg), PF]
    L.orc_bf16.restype = C.c_double
    L.orc_bf16.argtypes = [C.c_double]
    L.orc_features.restype = None
    L.orc_features.argtypes = [_P, _P, C.c_double, C.c_double, _P]
    L.orc_mlp_logit.restype = C.c_double
    L.orc_mlp_logit.argtypes = [_P, _P]
    L.orc_char_eig.restype = None
    L.orc_char_eig.argtypes = [_P, C.c_double, C.c_double, _P, _P, _P]
    L.orc_char_slope.restype = None
    L.orc_char_slope.argtypes = [_P, _P, _P, C.c_double, C.c_double, _P]
    L.orc_switch_logits.restype = None
    L.orc_switch_logits.argtypes = [C.POINTER(_Cfg), PP, PF, _P]
    return L


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _vec(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


# ---------------------------------------------------------------- single face

def mc_slope(qm: float, q0: float, qp: float) -> float:
    return lib().orc_mc_slope(qm, q0, qp)


def fast_speed(w, bn: float, gamma: float) -> float:
    w = _vec(w, 7)
    return lib().orc_fast_speed(_ptr(w), bn, gamma)


def phys_flux(w, bn: float, gamma: float) -> np.ndarray:
    w = _vec(w, 7)
    f = np.zeros(7)
    lib().orc_phys_flux(_ptr(w), bn, gamma, _ptr(f))
    return f


def hlld(wl, wr, bn: float, gamma: float) -> np.ndarray:
    wl, wr = _vec(wl, 7), _vec(wr, 7)
    f = np.zeros(7)
    lib().orc_hlld(_ptr(wl), _ptr(wr), bn, gamma, _ptr(f))
    return f


def hlld_region(wl, wr, bn: float, gamma: float):
    """(HLLD flux, name of the region it came from, number of star states
    that took the degenerate branch)."""
    wl, wr = _vec(wl, 7), _vec(wr, 7)
    f = np.zeros(7)
    reg, deg = C.c_int(-1), C.c_int(0)
    lib().orc_hlld_region(_ptr(wl), _ptr(wr), bn, gamma, _ptr(f), C.byref(reg), C.byref(deg))
    return f, HLLD_REGIONS[reg.value], deg.value


def hll(wl, wr, bn: float, gamma: float) -> np.ndarray:
    wl, wr = _vec(wl, 7), _vec(wr, 7)
    f = np.zeros(7)
    lib().orc_hll(_ptr(wl), _ptr(wr), bn, gamma, _ptr(f))
    return f


# ---------------------------------------------------------------- whole grid

@dataclass
class Stats:
    rho_floor_hits: int = 0
    p_floor_hits: int = 0
    faces_hll: int = 0
    faces_hlld: int = 0
    # HLLD faces by region (keys HLLD_REGIONS) and degenerate star states
    hlld_region: dict = field(default_factory=lambda: dict.fromkeys(HLLD_REGIONS, 0))
    hlld_degenerate: int = 0

    def add(self, st):
        self.rho_floor_hits += st.rho_floor_hits
        self.p_floor_hits += st.p_floor_hits
        self.faces_hll += st.faces_hll
        self.faces_hlld += st.faces_hlld
        for r, name in enumerate(HLLD_REGIONS):
            self.hlld_region[name] += st.hlld_region[r]
        self.hlld_degenerate += st.hlld_degenerate


def _state_ptrs(cfg: Config, cell: np.ndarray, face):
    assert cell.shape == (5, cfg.nz, cfg.ny, cfg.nx), cell.shape
    shapes = cfg.face_shapes()
    for d in range(3):
        assert face[d].shape == shapes[d], (d, face[d].shape, shapes[d])
    cp = (_P * 5)(*[_ptr(cell[v]) for v in range(5)])
    fp = (_P * 3)(*[_ptr(face[d]) for d in range(3)])
    return cp, fp


def copy_state(cell, face):
    return np.array(cell, dtype=np.float64, order="C"), [np.array(f, dtype=np.float64, order="C") for f in face]


def _stepper(cfg: Config):
    if cfg.integrator == "rk3":
        return lib().orc_step_rk3
    assert cfg.integrator == "rk2", cfg.integrator
    return lib().orc_step


def step(cfg: Config, cell, face, dt: float, nsteps: int = 1, stats: Stats | None = None):
    """Advance ``nsteps`` RK2 steps with a fixed ``dt`` (dt <= 0: CFL dt each
    step).  Returns new (cell, face, dts); the inputs are left untouched."""
    cell, face = copy_state(cell, face)
    c = cfg.c()
    st = _Stats(0, 0, 0, 0)
    cp, fp = _state_ptrs(cfg, cell, face)
    dts = []
    for _ in range(nsteps):
        h = dt if dt > 0 else lib().orc_cfl_dt(C.byref(c), cp, fp)
        _stepper(cfg)(C.byref(c), cp, fp, h, C.byref(st))
        dts.append(h)
    if stats is not None:
        stats.add(st)
    return cell, face, dts


def step_dts(cfg: Config, cell, face, dts):
    """Advance one RK2 step per entry of ``dts``."""
    cell, face = copy_state(cell, face)
    c = cfg.c()
    cp, fp = _state_ptrs(cfg, cell, face)
    for h in dts:
        _stepper(cfg)(C.byref(c), cp, fp, float(h), None)
    return cell, face


def rhs(cfg: Config, cell, face, stats: Stats | None = None):
    """Spatial operator L(U): returns (dU of shape (5, nz, ny, nx), [dBx, dBy, dBz])."""
    cell, face = copy_state(cell, face)
    du = np.zeros_like(cell)
    db = [np.zeros_like(f) for f in face]
    c = cfg.c()
    st = _Stats(0, 0, 0, 0)
    cp, fp = _state_ptrs(cfg, cell, face)
    dp, dbp = _state_ptrs(cfg, du, db)
    lib().orc_rhs(C.byref(c), cp, fp, dp, dbp, C.byref(st))
    if stats is not None:
        stats.add(st)
    return du, db


def bf16(x: float) -> float:
    """Nearest bfloat16 of x (rounded to binary32 first), ties to even."""
    return lib().orc_bf16(float(x))


def switch_features(wl, wr, bn: float, gamma: float) -> np.ndarray:
    """The 16 features of the learned switch (C restatement)."""
    wl, wr = _vec(wl, 7), _vec(wr, 7)
    f = np.zeros(16)
    lib().orc_features(_ptr(wl), _ptr(wr), bn, gamma, _ptr(f))
    return f


def switch_logit(params, f) -> float:
    """Logit of the switch network (bf16 inputs, weights and activations, FP64 sums)."""
    p = _vec(params, 1633)
    f = _vec(f, 16)
    return lib().orc_mlp_logit(_ptr(p), _ptr(f))


def char_eig(w, bn: float, gamma: float):
    """(eigenvalues (7,), R (7, 7) with eigenvectors as columns, L (7, 7) with
    left eigenvectors as rows) of the primitive Jacobian, Roe-Balsara normalised."""
    w = _vec(w, 7)
    lam, R, L = np.zeros(7), np.zeros((7, 7)), np.zeros((7, 7))
    lib().orc_char_eig(_ptr(w), bn, gamma, _ptr(lam), _ptr(R), _ptr(L))
    return lam, R, L


def char_slope(wm, w0, wp, bn0: float, gamma: float) -> np.ndarray:
    wm, w0, wp = _vec(wm, 7), _vec(w0, 7), _vec(wp, 7)
    out = np.zeros(7)
    lib().orc_char_slope(_ptr(wm), _ptr(w0), _ptr(wp), bn0, gamma, _ptr(out))
    return out


def switch_logits(cfg: Config, cell, face) -> np.ndarray:
    """LEARNED: the network's logit on every cell's lower face, shape (3, nz, ny, nx)."""
    assert cfg.riemann == LEARNED
    cell, face = copy_state(cell, face)
    c = cfg.c()
    cp, fp = _state_ptrs(cfg, cell, face)
    z = np.zeros((3, cfg.nz, cfg.ny, cfg.nx))
    lib().orc_switch_logits(C.byref(c), cp, fp, _ptr(z))
    return z


def cfl_dt(cfg: Config, cell, face) -> float:
    cell, face = copy_state(cell, face)
    c = cfg.c()
    cp, fp = _state_ptrs(cfg, cell, face)
    return lib().orc_cfl_dt(C.byref(c), cp, fp)


def divb_max(cfg: Config, face) -> float:
    face = [np.ascontiguousarray(f, dtype=np.float64) for f in face]
    c = cfg.c()
    fp = (_P * 3)(*[_ptr(face[d]) for d in range(3)])
    return lib().orc_divb_max(C.byref(c), fp)
