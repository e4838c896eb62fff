"""ctypes binding of the C ABI in ``include/mhd_gb300.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``libmhd_gb300.so``.  The functions keep the C names (``mhd_create``,
``mhd_set_state``, ``mhd_step``, ...); :class:`Solver` is a thin owner of one
handle that moves numpy arrays (host) or torch CUDA tensors (device) through
those calls.  There is no CPU fallback: if the library is missing or cannot be
loaded, importing it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MHD_OK = 0
MHD_ERR_INVALID, MHD_ERR_CUDA, MHD_ERR_NONFINITE, MHD_ERR_TIMEOUT, MHD_ERR_NOMEM, MHD_ERR_FLOOR = -1, -2, -3, -4, -5, -6
MHD_ERR_BOUNDS = -7
MHD_FLOOR_COUNT, MHD_FLOOR_ERROR = 0, 1
MHD_COPY_AUTO, MHD_COPY_GATHER = 0, 1
MHD_BC_PERIODIC, MHD_BC_OUTFLOW = 0, 1
MHD_FP64, MHD_MIXED, MHD_FP32 = 0, 1, 2
MHD_HLLD, MHD_HLL, MHD_LEARNED = 0, 1, 2
MHD_EMF_UPWIND, MHD_EMF_MEAN = 0, 1
MHD_RK2, MHD_RK3 = 0, 1
MHD_RECON_PRIMITIVE, MHD_RECON_CHARACTERISTIC = 0, 1
RECONS = {"primitive": MHD_RECON_PRIMITIVE, "characteristic": MHD_RECON_CHARACTERISTIC}
INTEGRATORS = {"rk2": MHD_RK2, "rk3": MHD_RK3}

PRECISIONS = {"fp64": MHD_FP64, "mixed": MHD_MIXED, "fp32": MHD_FP32}
RIEMANN = {"hlld": MHD_HLLD, "hll": MHD_HLL, "learned": MHD_LEARNED}


class mhd_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("gamma", C.c_double), ("cfl", C.c_double),
                ("bc", C.c_int * 3),
                ("precision", C.c_int), ("riemann", C.c_int), ("emf", C.c_int),
                ("rho_floor", C.c_double), ("p_floor", C.c_double),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("tile_z", C.c_int),
                ("integrator", C.c_int), ("recon", C.c_int), ("floor_policy", C.c_int), ("plane_copy", C.c_int)]


class mhd_stats(C.Structure):
    _fields_ = [("rho_floor_hits", C.c_longlong), ("p_floor_hits", C.c_longlong),
                ("faces_hll", C.c_longlong), ("faces_hlld", C.c_longlong),
                ("last_dt", C.c_double), ("status", C.c_int), ("steps", C.c_int), ("tma_planes", C.c_longlong)]


class mhd_pipe_peaks(C.Structure):
    _fields_ = [("fp64_fma_tflops", C.c_double), ("fp32_fma_tflops", C.c_double),
                ("bf16_mma_sync_tflops", C.c_double), ("ms", C.c_double * 3)]


class MHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_VP = C.c_void_p
_H = C.c_void_p
EXPORTS = ["mhd_default_config", "mhd_create", "mhd_set_state", "mhd_get_state", "mhd_step",
           "mhd_step_async", "mhd_rhs", "mhd_set_profiling", "mhd_get_profile", "mhd_cfl_dt", "mhd_divb_max",
           "mhd_get_stats", "mhd_destroy", "mhd_last_error", "mhd_step_noalloc",
           "mhd_batch_create", "mhd_batch_set_state", "mhd_batch_get_state", "mhd_batch_step",
           "mhd_batch_step_async", "mhd_batch_set_tile", "mhd_batch_get_tile", "mhd_batch_autotune",
           "mhd_batch_set_barrier_timeout", "mhd_batch_inject_missed_arrival", "mhd_batch_box_dt",
           "mhd_batch_get_stats", "mhd_batch_destroy", "mhd_batch_last_error",
           "mlp_param_bytes", "mlp_init", "mlp_forward", "mlp_backward", "mlp_adam", "mhd_dump_faces",
           "mhd_set_switch", "mhd_switch_choices", "mhd_measure_pipe_peaks", "mhd_stream_step",
           "mhd_stream_sync"]

_lib = None


def library_variant() -> str:
    """Which build of the library this process loads: "release", or
    "bounds" (every kernel index checked) when MHD_LIBRARY_VARIANT says so."""
    v = os.environ.get("MHD_LIBRARY_VARIANT", "release")
    if v not in _build.VARIANTS:
        raise RuntimeError(f"unknown MHD_LIBRARY_VARIANT {v!r} (one of {sorted(_build.VARIANTS)})")
    return v


def library_path() -> str:
    return _build.variant_path(library_variant())


def load(build: bool = True):
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    variant = library_variant()
    path = _build.variant_path(variant)
    if build and _build.needs_build(variant):
        _build.build(variant=variant)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    L.mhd_default_config.restype = None
    L.mhd_default_config.argtypes = [C.POINTER(mhd_config), C.c_int, C.c_int, C.c_int]
    L.mhd_create.restype = C.c_int
    L.mhd_create.argtypes = [C.POINTER(mhd_config), _VP, C.POINTER(_H)]
    L.mhd_set_state.restype = C.c_int
    L.mhd_set_state.argtypes = [_H, _VP * 5, _VP * 3, C.c_int]
    L.mhd_get_state.restype = C.c_int
    L.mhd_get_state.argtypes = [_H, _VP * 5, _VP * 3, C.c_int]
    L.mhd_step.restype = C.c_int
    L.mhd_step.argtypes = [_H, C.c_double, C.c_int]
    L.mhd_step_async.restype = C.c_int
    L.mhd_step_async.argtypes = [_H, C.c_double, C.c_int]
    L.mhd_rhs.restype = C.c_int
    L.mhd_rhs.argtypes = [_H, _VP * 5, _VP * 3, C.c_int]
    L.mhd_set_profiling.restype = C.c_int
    L.mhd_set_profiling.argtypes = [_H, C.c_int]
    L.mhd_get_profile.restype = C.c_int
    L.mhd_get_profile.argtypes = [_H, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.mhd_cfl_dt.restype = C.c_int
    L.mhd_cfl_dt.argtypes = [_H, C.POINTER(C.c_double)]
    L.mhd_divb_max.restype = C.c_int
    L.mhd_divb_max.argtypes = [_H, C.POINTER(C.c_double)]
    L.mhd_get_stats.restype = C.c_int
    L.mhd_get_stats.argtypes = [_H, C.POINTER(mhd_stats)]
    L.mhd_destroy.restype = None
    L.mhd_destroy.argtypes = [_H]
    L.mhd_step_noalloc.restype = C.c_int
    L.mhd_step_noalloc.argtypes = [C.POINTER(mhd_config), _VP, _VP * 5, _VP * 3, _VP * 5, _VP * 3, C.c_double,
                                   C.POINTER(C.c_double)]
    L.mhd_batch_create.restype = C.c_int
    L.mhd_batch_create.argtypes = [C.c_int, C.POINTER(mhd_config), _VP, C.POINTER(_H)]
    for name in ("mhd_batch_set_state", "mhd_batch_get_state"):
        getattr(L, name).restype = C.c_int
        getattr(L, name).argtypes = [_H, C.c_int, _VP * 5, _VP * 3, C.c_int]
    for name in ("mhd_batch_step", "mhd_batch_step_async"):
        getattr(L, name).restype = C.c_int
        getattr(L, name).argtypes = [_H, C.c_double, C.c_int]
    L.mhd_batch_set_tile.restype = C.c_int
    L.mhd_batch_set_tile.argtypes = [_H, C.c_int, C.c_int, C.c_int]
    L.mhd_batch_get_tile.restype = C.c_int
    L.mhd_batch_get_tile.argtypes = [_H, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
    L.mhd_batch_autotune.restype = C.c_int
    L.mhd_batch_autotune.argtypes = [_H, C.c_int, C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.mhd_batch_set_barrier_timeout.restype = C.c_int
    L.mhd_batch_set_barrier_timeout.argtypes = [_H, C.c_double]
    L.mhd_batch_inject_missed_arrival.restype = C.c_int
    L.mhd_batch_inject_missed_arrival.argtypes = [_H, C.c_int]
    L.mhd_batch_box_dt.restype = C.c_int
    L.mhd_batch_box_dt.argtypes = [_H, C.c_int, C.POINTER(C.c_double)]
    L.mhd_batch_get_stats.restype = C.c_int
    L.mhd_batch_get_stats.argtypes = [_H, C.POINTER(mhd_stats)]
    L.mhd_batch_destroy.restype = None
    L.mhd_batch_destroy.argtypes = [_H]
    L.mhd_batch_last_error.restype = C.c_char_p
    L.mhd_batch_last_error.argtypes = [_H]
    L.mlp_param_bytes.restype = C.c_size_t
    L.mlp_param_bytes.argtypes = []
    L.mlp_init.restype = C.c_int
    L.mlp_init.argtypes = [_VP, C.POINTER(C.c_float), _VP]
    L.mlp_forward.restype = C.c_int
    L.mlp_forward.argtypes = [_VP, _VP, C.c_longlong, _VP, _VP]
    L.mlp_backward.restype = C.c_int
    L.mlp_backward.argtypes = [_VP, _VP, _VP, C.c_longlong, _VP, _VP]
    L.mlp_adam.restype = C.c_int
    L.mlp_adam.argtypes = [_VP, _VP, _VP, _VP, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, _VP]
    L.mhd_dump_faces.restype = C.c_int
    L.mhd_dump_faces.argtypes = [_H, _VP, C.c_longlong, _VP, _VP, _VP]
    L.mhd_set_switch.restype = C.c_int
    L.mhd_set_switch.argtypes = [_H, _VP, C.c_double]
    L.mhd_switch_choices.restype = C.c_int
    L.mhd_switch_choices.argtypes = [_H, _VP, _VP]
    L.mhd_stream_step.restype = C.c_int
    L.mhd_stream_step.argtypes = [_H, _VP * 5, _VP * 3, _VP * 5, _VP * 3, C.c_double]
    L.mhd_stream_sync.restype = C.c_int
    L.mhd_stream_sync.argtypes = [_H]
    L.mhd_measure_pipe_peaks.restype = C.c_int
    L.mhd_measure_pipe_peaks.argtypes = [_VP, C.POINTER(mhd_pipe_peaks)]
    L.mhd_last_error.restype = C.c_char_p
    L.mhd_last_error.argtypes = [_H]
    _lib = L
    return L


# ---- the C calls under their own names -------------------------------------

def mhd_default_config(nx, ny, nz) -> mhd_config:
    c = mhd_config()
    load().mhd_default_config(C.byref(c), nx, ny, nz)
    return c


def _check(h, rc):
    if rc != MHD_OK:
        msg = load().mhd_last_error(h)
        raise MHDError(rc, msg.decode() if msg else "")


def mhd_create(cfg: mhd_config, stream=None):
    h = _H()
    rc = load().mhd_create(C.byref(cfg), _VP(stream or 0), C.byref(h))
    _check(None, rc)
    return h


def mhd_set_state(h, cell_ptrs, face_ptrs, on_device: int):
    _check(h, load().mhd_set_state(h, (_VP * 5)(*cell_ptrs), (_VP * 3)(*face_ptrs), on_device))


def mhd_get_state(h, cell_ptrs, face_ptrs, on_device: int):
    _check(h, load().mhd_get_state(h, (_VP * 5)(*cell_ptrs), (_VP * 3)(*face_ptrs), on_device))


def mhd_step(h, dt: float, nsteps: int = 1):
    _check(h, load().mhd_step(h, dt, nsteps))


def mhd_step_async(h, dt: float, nsteps: int = 1):
    _check(h, load().mhd_step_async(h, dt, nsteps))


def mhd_rhs(h, cell_ptrs, face_ptrs, on_device: int):
    _check(h, load().mhd_rhs(h, (_VP * 5)(*cell_ptrs), (_VP * 3)(*face_ptrs), on_device))


def mhd_set_profiling(h, on: bool):
    _check(h, load().mhd_set_profiling(h, 1 if on else 0))


def mhd_get_profile(h):
    """(ms per stage kernel, launches per stage kernel): 3 entries, the third
    used by RK3 only."""
    ms = (C.c_double * 3)()
    n = (C.c_longlong * 3)()
    _check(h, load().mhd_get_profile(h, ms, n))
    return [ms[0], ms[1], ms[2]], [n[0], n[1], n[2]]


def mhd_cfl_dt(h) -> float:
    out = C.c_double()
    _check(h, load().mhd_cfl_dt(h, C.byref(out)))
    return out.value


def mhd_divb_max(h) -> float:
    out = C.c_double()
    _check(h, load().mhd_divb_max(h, C.byref(out)))
    return out.value


def mhd_stream_step(h, cell_in, face_in, cell_out, face_out, dt: float):
    """Enqueue copy-in, one step and copy-out of one host state (pointers)."""
    _check(h, load().mhd_stream_step(h, (_VP * 5)(*cell_in), (_VP * 3)(*face_in), (_VP * 5)(*cell_out),
                                     (_VP * 3)(*face_out), dt))


def mhd_stream_sync(h):
    _check(h, load().mhd_stream_sync(h))


def mhd_measure_pipe_peaks(stream=None) -> dict:
    """Measured FP64-FMA, FP32-FMA and BF16 mma.sync peaks (TFLOP/s) of the current device."""
    p = mhd_pipe_peaks()
    _check(None, load().mhd_measure_pipe_peaks(_VP(stream or 0), C.byref(p)))
    return {"fp64_fma_tflops": p.fp64_fma_tflops, "fp32_fma_tflops": p.fp32_fma_tflops,
            "bf16_mma_sync_tflops": p.bf16_mma_sync_tflops, "ms": list(p.ms)}


def mhd_get_stats(h) -> dict:
    s = mhd_stats()
    _check(h, load().mhd_get_stats(h, C.byref(s)))
    return {k: getattr(s, k) for k, _ in mhd_stats._fields_}


def mhd_destroy(h):
    if h:
        load().mhd_destroy(h)


def mhd_step_noalloc(cfg: mhd_config, cell_in, face_in, cell_out, face_out, dt: float, stream=None) -> float:
    """One RK2 step that allocates no device memory (see include/mhd_gb300.h).
    The pointer lists hold device addresses; returns the dt taken."""
    used = C.c_double(0.0)
    rc = load().mhd_step_noalloc(C.byref(cfg), _VP(stream or 0), (_VP * 5)(*cell_in), (_VP * 3)(*face_in),
                                 (_VP * 5)(*cell_out), (_VP * 3)(*face_out), dt, C.byref(used))
    _check(None, rc)
    return used.value


def mhd_last_error(h=None) -> str:
    m = load().mhd_last_error(h)
    return m.decode() if m else ""


# ---- convenience owner -----------------------------------------------------

class Solver:
    """One box on the GPU.  ``box`` is any object with nx, ny, nz, dx, dy, dz,
    bc, gamma (and optionally cfl) -- e.g. ``inputs.Box``."""

    def __init__(self, box, precision="fp64", riemann="hlld", emf="upwind", tile=(0, 0, 0),
                 stream=None, cfl=None, rho_floor=1e-10, p_floor=1e-10, integrator="rk2", recon="primitive",
                 floor_policy="count", plane_copy="auto"):
        c = mhd_default_config(box.nx, box.ny, box.nz)
        c.dx, c.dy, c.dz = box.dx, box.dy, box.dz
        c.gamma = box.gamma
        c.cfl = cfl if cfl is not None else getattr(box, "cfl", 0.4)
        c.bc = (C.c_int * 3)(*box.bc)
        c.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        c.riemann = RIEMANN[riemann] if isinstance(riemann, str) else riemann
        c.emf = MHD_EMF_MEAN if emf == "mean" else MHD_EMF_UPWIND
        c.rho_floor, c.p_floor = rho_floor, p_floor
        c.tile_x, c.tile_y, c.tile_z = tile
        c.integrator = INTEGRATORS[integrator] if isinstance(integrator, str) else integrator
        c.recon = RECONS[recon] if isinstance(recon, str) else recon
        c.floor_policy = {"count": MHD_FLOOR_COUNT, "error": MHD_FLOOR_ERROR}[floor_policy]
        c.plane_copy = {"auto": MHD_COPY_AUTO, "gather": MHD_COPY_GATHER}[plane_copy]
        self.cfg = c
        self.dims = (box.nx, box.ny, box.nz)
        self.bc = tuple(box.bc)
        self.dtype = np.float32 if c.precision == MHD_FP32 else np.float64
        self.h = mhd_create(c, stream)

    def face_shapes(self):
        nx, ny, nz = self.dims
        o = [1 if b == MHD_BC_OUTFLOW else 0 for b in self.bc]
        return [(nz, ny, nx + o[0]), (nz, ny + o[1], nx), (nz + o[2], ny, nx)]

    def set_state(self, cell, face):
        """Host numpy arrays (converted to the handle's element type) or torch
        CUDA tensors of that type."""
        if hasattr(cell, "data_ptr") and getattr(cell, "is_cuda", False):
            cp = [cell[v].data_ptr() for v in range(5)]
            fp = [f.data_ptr() for f in face]
            for t in [cell] + list(face):
                assert t.is_contiguous()
            mhd_set_state(self.h, cp, fp, 1)
            return
        self._keep = [np.ascontiguousarray(cell, dtype=self.dtype)] + \
                     [np.ascontiguousarray(f, dtype=self.dtype) for f in face]
        c = self._keep[0]
        assert c.shape == (5,) + self.dims[::-1], c.shape
        for f, s in zip(self._keep[1:], self.face_shapes()):
            assert f.shape == s, (f.shape, s)
        mhd_set_state(self.h, [c[v].ctypes.data for v in range(5)], [f.ctypes.data for f in self._keep[1:]], 0)

    def get_state(self):
        cell = np.empty((5,) + self.dims[::-1], dtype=self.dtype)
        face = [np.empty(s, dtype=self.dtype) for s in self.face_shapes()]
        mhd_get_state(self.h, [cell[v].ctypes.data for v in range(5)], [f.ctypes.data for f in face], 0)
        return cell, face

    def rhs(self):
        """L(U) of the current state as (dU/dt cells, [dBx/dt, dBy/dt, dBz/dt])
        in the increment type (float64 for fp64, float32 otherwise)."""
        kt = np.float64 if self.cfg.precision == MHD_FP64 else np.float32
        cell = np.empty((5,) + self.dims[::-1], dtype=kt)
        face = [np.empty(s, dtype=kt) for s in self.face_shapes()]
        mhd_rhs(self.h, [cell[v].ctypes.data for v in range(5)], [f.ctypes.data for f in face], 0)
        return cell, face

    def step(self, dt: float, nsteps: int = 1):
        mhd_step(self.h, dt, nsteps)

    def step_async(self, dt: float, nsteps: int = 1):
        mhd_step_async(self.h, dt, nsteps)

    def stream_step(self, cell_in, face_in, cell_out, face_out, dt: float = -1.0):
        """Enqueue one streamed step of a host state: arrays with ``data_ptr``
        (pinned torch CPU tensors) or numpy arrays of the handle's element
        type, which must stay alive and untouched until stream_sync()."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        mhd_stream_step(self.h, [ptr(cell_in[v]) for v in range(5)], [ptr(f) for f in face_in],
                        [ptr(cell_out[v]) for v in range(5)], [ptr(f) for f in face_out], dt)

    def stream_sync(self):
        mhd_stream_sync(self.h)

    def cfl_dt(self) -> float:
        return mhd_cfl_dt(self.h)

    def set_profiling(self, on: bool):
        mhd_set_profiling(self.h, on)

    def profile(self):
        """(ms per stage kernel, launches per stage kernel) since the last call."""
        return mhd_get_profile(self.h)

    def divb_max(self) -> float:
        return mhd_divb_max(self.h)

    def stats(self) -> dict:
        return mhd_get_stats(self.h)

    def set_switch(self, block_ptr, tau: float):
        """Network (device parameter block, copied) and threshold of the learned switch."""
        mhd_set_switch(self.h, block_ptr, tau)

    def switch_choices(self, choices_ptr, logits_ptr=None):
        """Per-face choices (device uint8[3 * ncell], 1 = HLLD) and logits of the current state."""
        mhd_switch_choices(self.h, choices_ptr, logits_ptr)

    def close(self):
        if self.h:
            mhd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batches ---------------------------------------------------------------

def _bcheck(b, rc):
    if rc != MHD_OK:
        msg = load().mhd_batch_last_error(b)
        raise MHDError(rc, msg.decode() if msg else "")


def box_config(box, precision="fp32", riemann="hlld", emf="upwind", tile=(0, 0, 0), cfl=None):
    c = mhd_default_config(box.nx, box.ny, box.nz)
    c.dx, c.dy, c.dz = box.dx, box.dy, box.dz
    c.gamma = box.gamma
    c.cfl = cfl if cfl is not None else getattr(box, "cfl", 0.4)
    c.bc = (C.c_int * 3)(*box.bc)
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
    c.riemann = RIEMANN[riemann] if isinstance(riemann, str) else riemann
    c.emf = MHD_EMF_MEAN if emf == "mean" else MHD_EMF_UPWIND
    c.tile_x, c.tile_y, c.tile_z = tile
    return c


class Batch:
    """Many boxes advanced in one persistent launch (``mhd_batch_*``)."""

    def __init__(self, boxes, precision="fp32", riemann="hlld", emf="upwind", tile=(0, 0, 0), stream=None):
        cfgs = (mhd_config * len(boxes))(*[box_config(b, precision, riemann, emf, tile) for b in boxes])
        h = _H()
        _bcheck(None, load().mhd_batch_create(len(boxes), cfgs, _VP(stream or 0), C.byref(h)))
        self.h = h
        self.boxes = boxes
        self.cfgs = cfgs
        self.dtype = np.float32 if cfgs[0].precision == MHD_FP32 else np.float64

    def _shapes(self, i):
        b = self.boxes[i]
        o = [1 if x == MHD_BC_OUTFLOW else 0 for x in b.bc]
        return (5, b.nz, b.ny, b.nx), [(b.nz, b.ny, b.nx + o[0]), (b.nz, b.ny + o[1], b.nx), (b.nz + o[2], b.ny, b.nx)]

    def set_state(self, i, cell, face):
        cs, fs = self._shapes(i)
        c = np.ascontiguousarray(cell, dtype=self.dtype)
        f = [np.ascontiguousarray(x, dtype=self.dtype) for x in face]
        assert c.shape == cs and [x.shape for x in f] == fs
        _bcheck(self.h, load().mhd_batch_set_state(self.h, i, (_VP * 5)(*[c[v].ctypes.data for v in range(5)]),
                                                   (_VP * 3)(*[x.ctypes.data for x in f]), 0))

    def get_state(self, i):
        cs, fs = self._shapes(i)
        c = np.empty(cs, dtype=self.dtype)
        f = [np.empty(s, dtype=self.dtype) for s in fs]
        _bcheck(self.h, load().mhd_batch_get_state(self.h, i, (_VP * 5)(*[c[v].ctypes.data for v in range(5)]),
                                                   (_VP * 3)(*[x.ctypes.data for x in f]), 0))
        return c, f

    def step(self, dt, nsteps=1):
        _bcheck(self.h, load().mhd_batch_step(self.h, dt, nsteps))

    def step_async(self, dt, nsteps=1):
        _bcheck(self.h, load().mhd_batch_step_async(self.h, dt, nsteps))

    def set_tile(self, tx, ty, tz):
        _bcheck(self.h, load().mhd_batch_set_tile(self.h, tx, ty, tz))

    def tile(self):
        t = (C.c_int * 3)()
        items = C.c_longlong()
        grid = C.c_int()
        _bcheck(self.h, load().mhd_batch_get_tile(self.h, t, C.byref(items), C.byref(grid)))
        return (t[0], t[1], t[2]), items.value, grid.value

    def autotune(self, trial_steps=3, cache_path=None):
        t = (C.c_int * 3)()
        ms = C.c_double()
        _bcheck(self.h, load().mhd_batch_autotune(self.h, trial_steps, cache_path.encode() if cache_path else None,
                                                  t, C.byref(ms)))
        return (t[0], t[1], t[2]), ms.value

    def set_barrier_timeout(self, seconds):
        _bcheck(self.h, load().mhd_batch_set_barrier_timeout(self.h, seconds))

    def inject_missed_arrival(self, on=True):
        _bcheck(self.h, load().mhd_batch_inject_missed_arrival(self.h, 1 if on else 0))

    def box_dt(self, i):
        out = C.c_double()
        _bcheck(self.h, load().mhd_batch_box_dt(self.h, i, C.byref(out)))
        return out.value

    def stats(self):
        s = mhd_stats()
        _bcheck(self.h, load().mhd_batch_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in mhd_stats._fields_}

    def close(self):
        if self.h:
            load().mhd_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned face switch ------------------------------------------------------

MLP_NPARAM = 1633


def mlp_param_bytes() -> int:
    return int(load().mlp_param_bytes())


def _rc(rc, what):
    if rc != MHD_OK:
        raise MHDError(rc, what)


def mlp_init(block_ptr, master_host: np.ndarray, stream=None):
    m = np.ascontiguousarray(master_host, dtype=np.float32)
    assert m.size == MLP_NPARAM
    _rc(load().mlp_init(_VP(block_ptr), m.ctypes.data_as(C.POINTER(C.c_float)), _VP(stream or 0)), "mlp_init")


def mlp_forward(block_ptr, x_ptr, n, z_ptr, stream=None):
    _rc(load().mlp_forward(_VP(block_ptr), _VP(x_ptr), n, _VP(z_ptr), _VP(stream or 0)), "mlp_forward")


def mlp_backward(block_ptr, x_ptr, y_ptr, n, grad_ptr, stream=None):
    _rc(load().mlp_backward(_VP(block_ptr), _VP(x_ptr), _VP(y_ptr), n, _VP(grad_ptr), _VP(stream or 0)),
        "mlp_backward")


def mlp_adam(block_ptr, m_ptr, v_ptr, grad_ptr, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _rc(load().mlp_adam(_VP(block_ptr), _VP(m_ptr), _VP(v_ptr), _VP(grad_ptr), step, lr, beta1, beta2, eps,
                        _VP(stream or 0)), "mlp_adam")


def mhd_dump_faces(h, ids_ptr, n, x_ptr, y_ptr, score_ptr=None):
    _check(h, load().mhd_dump_faces(h, _VP(ids_ptr), n, _VP(x_ptr), _VP(y_ptr), _VP(score_ptr or 0)))


def mhd_set_switch(h, block_ptr, tau):
    _check(h, load().mhd_set_switch(h, _VP(block_ptr), tau))


def mhd_switch_choices(h, choices_ptr, logits_ptr=None):
    _check(h, load().mhd_switch_choices(h, _VP(choices_ptr), _VP(logits_ptr or 0)))
