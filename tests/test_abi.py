"""The C-ABI library loads, exports every symbol the header declares, and
rejects bad configurations on the host (no GPU needed: validation runs before
any CUDA call)."""
import ctypes as C
import os
import re

import pytest

from paper_2606_12753_gb300 import mhd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = mhd.load()
    names = declared_functions()
    assert "mhd_create" in names and "mhd_step" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    for n in mhd.EXPORTS:
        assert n in names


def test_default_config_host_only():
    c = mhd.mhd_default_config(32, 16, 8)
    assert (c.nx, c.ny, c.nz) == (32, 16, 8)
    assert c.gamma == pytest.approx(5 / 3) and c.cfl == pytest.approx(0.4)
    assert c.dx == pytest.approx(1 / 32)


@pytest.mark.parametrize("field,value", [("nx", 0), ("gamma", 1.0), ("cfl", 0.0), ("precision", 7),
                                         ("riemann", 9), ("emf", 3), ("rho_floor", 0.0), ("tile_x", 65),
                                         ("tile_y", -1), ("floor_policy", 2), ("plane_copy", 5)])
def test_invalid_config_rejected(field, value):
    c = mhd.mhd_default_config(16, 16, 16)
    setattr(c, field, value)
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert ei.value.code == mhd.MHD_ERR_INVALID
    assert mhd.mhd_last_error(None)


def test_outflow_axis_needs_two_cells():
    c = mhd.mhd_default_config(1, 16, 16)
    c.bc = (C.c_int * 3)(1, 0, 0)
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert ei.value.code == mhd.MHD_ERR_INVALID


def test_tile_smem_limit():
    c = mhd.mhd_default_config(64, 64, 64)
    c.tile_x, c.tile_y = 64, 64
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert "instantiated" in str(ei.value) or "shared memory" in str(ei.value)


def test_learned_switch_needs_the_16x8_tile():
    c = mhd.mhd_default_config(32, 32, 32)
    c.riemann = mhd.MHD_LEARNED
    c.precision = mhd.MHD_MIXED
    c.tile_x, c.tile_y = 8, 8
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert "16x8" in str(ei.value)


def test_batch_rejects_the_learned_switch():
    from paper_2606_12753_gb300 import inputs as I
    boxes = [I.uniform_state((16, 16, 16)), I.uniform_state((8, 16, 16))]
    with pytest.raises(mhd.MHDError) as ei:
        mhd.Batch(boxes, precision="fp32", riemann="learned")
    assert "learned" in str(ei.value)


def test_rk3_validation():
    from paper_2606_12753_gb300 import inputs as I
    c = mhd.mhd_default_config(32, 32, 32)
    assert c.integrator == mhd.MHD_RK2
    c.integrator = mhd.MHD_RK3
    c.tile_x, c.tile_y = 8, 8
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert "16x8" in str(ei.value)
    c.tile_x, c.tile_y = 0, 0
    c.riemann = mhd.MHD_LEARNED
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert "RK2" in str(ei.value)
    c.integrator = 7
    c.riemann = mhd.MHD_HLLD
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_create(c)
    assert "integrator" in str(ei.value)
    boxes = [I.uniform_state((16, 16, 16)), I.uniform_state((8, 16, 16))]
    cfgs = (mhd.mhd_config * 2)(*[mhd.box_config(b, "fp32") for b in boxes])
    for k in range(2):
        cfgs[k].integrator = mhd.MHD_RK3
    h = mhd.C.c_void_p()
    rc = mhd.load().mhd_batch_create(2, cfgs, None, mhd.C.byref(h))
    assert rc == mhd.MHD_ERR_INVALID


def test_char_recon_validation():
    from paper_2606_12753_gb300 import inputs as I
    c = mhd.mhd_default_config(32, 32, 32)
    assert c.recon == mhd.MHD_RECON_PRIMITIVE
    c.recon = mhd.MHD_RECON_CHARACTERISTIC
    for field, value in (("tile_x", 8), ("integrator", mhd.MHD_RK3), ("riemann", mhd.MHD_LEARNED)):
        d = mhd.mhd_config.from_buffer_copy(c)
        setattr(d, field, value)
        if field == "tile_x":
            d.tile_y = 8
        with pytest.raises(mhd.MHDError) as ei:
            mhd.mhd_create(d)
        assert "characteristic" in str(ei.value) or "16x8" in str(ei.value) or "RK2" in str(ei.value)
    c.recon = 5
    with pytest.raises(mhd.MHDError):
        mhd.mhd_create(c)
    boxes = [I.uniform_state((16, 16, 16)), I.uniform_state((8, 16, 16))]
    cfgs = (mhd.mhd_config * 2)(*[mhd.box_config(b, "fp32") for b in boxes])
    for k in range(2):
        cfgs[k].recon = mhd.MHD_RECON_CHARACTERISTIC
    h = mhd.C.c_void_p()
    assert mhd.load().mhd_batch_create(2, cfgs, None, mhd.C.byref(h)) == mhd.MHD_ERR_INVALID


def test_null_handles_and_arguments_are_rejected():
    """Every entry point that takes a handle answers a null one (or null
    output pointers) with MHD_ERR_INVALID on the host, before any CUDA call,
    and the destroy calls accept null."""
    from paper_2606_12753_gb300 import _build
    L = C.CDLL(_build.LIB)   # a separate instance: plain ctypes arguments
    P, I, D = C.c_void_p(None), C.c_int, C.c_double
    calls = {
        "mhd_set_state": (P, P, P, I(0)),
        "mhd_get_state": (P, P, P, I(0)),
        "mhd_step": (P, D(1e-3), I(1)),
        "mhd_step_async": (P, D(1e-3), I(1)),
        "mhd_stream_step": (P, P, P, P, P, D(1e-3)),
        "mhd_stream_sync": (P,),
        "mhd_set_profiling": (P, I(1)),
        "mhd_get_profile": (P, P, P),
        "mhd_rhs": (P, P, P, I(0)),
        "mhd_cfl_dt": (P, P),
        "mhd_divb_max": (P, P),
        "mhd_get_stats": (P, P),
        "mhd_dump_faces": (P, P, C.c_longlong(0), P, P, P),
        "mhd_set_switch": (P, P, D(0.5)),
        "mhd_switch_choices": (P, P, P),
        "mhd_batch_set_state": (P, I(0), P, P, I(0)),
        "mhd_batch_get_state": (P, I(0), P, P, I(0)),
        "mhd_batch_step": (P, D(-1.0), I(1)),
        "mhd_batch_step_async": (P, D(-1.0), I(1)),
        "mhd_batch_set_tile": (P, I(16), I(8), I(8)),
        "mhd_batch_get_tile": (P, P, P, P),
        "mhd_batch_autotune": (P, I(1), C.c_char_p(None), P, P),
        "mhd_batch_set_barrier_timeout": (P, D(1.0)),
        "mhd_batch_inject_missed_arrival": (P, I(1)),
        "mhd_batch_box_dt": (P, I(0), P),
        "mhd_batch_get_stats": (P, P),
        "mhd_create": (P, P, P),
        "mhd_batch_create": (I(1), P, P, P),
        "mhd_measure_pipe_peaks": (P, P),
    }
    for name, args in calls.items():
        f = getattr(L, name)
        f.restype = C.c_int
        assert f(*args) == mhd.MHD_ERR_INVALID, name
    L.mhd_destroy(P)
    L.mhd_batch_destroy(P)
    L.mhd_last_error.restype = C.c_char_p
    L.mhd_batch_last_error.restype = C.c_char_p
    assert L.mhd_last_error(P) is not None
    assert L.mhd_batch_last_error(P) is not None


def test_noalloc_rejects_the_learned_switch_on_the_host():
    """The allocation-free step runs HLLD or HLL; a learned-switch config is
    refused with its own message before any CUDA call."""
    c = mhd.mhd_default_config(8, 8, 8)
    c.riemann = mhd.MHD_LEARNED
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_step_noalloc(c, [1] * 5, [1] * 3, [1] * 5, [1] * 3, 1e-3)
    assert ei.value.code == mhd.MHD_ERR_INVALID
    assert "learned" in mhd.mhd_last_error(None)


def test_error_text_without_a_handle_is_per_thread():
    """A failed call without a handle leaves its text on its own host thread."""
    import threading
    c = mhd.mhd_default_config(16, 16, 16)
    c.gamma = 1.0
    with pytest.raises(mhd.MHDError):
        mhd.mhd_create(c)
    mine = mhd.mhd_last_error(None)
    seen = {}

    def other():
        seen["before"] = mhd.mhd_last_error(None)
        c2 = mhd.mhd_default_config(16, 16, 16)
        c2.cfl = 0.0
        try:
            mhd.mhd_create(c2)
        except mhd.MHDError:
            pass
        seen["after"] = mhd.mhd_last_error(None)

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert "gamma" in mine and seen["before"] == "" and "cfl" in seen["after"]
    assert mhd.mhd_last_error(None) == mine


def test_mlp_feature_rows_must_be_16_byte_aligned():
    """The tensor-core kernels read each feature row with 16-byte loads, so a
    misaligned feature pointer is refused on the host before any launch."""
    for call in (lambda: mhd.mlp_forward(256, 260, 10, 512),
                 lambda: mhd.mlp_backward(256, 264, 512, 10, 768)):
        with pytest.raises(mhd.MHDError) as ei:
            call()
        assert ei.value.code == mhd.MHD_ERR_INVALID
