"""The allocation-free RK2 step against the regular entry point.

mhd_step_noalloc exists for callers that must not allocate device memory
while they run (services that reserve their memory up front, frameworks whose
pool accounts for every byte, loops that cannot absorb the synchronisation an
allocation may cause).  It keeps its scratch in a static device array of
MHD_NOALLOC_SCRATCH_BYTES; these tests call it through the C ABI twice in a
row (the second call starts from the first call's output, so the shared
scratch is reused) and compare each result with mhd_step on the same state.
This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2606_12753_gb300 import inputs as I
from helpers import state_errors

pytestmark = pytest.mark.gpu


def _device_state(torch, cell, face, dtype):
    c = torch.tensor(np.asarray(cell), dtype=dtype, device="cuda")
    f = [torch.tensor(np.asarray(x), dtype=dtype, device="cuda") for x in face]
    return c, f


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_noalloc_step_matches_regular_step_twice(precision):
    """Both entry points launch the same kernels on the same state with the
    same dt, so their results are equal bit for bit (a wrong offset into the
    scratch, or two buffers aliased in it, would move results by far less
    than the oracle tolerances)."""
    import torch
    from paper_2606_12753_gb300 import mhd

    box = I.random_state((24, 20, 12), seed=77, bc=(0, 1, 0))
    ref = mhd.Solver(box, precision=precision)
    ref.set_state(box.cell, box.face)
    dt = 0.8 * ref.cfl_dt()
    cfg = ref.cfg
    tdtype = torch.float32 if precision == "fp32" else torch.float64

    cin, fin = _device_state(torch, box.cell, box.face, tdtype)
    cout = torch.empty_like(cin)
    fout = [torch.empty_like(x) for x in fin]
    torch.cuda.synchronize()
    for call in range(2):
        # the regular entry point from the same input state (its primitives
        # recovered afresh, as the allocation-free call does)
        ref.set_state(cin, fin)
        used = mhd.mhd_step_noalloc(cfg, [cin[v].data_ptr() for v in range(5)], [x.data_ptr() for x in fin],
                                    [cout[v].data_ptr() for v in range(5)], [x.data_ptr() for x in fout], dt)
        assert used == dt
        ref.step(dt, 1)
        rc, rf = ref.get_state()
        gc = cout.cpu().numpy()
        gf = [x.cpu().numpy() for x in fout]
        assert gc.dtype == rc.dtype
        assert np.array_equal(gc, rc), (call, state_errors(gc, gf, rc, rf))
        for d in range(3):
            assert np.array_equal(gf[d], rf[d]), (call, d)
        cin, cout = cout, cin
        fin, fout = fout, fin
    ref.close()


def test_noalloc_cfl_dt_and_size_limit():
    import torch
    from paper_2606_12753_gb300 import mhd

    box = I.random_state((16, 12, 10), seed=78)
    ref = mhd.Solver(box, precision="fp64")
    ref.set_state(box.cell, box.face)
    dt_ref = ref.cfl_dt()
    cin, fin = _device_state(torch, box.cell, box.face, torch.float64)
    cout = torch.empty_like(cin)
    fout = [torch.empty_like(x) for x in fin]
    used = mhd.mhd_step_noalloc(ref.cfg, [cin[v].data_ptr() for v in range(5)], [x.data_ptr() for x in fin],
                                [cout[v].data_ptr() for v in range(5)], [x.data_ptr() for x in fout], -1.0)
    assert used == pytest.approx(dt_ref, rel=1e-12)
    ref.step(used, 1)
    rc, rf = ref.get_state()
    errs = state_errors(cout.cpu().numpy(), [x.cpu().numpy() for x in fout], rc, rf)
    assert max(errs.values()) <= 1e-12, errs
    ref.close()
    # a box beyond the static scratch is refused before any device work
    big = mhd.mhd_default_config(64, 64, 64)
    with pytest.raises(mhd.MHDError) as ei:
        mhd.mhd_step_noalloc(big, [1] * 5, [1] * 3, [1] * 5, [1] * 3, 1e-3)
    assert ei.value.code == mhd.MHD_ERR_INVALID
    assert "MHD_NOALLOC_SCRATCH_BYTES" in mhd.mhd_last_error(None)
