"""Host streaming (mhd_stream_step / mhd_stream_sync): a sequence of
independent host states, each copied in, advanced one step and copied out,
with the copies overlapping neighbouring steps.  Every streamed result must
equal, bit for bit, the same step through set_state / step / get_state, and
the handle's state after the sync is the last result."""
import numpy as np
import pytest

from paper_2606_12753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,integrator", [("mixed", "rk2"), ("fp64", "rk2"), ("fp32", "rk3")])
def test_stream_matches_sequential(precision, integrator):
    import torch
    from paper_2606_12753_gb300 import mhd
    dims = (24, 20, 16)
    boxes = [I.random_state(dims, seed=s, bc=(0, 0, 0)) for s in (41, 42, 43)]
    s = mhd.Solver(boxes[0], precision=precision, integrator=integrator)
    dt_np = np.float32 if precision == "fp32" else np.float64
    ref = []
    for b in boxes:
        s.set_state(b.cell, b.face)
        s.step(-1.0, 1)
        c, f = s.get_state()
        ref.append((c.copy(), [x.copy() for x in f]))
    tdt = torch.float32 if precision == "fp32" else torch.float64
    ins = [(torch.from_numpy(b.cell.astype(dt_np)).pin_memory(),
            [torch.from_numpy(x.astype(dt_np)).pin_memory() for x in b.face]) for b in boxes]
    order = [0, 1, 2, 1, 0]
    outs = [(torch.empty(ins[0][0].shape, dtype=tdt).pin_memory(),
             [torch.empty(x.shape, dtype=tdt).pin_memory() for x in ins[0][1]]) for _ in order]
    for k, i in enumerate(order):
        s.stream_step(ins[i][0], ins[i][1], outs[k][0], outs[k][1], -1.0)
    s.stream_sync()
    for k, i in enumerate(order):
        assert np.array_equal(outs[k][0].numpy(), ref[i][0]), (k, i)
        for d in range(3):
            assert np.array_equal(outs[k][1][d].numpy(), ref[i][1][d]), (k, i, d)
    c, f = s.get_state()
    assert np.array_equal(c, ref[order[-1]][0])
    # the handle keeps working as an ordinary solver afterwards
    s.set_state(boxes[2].cell, boxes[2].face)
    s.step(-1.0, 1)
    c, f = s.get_state()
    assert np.array_equal(c, ref[2][0])
    s.close()


def test_stream_rejects_null_arrays():
    from paper_2606_12753_gb300 import mhd
    b = I.random_state((8, 8, 8), seed=1, bc=(0, 0, 0))
    s = mhd.Solver(b, precision="mixed")
    with pytest.raises(mhd.MHDError):
        mhd.mhd_stream_step(s.h, [0] * 5, [0] * 3, [0] * 5, [0] * 3, -1.0)
    s.close()
