"""What the trained switch gains over the method without it.  A network is
trained on the GPU on faces of FP64 turbulence runs (seed 5) and used on an
unseen start (seed 77) in the mixed-precision step; against the FP64 HLLD
path (itself held to the oracle at 1e-12) it is compared with the method
without the switch (HLLD on every face) and with HLL on every face, on the
same dt sequence: error, fraction of faces cleared for HLL, time per step."""
import numpy as np
import pytest

from paper_2606_12753_gb300 import inputs as I
from helpers import state_errors

pytestmark = pytest.mark.gpu

N, STEPS = 64, 20


def _run(box, precision, riemann, dts, sw=None, tau=None):
    import torch
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, riemann=riemann)
    if sw is not None:
        s.set_switch(sw.block.data_ptr(), tau)
    s.set_state(box.cell, box.face)
    s.step(float(dts[0]), 1)                       # warm-up launch outside the timing
    s.set_state(box.cell, box.face)
    st0 = s.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for h in dts:
        s.step_async(float(h), 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / len(dts)
    st = s.stats()
    out = s.get_state()
    s.close()
    return out, ms, st["faces_hll"] - st0["faces_hll"], st["faces_hlld"] - st0["faces_hlld"]


def test_trained_switch_gain():
    from paper_2606_12753_gb300 import mhd, switch_train as T
    sw, tau, rep = T.train_switch(n=N, nfaces=1_000_000, seed=5, steps=1500, batch=8192,
                                  snapshots=(2, 6, 12, 24))
    print("\ntraining:", rep)
    assert rep["val_loss"] < 0.6 * rep["val_loss_init"], rep
    assert rep["val_recall"] >= 0.99, rep
    assert 0.0 < rep["label1_frac"] < 1.0
    box = I.turbulence_3d(N, seed=77)
    # dt sequence of the FP64 HLLD reference
    s = mhd.Solver(box, precision="fp64")
    s.set_state(box.cell, box.face)
    dts = []
    for _ in range(STEPS):
        dts.append(s.cfl_dt())
        s.step(dts[-1], 1)
    ref = s.get_state()
    s.close()
    res = {}
    for name, riemann in (("hlld", "hlld"), ("hll", "hll"), ("learned", "learned")):
        kw = {"sw": sw, "tau": tau} if riemann == "learned" else {}
        (c, f), ms, nh, nd = _run(box, "mixed", riemann, dts, **kw)
        err = state_errors(c, f, ref[0], ref[1])
        res[name] = {"err_max": max(err.values()), "err_rho": err["rho"], "ms": ms,
                     "hll_frac": nh / max(nh + nd, 1)}
    print("gain:", res)
    hlld, hll, lrn = res["hlld"], res["hll"], res["learned"]
    # the switch keeps most of HLLD's accuracy over HLL everywhere ...
    assert lrn["err_max"] < 0.5 * hll["err_max"], res
    # ... while clearing a real share of the faces for the cheaper solver
    assert lrn["hll_frac"] > 0.1, res
    assert hll["hll_frac"] == 0.0 and hlld["hll_frac"] == 0.0   # counters only count the learned mode
