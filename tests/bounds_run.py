"""Small cases of every kernel kind on the bounds-checked build of the library
(run in a process of its own by test_gpu_bounds.py, with
MHD_LIBRARY_VARIANT=bounds).  Prints one JSON object: per case the status the
library returned and the relative L1 error against the FP64 oracle.

In that build every index a kernel forms into global memory, every ring,
lower-face and flux-slot index into shared memory and every TMA box
coordinate is checked; one out of range raises a status bit (no trap), and
the next synchronising call returns MHD_ERR_BOUNDS.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2606_12753_gb300 import inputs as I  # noqa: E402
from paper_2606_12753_gb300 import mhd  # noqa: E402
from helpers import ocfg, state_errors  # noqa: E402


def single(box, precision, nsteps=2, **kw):
    integ = kw.get("integrator", "rk2")
    recon = 1 if kw.get("recon") == "characteristic" else 0
    cfg = ocfg(box, precision, integrator=integ, recon=recon)
    dt = O.cfl_dt(cfg, box.cell, box.face)
    dts = [dt * (1.0 - 0.05 * s) for s in range(nsteps)]
    rc, rf = O.step_dts(cfg, box.cell, box.face, dts)
    try:
        with mhd.Solver(box, precision=precision, **kw) as s:
            s.set_state(box.cell, box.face)
            for d in dts:
                s.step(d, 1)
            c, f = s.get_state()
            st = s.stats()
    except mhd.MHDError as e:
        return {"code": e.code, "error": str(e)}
    return {"code": 0, "l1": max(state_errors(c, f, rc, rf).values()), "tma_planes": st["tma_planes"]}


def batch(boxes, precision):
    dt = min(O.cfl_dt(ocfg(b, precision), b.cell, b.face) for b in boxes)
    try:
        with mhd.Batch(boxes, precision=precision, tile=(16, 8, 8)) as bt:
            for i, b in enumerate(boxes):
                bt.set_state(i, b.cell, b.face)
            bt.step(dt, 2)
            out = [bt.get_state(i) for i in range(len(boxes))]
    except mhd.MHDError as e:
        return {"code": e.code, "error": str(e)}
    worst = 0.0
    for b, (c, f) in zip(boxes, out):
        rc, rf = O.step_dts(ocfg(b, precision), b.cell, b.face, [dt, dt])
        worst = max(worst, max(state_errors(c, f, rc, rf).values()))
    return {"code": 0, "l1": worst}


def noalloc(box):
    import torch
    cfg = ocfg(box, "fp64")
    dt = O.cfl_dt(cfg, box.cell, box.face)
    rc, rf = O.step_dts(cfg, box.cell, box.face, [dt])
    ref = mhd.Solver(box, precision="fp64")
    cin = torch.tensor(box.cell, dtype=torch.float64, device="cuda")
    fin = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in box.face]
    cout = torch.empty_like(cin)
    fout = [torch.empty_like(x) for x in fin]
    try:
        mhd.mhd_step_noalloc(ref.cfg, [cin[v].data_ptr() for v in range(5)], [x.data_ptr() for x in fin],
                             [cout[v].data_ptr() for v in range(5)], [x.data_ptr() for x in fout], dt)
    except mhd.MHDError as e:
        return {"code": e.code, "error": str(e)}
    finally:
        ref.close()
    errs = state_errors(cout.cpu().numpy(), [x.cpu().numpy() for x in fout], rc, rf)
    return {"code": 0, "l1": max(errs.values())}


def main():
    assert mhd.library_variant() == "bounds", "run with MHD_LIBRARY_VARIANT=bounds"
    res = {}
    res["fp64_8cube_periodic"] = single(I.random_state((8, 8, 8), seed=81), "fp64")
    res["fp64_16cube_outflow"] = single(I.random_state((16, 16, 16), seed=82, bc=(1, 1, 1)), "fp64")
    res["fp64_2d"] = single(I.random_state((16, 16, 1), seed=83), "fp64")
    res["mixed_16cube_periodic"] = single(I.random_state((16, 16, 16), seed=84), "mixed")
    res["mixed_tma_box"] = single(I.random_state((48, 24, 10), seed=85), "mixed")
    res["fp32_16cube_outflow"] = single(I.random_state((16, 16, 16), seed=86, bc=(1, 1, 1)), "fp32")
    res["fp32_tma_box_outflow_z"] = single(I.random_state((48, 24, 10), seed=87, bc=(0, 0, 1)), "fp32")
    res["mixed_rk3"] = single(I.random_state((16, 16, 12), seed=88), "mixed", integrator="rk3")
    res["fp64_characteristic"] = single(I.random_state((16, 16, 8), seed=89), "fp64", recon="characteristic")
    res["batch_fp32"] = batch([I.random_state(d, seed=90 + i, bc=(1, 1, 1)) for i, d in
                               enumerate([(16, 16, 8), (20, 12, 9), (9, 17, 11)])], "fp32")
    res["noalloc_fp64"] = noalloc(I.random_state((12, 10, 8), seed=93))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
