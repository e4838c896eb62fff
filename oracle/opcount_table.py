"""Write ``opcount_table.json``: algorithmic operation counts per cell-update of
the benchmarked workloads, from the operation-counting build of the oracle
(``opcount.py``) -- TEST INFRASTRUCTURE, calls only ``oracle/`` and the seeded
input generators.

Each workload is counted on a 32^3 periodic pattern of its own start state
(same generator and seed as the benchmark, at n = 32), tiled 1..4 times per
axis; the per-cell figure is the n^3 coefficient of a cubic fit, so ghost-layer
work drops out.  Flops: add/subtract, multiply, divide and square root count
one each (the oracle has no fused multiply-adds); compares and
abs/min/max/copysign are listed separately and not counted as flops.

    python -m oracle.opcount_table            # rewrites oracle/opcount_table.json
"""
from __future__ import annotations

import json
import os
import sys
import time

import oracle as O
from oracle import opcount as OC

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "opcount_table.json")
N0 = 32


def workloads():
    from paper_2606_12753_gb300 import inputs as I
    return {
        # name: (start state, integrator, reconstruction)
        "turbulence_3d (RK2, PLM-MC primitive, HLLD, upwind CT)": (I.turbulence_3d(N0, seed=2606), "rk2", 0),
        "turbulence_3d (RK2, PLM-MC characteristic, HLLD, upwind CT)": (I.turbulence_3d(N0, seed=2606), "rk2", 1),
        "orszag_tang_3d (RK2, PLM-MC primitive, HLLD, upwind CT)": (I.orszag_tang_3d(N0, seed=12753), "rk2", 0),
        "orszag_tang_3d (SSP-RK3, PLM-MC primitive, HLLD, upwind CT)": (I.orszag_tang_3d(N0, seed=12753), "rk3", 0),
    }


def main(n0: int = N0) -> dict:
    table = {"pattern_n": n0, "tiles": [1, 2, 3, 4], "unit": "operations per cell-update (one full step)",
             "flop_categories": list(OC.FLOP_CATEGORIES), "workloads": {}}
    for name, (box, integ, recon) in workloads().items():
        t = time.time()
        cfg = O.Config(n0, n0, n0, box.dx, box.dy, box.dz, gamma=box.gamma, integrator=integ, recon=recon)
        dt = O.cfl_dt(cfg, box.cell, box.face)
        pc = OC.per_cell(cfg, box.cell, box.face, dt)
        sp = OC.split(pc)
        table["workloads"][name] = {"counts": {k: {c: round(v, 3) for c, v in d.items()} for k, d in pc.items()},
                                    "flops": {k: round(v, 3) for k, v in sp.items()}}
        print(f"{name}: {sp['total']:.1f} flops per cell-update ({time.time() - t:.1f} s)", file=sys.stderr)
    return table


if __name__ == "__main__":
    tab = main()
    with open(OUT, "w") as f:
        json.dump(tab, f, indent=1)
        f.write("\n")
    print(OUT)
