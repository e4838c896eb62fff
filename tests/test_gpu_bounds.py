"""The bounds-checked build on small grids (the sanitizer substitute).

A second build of the library checks every index its kernels form: global
arrays, the shared-memory ring, lower-face and flux-slot indices, and the TMA
box coordinates.  An index out of range sets a status bit (no trap, the
access goes to element 0), and the next synchronising call returns
MHD_ERR_BOUNDS.  tests/bounds_run.py runs 8^3-48x24x10 cases of every kernel
kind (FP64, mixed, FP32, 2D, outflow and periodic, TMA boxes, RK3,
characteristic reconstruction, the batch, the allocation-free step) in a
child process that loads that build; every case must end without a bounds
violation and match the FP64 oracle at its form's bar.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 1e-5}


def test_bounds_checked_build_on_small_grids():
    from paper_2606_12753_gb300 import _build
    _build.build(variant="bounds")
    env = dict(os.environ, MHD_LIBRARY_VARIANT="bounds")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_run.py")], capture_output=True, text=True,
                       env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for name, out in res.items():
        assert out["code"] == 0, (name, out)
        form = next(f for f in TOL if f in name.split("_"))
        assert out["l1"] <= TOL[form], (name, out)
    assert res["mixed_tma_box"]["tma_planes"] > 0 and res["fp32_tma_box_outflow_z"]["tma_planes"] > 0
