"""The GPU parity inputs reach every region of the HLLD flux.

The oracle counts, per operator evaluation, the faces whose flux comes from
each region (L, L*, L**, R**, R*, R) and the star states that take the
degenerate branch.  Over the edge cases of the GPU parity suite, both stages
of a step, every count is nonzero, so the GPU's agreement with the oracle on
those inputs covers every branch of the solver.
"""
import numpy as np

import oracle as O
from edge_cases import CASES
from helpers import ocfg


def test_edge_cases_reach_every_hlld_region_and_the_degenerate_branch():
    total = O.Stats()
    per_case = {}
    for name, make in CASES.items():
        box = make()
        st = O.Stats()
        c, f, _ = O.step(ocfg(box), box.cell, box.face, -1.0, nsteps=1, stats=st)
        assert np.isfinite(c).all(), name
        for r in O.HLLD_REGIONS:
            total.hlld_region[r] += st.hlld_region[r]
        total.hlld_degenerate += st.hlld_degenerate
        total.p_floor_hits += st.p_floor_hits
        per_case[name] = (dict(st.hlld_region), st.hlld_degenerate, st.p_floor_hits)
    missing = [r for r in O.HLLD_REGIONS if total.hlld_region[r] == 0]
    assert not missing, (missing, per_case)
    assert total.hlld_degenerate > 0, per_case
    assert total.p_floor_hits > 0, per_case
    # the regions each edge case is there for
    assert per_case["supersonic"][0]["L"] > 0 and per_case["supersonic"][0]["R"] > 0
    assert per_case["alfvenic_shear"][1] > 0
