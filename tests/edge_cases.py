"""The method's edge cases used by the GPU parity tests
(``test_gpu_edge_cases.py``) and by the CPU census that shows these inputs
reach every HLLD region (``test_edge_case_census.py``).

Each entry: name -> a function returning the Box.  Sizes span several tiles
of the default 16 x 8 launch and leave ragged tails.
"""
import numpy as np

from paper_2606_12753_gb300 import inputs as I


def brio_wu_3d(axis, n=80, other=(5, 3)):
    """Brio-Wu along `axis` (outflow ends), replicated over a few cells along
    the two other (periodic) axes, so that the tube runs through a 3D launch."""
    b = I.brio_wu(n, axis=axis)
    dims = [0, 0, 0]
    dims[axis] = n
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    dims[t1], dims[t2] = other
    reps = [1, 1, 1]                      # along (z, y, x) array axes
    reps[2 - t1], reps[2 - t2] = other[0], other[1]
    cell = np.ascontiguousarray(np.tile(b.cell, [1] + reps))
    face = [np.ascontiguousarray(np.tile(f, reps)) for f in b.face]
    return I.Box(dims[0], dims[1], dims[2], b.dx, b.dx, b.dx, b.bc, b.gamma, cell, face,
                 name=f"brio_wu_{'xyz'[axis]}")


CASES = {
    "brio_wu_x": lambda: brio_wu_3d(0),
    "brio_wu_y": lambda: brio_wu_3d(1),
    "brio_wu_z": lambda: brio_wu_3d(2),
    "supersonic": lambda: I.supersonic_state((37, 21, 11), seed=3),
    "transverse_field_3d": lambda: I.transverse_field_state((35, 19, 9), seed=4),
    "transverse_field_2d": lambda: I.transverse_field_state((41, 27, 1), seed=7),
    "alfvenic_shear": lambda: I.alfvenic_shear_state((34, 19, 10), seed=5),
    "near_floor": lambda: I.near_floor_state((29, 21, 11), seed=6),
}
