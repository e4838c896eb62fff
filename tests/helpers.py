"""Shared helpers of the test suite (error metrics, oracle configs)."""
import numpy as np

import oracle as O


def ocfg(b, **kw):
    return O.Config(b.nx, b.ny, b.nz, b.dx, b.dy, b.dz, b.gamma, getattr(b, "cfl", 0.4), tuple(b.bc), **kw)


def rel_l1(q, ref, floor=0.0):
    """Relative L1 error sum|q - ref| / max(sum|ref|, floor); with a zero
    denominator, the mean absolute error instead."""
    q = np.asarray(q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = max(float(np.abs(ref).sum()), floor)
    num = float(np.abs(q - ref).sum())
    return num / den if den > 0 else num / max(ref.size, 1)


def state_errors(cell, face, ref_cell, ref_face):
    """Per-variable relative L1 errors.  A vector component is measured
    against max(its own L1 norm, 1e-3 x the L1 norm of the whole vector,
    1e-4 x an energy scale of that vector: sum sqrt(rho E) for momentum,
    sum sqrt(E) for the field), so a component that is zero up to rounding
    (v_z, B_z of a 2D problem, the momentum of a box at rest) is not divided by
    its own rounding noise."""
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz"]
    rc = np.asarray(ref_cell, dtype=np.float64)
    mnorm = float(np.abs(rc[1:4]).sum())
    bnorm = float(sum(np.abs(np.asarray(f, dtype=np.float64)).sum() for f in ref_face))
    e_pos = np.maximum(rc[4], 0.0)
    m_scale = float(np.sqrt(np.maximum(rc[0], 0.0) * e_pos).sum())
    b_scale = float(np.sqrt(e_pos).sum())
    errs = {}
    for v in range(5):
        floor = max(1e-3 * mnorm, 1e-4 * m_scale) if 1 <= v <= 3 else 0.0
        errs[names[v]] = rel_l1(cell[v], ref_cell[v], floor)
    for d in range(3):
        errs[names[5 + d]] = rel_l1(face[d], ref_face[d], max(1e-3 * bnorm, 1e-4 * b_scale))
    return errs


def subbox(cell, face, n, center, h, dx, gamma):
    """Outflow sub-box of (2h+1)^3 cells around center = (i, j, k), cut from a
    periodic state of n = (nx, ny, nz) cells (indices wrap).  Returns (Config,
    cell, face) for the oracle."""
    i, j, k = center
    nx, ny, nz = n
    xi = np.arange(i - h, i + h + 1) % nx
    yj = np.arange(j - h, j + h + 1) % ny
    zk = np.arange(k - h, k + h + 1) % nz
    xf = np.arange(i - h, i + h + 2) % nx
    yf = np.arange(j - h, j + h + 2) % ny
    zf = np.arange(k - h, k + h + 2) % nz
    c = np.ascontiguousarray(cell[:, zk][:, :, yj][:, :, :, xi])
    bx = np.ascontiguousarray(face[0][zk][:, yj][:, :, xf])
    by = np.ascontiguousarray(face[1][zk][:, yf][:, :, xi])
    bz = np.ascontiguousarray(face[2][zf][:, yj][:, :, xi])
    m = 2 * h + 1
    cfg = O.Config(m, m, m, dx[0], dx[1], dx[2], gamma, 0.4, (O.OUTFLOW,) * 3)
    return cfg, c, [bx, by, bz]
