"""Shared helpers of the test suite (error metrics, oracle configs)."""
import numpy as np

import oracle as O


def thresholds(precision):
    """The oracle's branch thresholds for a GPU form: the FP32-bulk forms
    (mixed, fp32) take the HLLD-degeneracy, mass-flux-deadband and
    characteristic-degeneracy decisions at 1e-6, the FP64 form at 1e-12,
    1e-10, 1e-12."""
    return O.THRESH_FP32 if precision in ("mixed", "fp32") else O.THRESH_FP64


def ocfg(b, precision=None, **kw):
    """Oracle config of a box; `precision` (the GPU form it is compared with)
    selects the branch thresholds."""
    kw.setdefault("thresholds", thresholds(precision))
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


def subbox(cell, face, n, center, h, dx, gamma, precision=None):
    """Outflow sub-box of (2h+1)^3 cells around center = (i, j, k), cut from a
    periodic state of n = (nx, ny, nz) cells (indices wrap).  Returns (Config,
    cell, face) for the oracle, with the branch thresholds of `precision`."""
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
    cfg = O.Config(m, m, m, dx[0], dx[1], dx[2], gamma, 0.4, (O.OUTFLOW,) * 3, thresholds=thresholds(precision))
    return cfg, c, [bx, by, bz]


def max_elementwise_rel(cell, face, ref_cell, ref_face, floor_frac=1e-6):
    """Largest per-element relative error over all 8 variables:
    |q - ref| / max(|ref|, floor_frac x scale), where the scale of rho and E
    is their own largest magnitude and the scale of a momentum or field
    component is the largest magnitude of any component of that vector (a
    component that is zero up to rounding, such as B_z of a 1D tube, is not
    divided by its own rounding noise).  Returns (worst value, variable name,
    flat index)."""
    names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz"]
    arrs = [(np.asarray(cell[v], np.float64), np.asarray(ref_cell[v], np.float64)) for v in range(5)]
    arrs += [(np.asarray(face[d], np.float64), np.asarray(ref_face[d], np.float64)) for d in range(3)]
    top_of = lambda a: float(np.abs(a).max()) if a.size else 0.0
    m_top = max(top_of(arrs[v][1]) for v in (1, 2, 3))
    b_top = max(top_of(arrs[v][1]) for v in (5, 6, 7))
    worst = (0.0, "", -1)
    for v, (name, (q, r)) in enumerate(zip(names, arrs)):
        top = m_top if v in (1, 2, 3) else (b_top if v >= 5 else top_of(r))
        den = np.maximum(np.abs(r), floor_frac * top) if top > 0 else np.ones_like(r)
        e = np.abs(q - r) / den
        i = int(np.argmax(e)) if e.size else -1
        if e.size and float(e.flat[i]) > worst[0]:
            worst = (float(e.flat[i]), name, i)
    return worst


def perturbed(cell, face, rel=6e-8, seed=0):
    """The state with every value multiplied by (1 + rel xi), xi = +-1 seeded:
    FP32 rounding-sized noise (half an FP32 ulp is 6e-8 relative)."""
    rng = np.random.default_rng(seed)
    c = np.asarray(cell, np.float64) * (1.0 + rel * rng.choice([-1.0, 1.0], size=np.shape(cell)))
    f = [np.asarray(x, np.float64) * (1.0 + rel * rng.choice([-1.0, 1.0], size=np.shape(x))) for x in face]
    return np.ascontiguousarray(c), [np.ascontiguousarray(x) for x in f]


# Relative input noise of a form's rounding (4 ulp in FP64; half an FP32 ulp
# for the FP32-bulk forms) and the relative error with which a form computes
# the quantities its branch thresholds decide on (the mass flux against the
# upwind deadband: ~1e-7 of rho c against 1e-6 in the FP32-bulk forms).
NOISE = {"fp64": 4 * 2.0 ** -53, "mixed": 6e-8, "fp32": 6e-8}
THRESH_SPREAD = {"fp64": 1e-5, "mixed": 0.1, "fp32": 0.1}


def control(cfg, cell, face, dts, rc, rf, precision):
    """How far the oracle's own result (rc, rf after the steps dts) moves
    under the rounding of the form's precision: input noise (two seeds) and
    branch thresholds scaled by 1 -/+ the decided quantities' relative error.
    Returns the per-variable relative L1 and the per-element figure, each the
    largest over the four runs."""
    runs = [(perturbed(cell, face, rel=NOISE[precision], seed=seed), 1.0) for seed in (1, 2)]
    runs += [((cell, face), 1.0 + s * THRESH_SPREAD[precision]) for s in (-1.0, 1.0)]
    move, elem = {}, 0.0
    for (c0, f0), scale in runs:
        cfg.thresh_scale = scale
        pc, pf = O.step_dts(cfg, c0, f0, dts)
        e = state_errors(pc, pf, rc, rf)
        move = {k: max(move.get(k, 0.0), v) for k, v in e.items()}
        elem = max(elem, max_elementwise_rel(pc, pf, rc, rf)[0])
    cfg.thresh_scale = 1.0
    return move, elem
