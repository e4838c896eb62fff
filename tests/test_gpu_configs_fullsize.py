"""Parity at the full sizes of the benchmark configurations not covered by
test_gpu_fullsize.py (turbulence 256^3, Orszag-Tang 352^3) and
test_gpu_riemann2d.py (3200^2), in the launch configuration the benchmark
times (default tiles):

* Orszag-Tang 2D, 128^2, FP64, the full 100 RK2 steps against the oracle on
  the oracle's own CFL dt sequence (the whole state; relative L1 1e-12);
* Orszag-Tang 3D, 512^3, mixed, one step: sampled cells against the oracle on
  periodic sub-boxes of radius 7 around them (one RK2 step is local to 4
  cells, test_oracle_locality.py), relative L1 over the samples 1e-5;
* the 64-box outflow blast batch (32-128 cells per axis, FP32, one
  persistent launch), one step with one explicit dt: sampled cells of several
  boxes against the oracle on sub-boxes clamped to each box (a side that
  meets the box edge is the box's own outflow boundary, the others lie 5
  cells from the sample), relative L1 per variable within max(1e-5, 3 x the
  movement of the oracle's own result when its input carries FP32-rounding-
  sized noise, 6e-8 relative): these low-beta boxes recover their pressure
  ill-conditioned, and the control measures by how much."""
import numpy as np
import pytest

import oracle as O
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, perturbed, state_errors, subbox

pytestmark = pytest.mark.gpu


def _sampled_errors(got_c, ref_c, got_f, ref_f):
    """Relative L1 per variable over samples, with the suite's state metric
    (helpers.state_errors): a vector component is measured against max(its
    own L1, 1e-3 x the vector's L1, 1e-4 x an energy scale: sum sqrt(rho E)
    for momentum, sum sqrt(E) for the field), so a component that is zero up
    to rounding (the momentum of gas at rest) is not divided by its noise."""
    got_c, ref_c, got_f, ref_f = (np.asarray(x, dtype=np.float64) for x in (got_c, ref_c, got_f, ref_f))
    e_pos = np.maximum(ref_c[:, 4], 0.0)
    m_floor = max(1e-3 * float(np.abs(ref_c[:, 1:4]).sum()),
                  1e-4 * float(np.sqrt(np.maximum(ref_c[:, 0], 0.0) * e_pos).sum()))
    b_floor = max(1e-3 * float(np.abs(ref_f).sum()), 1e-4 * float(np.sqrt(e_pos).sum()))
    names = ["rho", "mx", "my", "mz", "E"]
    errs = {}
    for v in range(5):
        den = max(float(np.abs(ref_c[:, v]).sum()), m_floor if 1 <= v <= 3 else 0.0, 1e-300)
        errs[names[v]] = float(np.abs(got_c[:, v] - ref_c[:, v]).sum()) / den
    for d in range(3):
        den = max(float(np.abs(ref_f[:, d]).sum()), b_floor, 1e-300)
        errs["B" + "xyz"[d]] = float(np.abs(got_f[:, d] - ref_f[:, d]).sum()) / den
    return errs


def test_orszag_tang_2d_128_full_run_fp64():
    from paper_2606_12753_gb300 import mhd
    box = I.orszag_tang_2d(128)
    cfg = ocfg(box)
    rc, rf, dts = O.step(cfg, box.cell, box.face, -1.0, nsteps=100)
    assert len(dts) == 100 and all(d > 0 for d in dts)
    s = mhd.Solver(box, precision="fp64")
    assert (s.cfg.tile_x, s.cfg.tile_y, s.cfg.tile_z) == (0, 0, 0)
    s.set_state(box.cell, box.face)
    for h in dts:
        s.step(float(h), 1)
    c, f = s.get_state()
    s.close()
    errs = state_errors(c, f, rc, rf)
    assert max(errs.values()) <= 1e-12, errs


def test_orszag_tang_3d_512_step_sampled_mixed():
    from paper_2606_12753_gb300 import mhd
    n = 512
    box = I.orszag_tang_3d(n)
    s = mhd.Solver(box, precision="mixed")
    s.set_state(box.cell, box.face)
    dt = s.cfl_dt()
    s.step(dt, 1)
    c, f = s.get_state()
    s.close()
    rng = np.random.default_rng(512)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (15, 7, 31), (16, 8, 32), (255, 256, 127), (n - 1, 0, 255)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(10)]
    h = 7
    got_c, ref_c, got_f, ref_f = [], [], [], []
    for (i, j, k) in pts:
        cfg, cell, face = subbox(box.cell, box.face, (n, n, n), (i, j, k), h, (box.dx, box.dy, box.dz), box.gamma,
                                 "mixed")
        r_c, r_f = O.step_dts(cfg, cell, face, [dt])
        ref_c.append(r_c[:, h, h, h])
        got_c.append(c[:, k, j, i])
        ref_f.append([r_f[0][h, h, h], r_f[1][h, h, h], r_f[2][h, h, h]])
        got_f.append([f[0][k, j, i], f[1][k, j, i], f[2][k, j, i]])
    errs = _sampled_errors(got_c, ref_c, got_f, ref_f)
    assert max(errs.values()) <= 1e-5, errs


def _clamped_subbox(box, centre, h):
    """Sub-box of an outflow box around centre = (i, j, k), clamped to the
    box; returns (Config, cell, face, centre inside the sub-box)."""
    n = (box.nx, box.ny, box.nz)
    lo = [max(0, centre[d] - h) for d in range(3)]
    hi = [min(n[d], centre[d] + h + 1) for d in range(3)]
    sx, sy, sz = (slice(lo[d], hi[d]) for d in range(3))
    cell = np.ascontiguousarray(box.cell[:, sz, sy, sx])
    bx = np.ascontiguousarray(box.face[0][sz, sy, lo[0]:hi[0] + 1])
    by = np.ascontiguousarray(box.face[1][sz, lo[1]:hi[1] + 1, sx])
    bz = np.ascontiguousarray(box.face[2][lo[2]:hi[2] + 1, sy, sx])
    cfg = O.Config(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], box.dx, box.dy, box.dz, box.gamma, 0.4,
                   (O.OUTFLOW,) * 3, thresholds=O.THRESH_FP32)
    return cfg, cell, [bx, by, bz], tuple(centre[d] - lo[d] for d in range(3))


def _kappa(box):
    """max over cells of E / (p / (gamma - 1)): how far a relative rounding
    error of the stored total energy is amplified in the pressure."""
    rho = box.cell[0]
    v2 = (box.cell[1:4] ** 2).sum(0) / rho ** 2
    bc = I.cell_b(box.face, (box.nx, box.ny, box.nz), box.bc)
    eth = box.cell[4] - 0.5 * rho * v2 - 0.5 * sum(b * b for b in bc)
    return float((box.cell[4] / eth).max())


def test_blast_batch64_step_sampled_fp32():
    from paper_2606_12753_gb300 import mhd
    boxes = I.blast_batch(64, seed=64)
    b = mhd.Batch(boxes, precision="fp32")
    for i, bx in enumerate(boxes):
        b.set_state(i, bx.cell, bx.face)
    dt = min(b.box_dt(i) for i in range(len(boxes)))
    b.step(dt, 1)
    assert b.stats()["status"] == 0
    sizes = [bx.ncell for bx in boxes]
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 0, 17, 33, 63})
    rng = np.random.default_rng(64)
    h = 5
    for bi in pick:
        bx = boxes[bi]
        c, f = b.get_state(bi)
        n = (bx.nx, bx.ny, bx.nz)
        pts = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (n[0] // 2, n[1] // 2, n[2] // 2), (15, 7, min(31, n[2] - 1))]
        pts += [tuple(int(rng.integers(0, n[d])) for d in range(3)) for _ in range(4)]
        got_c, ref_c, got_f, ref_f, mov_c, mov_f = [], [], [], [], [], []
        for (i, j, k) in pts:
            i, j, k = min(i, n[0] - 1), min(j, n[1] - 1), min(k, n[2] - 1)
            cfg, cell, face, (ci, cj, ck) = _clamped_subbox(bx, (i, j, k), h)
            r_c, r_f = O.step_dts(cfg, cell, face, [dt])
            p_c, p_f = O.step_dts(cfg, *perturbed(cell, face, seed=bi * 100 + i), [dt])
            mov_c.append(p_c[:, ck, cj, ci])
            mov_f.append([p_f[0][ck, cj, ci], p_f[1][ck, cj, ci], p_f[2][ck, cj, ci]])
            ref_c.append(r_c[:, ck, cj, ci])
            got_c.append(c[:, k, j, i])
            ref_f.append([r_f[0][ck, cj, ci], r_f[1][ck, cj, ci], r_f[2][ck, cj, ci]])
            got_f.append([f[0][k, j, i], f[1][k, j, i], f[2][k, j, i]])
        errs = _sampled_errors(got_c, ref_c, got_f, ref_f)
        # control: how far FP32-rounding-sized input noise moves the oracle
        move = _sampled_errors(mov_c, ref_c, mov_f, ref_f)
        over = {k: (errs[k], move[k]) for k in errs if not errs[k] <= max(1e-5, 3.0 * move[k])}
        print(bx.name, "kappa", round(_kappa(bx)), "error", max(errs.values()), "oracle movement", max(move.values()))
        assert not over, (bi, bx.name, over)
    b.close()
