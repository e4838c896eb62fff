"""The learned HLL/HLLD face switch inside the fused stage kernel, against
the oracle: a network that clears every face (or none) gives exactly the HLL
(HLLD) step; the kernel's per-face choices agree with the oracle network's
away from the threshold; and the operator L(U) with those choices matches the
oracle's operator run with the same choices element by element."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2606_12753_gb300 import inputs as I
from helpers import ocfg, state_errors

pytestmark = pytest.mark.gpu

RHS_TOL = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 1e-5}


def _params(seed, zero=False, b3=0.0):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 7)
    p["b1"] = 0.2 * rng.standard_normal(32)
    p["b2"] = 0.2 * rng.standard_normal(32)
    if zero:
        for k in p:
            p[k] = np.zeros_like(p[k])
    p["b3"] = np.array([b3])
    return M.flatten(p).astype(np.float32)     # the device keeps FP32 masters


def _block(torch, vec32):
    from paper_2606_12753_gb300 import mhd
    blk = torch.zeros(mhd.mlp_param_bytes(), dtype=torch.uint8, device="cuda")
    mhd.mlp_init(blk.data_ptr(), vec32)
    return blk


def _run(box, precision, riemann, nsteps, blk=None, tau=0.5, dt=None):
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, riemann=riemann)
    if blk is not None:
        s.set_switch(blk.data_ptr(), tau)
    s.set_state(box.cell, box.face)
    h = dt if dt is not None else -1.0
    s.step(h, nsteps)
    out = s.get_state()
    st = s.stats()
    s.close()
    return out, st


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_learned_switch_reduces_to_each_solver(precision):
    import torch
    box = I.turbulence_3d(24, seed=41)
    dt = O.cfl_dt(ocfg(box), box.cell, box.face)
    ncell = box.ncell
    for b3, pure in ((-4.0, "hll"), (4.0, "hlld")):
        blk = _block(torch, _params(0, zero=True, b3=b3))
        (c, f), st = _run(box, precision, "learned", 2, blk, dt=dt)
        (c0, f0), _ = _run(box, precision, pure, 2, dt=dt)
        # the same solver on every face; two kernels compiled separately may
        # contract a multiply-add differently, so the states agree to rounding
        errs = state_errors(c, f, c0, f0)
        assert max(errs.values()) <= (1e-13 if precision == "fp64" else 1e-6), (precision, pure, errs)
        # every face evaluation (halo faces recomputed by neighbouring tiles
        # included) took the chosen solver
        hll, hlld = st["faces_hll"], st["faces_hlld"]
        assert (hll == 0) if pure == "hlld" else (hlld == 0)
        assert hll + hlld >= 2 * 2 * 3 * ncell


def _choices(torch, box, precision, blk, tau):
    from paper_2606_12753_gb300 import mhd
    s = mhd.Solver(box, precision=precision, riemann="learned")
    s.set_switch(blk.data_ptr(), tau)
    s.set_state(box.cell, box.face)
    n = 3 * box.ncell
    ch = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    zl = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    s.switch_choices(ch.data_ptr(), zl.data_ptr())
    gc, gf = s.rhs()
    c, f = s.get_state()
    s.close()
    np.testing.assert_array_equal(c, box.cell.astype(c.dtype))      # state untouched
    return ch.cpu().numpy(), zl.cpu().numpy().astype(np.float64), (gc, gf)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_switch_choices_and_operator_match_the_oracle(precision):
    import torch
    box = I.random_state((29, 21, 13), seed=61, bc=(0, 0, 0), noise=0.0)
    vec = _params(5)
    blk = _block(torch, vec)
    cfg = ocfg(box, riemann=O.LEARNED, mlp=vec.astype(np.float64))
    zo = O.switch_logits(cfg, box.cell, box.face).reshape(-1)
    zt = float(np.median(zo))
    tau = 1.0 / (1.0 + np.exp(-zt))
    ch, zg, (gc, gf) = _choices(torch, box, precision, blk, tau)
    assert set(np.unique(ch)) <= {0, 1}, "every face reported"
    assert np.isfinite(zg).all()
    zt32 = float(np.float32(np.log(tau / (1 - tau))))
    # logits: FP32 accumulation against FP64, features in the kernel's precision
    d = np.abs(zg - zo)
    scale = 1.0 + np.abs(zo).max()
    assert np.quantile(d, 0.99) <= (1e-4 if precision == "fp64" else 3e-3) * scale, np.quantile(d, 0.99)
    assert d.max() <= 5e-2 * scale, d.max()
    # choices: the kernel's are exactly its own logits against the threshold,
    # and the oracle's wherever the oracle logit is clear of it
    assert np.array_equal(ch, (zg >= zt32).astype(np.uint8))
    # where the oracle logit is farther from the threshold than the largest
    # logit difference, both sides must take the same side
    clear = np.abs(zo - zt32) > d.max()
    assert np.array_equal(ch[clear], (zo[clear] >= zt32).astype(np.uint8))
    assert clear.mean() > 0.9, (clear.mean(), d.max())
    assert 0.3 < ch.mean() < 0.7
    # L(U) with the kernel's choices against the oracle operator with the same choices
    mcfg = ocfg(box, precision, riemann=O.MASK, choice=ch)
    st = O.Stats()
    du, db = O.rhs(mcfg, box.cell, box.face, st)
    assert st.faces_hlld == int(ch.sum())
    errs = state_errors(gc, gf, du, db)
    assert max(errs.values()) <= RHS_TOL[precision], errs


def test_learned_step_needs_a_network():
    from paper_2606_12753_gb300 import mhd
    box = I.uniform_state((16, 8, 4))
    s = mhd.Solver(box, precision="mixed", riemann="learned")
    s.set_state(box.cell, box.face)
    with pytest.raises(mhd.MHDError):
        s.step(1e-3, 1)
    s.close()
