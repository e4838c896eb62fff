"""Pins of the FP64 face-switch reference (oracle/mlp.py): gradients against
central finite differences, closed forms of the loss and of the first Adam
step, bfloat16 rounding on known values, scale invariance of the features and
the labels of faces whose HLL/HLLD answer is known exactly."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M

G = 5.0 / 3.0


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    params = M.init_params(4)
    for k in params:
        params[k] = params[k] + 0.1 * rng.standard_normal(params[k].shape)   # nonzero biases too
    X = rng.standard_normal((40, M.NF))
    y = (rng.uniform(size=40) < 0.4).astype(np.float64)
    z, cache = M.forward(params, X)
    g = M.backward(cache, z, y)
    vec = M.flatten(params)
    gvec = M.flatten(g)
    h = 1e-6
    idx = rng.choice(vec.size, 60, replace=False)
    for i in idx:
        vp, vm = vec.copy(), vec.copy()
        vp[i] += h
        vm[i] -= h
        lp = M.bce_loss(M.forward(M.unflatten(vp), X)[0], y)
        lm = M.bce_loss(M.forward(M.unflatten(vm), X)[0], y)
        fd = (lp - lm) / (2 * h)
        assert gvec[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), (i, gvec[i], fd)


def test_bce_closed_forms():
    assert M.bce_loss(np.zeros(5), np.ones(5)) == pytest.approx(math.log(2.0), rel=1e-15)
    assert M.bce_loss(np.array([40.0]), np.array([1.0])) < 1e-16
    assert M.bce_loss(np.array([-3.0]), np.array([0.0])) == pytest.approx(math.log1p(math.exp(-3.0)), rel=1e-14)


def test_first_adam_step_is_signed_learning_rate():
    params = {"W1": np.array([1.0, -2.0, 3.0])}
    grads = {"W1": np.array([0.5, -4.0, 1e-3])}
    out = M.adam_step(params, grads, {}, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(out["W1"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], rtol=0, atol=1e-10)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 3.0e38, 1.0 + 2.0 ** -7])
    exp = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, -2.5, 1.765625 * 2.0 ** 127, 1.0 + 2.0 ** -7])
    np.testing.assert_allclose(M.bf16(vals), exp, rtol=1e-7)


def _state(rng):
    return np.array([rng.uniform(0.3, 2), rng.normal(), rng.normal(), rng.normal(), rng.uniform(0.2, 2),
                     rng.normal(), rng.normal()])


def test_features_are_dimensionless():
    # rho -> a rho, p -> a p, B -> sqrt(a) B, v unchanged: a change of units
    rng = np.random.default_rng(5)
    for _ in range(20):
        wl, wr, bn = _state(rng), _state(rng), rng.normal()
        a = rng.uniform(0.1, 10)
        s = np.array([a, 1, 1, 1, a, math.sqrt(a), math.sqrt(a)])
        np.testing.assert_allclose(M.features(wl * s, wr * s, bn * math.sqrt(a), G), M.features(wl, wr, bn, G),
                                   rtol=1e-12, atol=1e-12)


def test_labels_of_known_faces():
    rng = np.random.default_rng(6)
    w = _state(rng)
    assert M.label(w, w, 0.7, G) == 0.0            # HLL = HLLD = F(U)
    # stationary Alfven discontinuity: HLLD exact, HLL smears it
    rho, p, bn = 1.3, 0.7, 0.9
    ca = bn / math.sqrt(rho)
    WL = np.array([rho, -ca, 0.2, -0.1, p, 0.8, 0.0])
    WR = np.array([rho, -ca, 0.2 - (0.8 * math.cos(1.1) - 0.8) / math.sqrt(rho),
                   -0.1 - 0.8 * math.sin(1.1) / math.sqrt(rho), p, 0.8 * math.cos(1.1), 0.8 * math.sin(1.1)])
    assert M.label(WL, WR, bn, G) == 1.0
    # both states supersonic to the right: every solver returns F_L
    WL = np.array([1.0, 9.0, 0.1, 0.2, 0.5, 0.3, 0.1])
    WR = np.array([0.8, 9.5, -0.1, 0.0, 0.6, 0.2, 0.4])
    assert M.label(WL, WR, 0.4, G) == 0.0


# ------------------------------------------------ the oracle's switch modes

def _cfg_box(n=10, seed=21):
    from paper_2606_12753_gb300 import inputs as I
    box = I.random_state((n, n - 1, n - 2), seed=seed, bc=(0, 0, 0), noise=0.3)
    cfg = O.Config(box.nx, box.ny, box.nz, box.dx, box.dy, box.dz, gamma=box.gamma)
    return cfg, box


def _net(seed, zero=False, b3=0.0):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 7)
    p["b1"] = 0.2 * rng.standard_normal(32)
    p["b2"] = 0.2 * rng.standard_normal(32)
    if zero:
        for k in p:
            p[k] = np.zeros_like(p[k])
    p["b3"] = np.array([b3])
    return M.flatten(p)


def test_c_features_and_logit_match_the_numpy_definitions():
    rng = np.random.default_rng(31)
    vec = _net(3)
    params = M.unflatten(vec)
    for _ in range(30):
        wl, wr, bn = _state(rng), _state(rng), rng.normal()
        f = O.switch_features(wl, wr, bn, G)
        np.testing.assert_allclose(f, M.features(wl, wr, bn, G), rtol=1e-14, atol=1e-15)
        z, _ = M.forward(params, f[None, :], bf16_inputs=True)
        assert O.switch_logit(vec, f) == pytest.approx(z[0], rel=1e-12, abs=1e-12)
    for v in (1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 3.0e38):
        assert O.bf16(v) == M.bf16(np.array([v]))[0]


def test_learned_mode_reduces_to_each_solver():
    # a network with zero weights outputs b3 everywhere: b3 below the
    # threshold is HLL on every face, above it HLLD on every face
    cfg, box = _cfg_box()
    ref = {}
    for mode in (O.HLL, O.HLLD):
        cfg.riemann = mode
        ref[mode] = O.rhs(cfg, box.cell, box.face)
    for b3, mode in ((-3.0, O.HLL), (3.0, O.HLLD)):
        cfg.riemann, cfg.mlp, cfg.mlp_zt = O.LEARNED, _net(0, zero=True, b3=b3), 0.0
        st = O.Stats()
        du, db = O.rhs(cfg, box.cell, box.face, st)
        assert np.array_equal(du, ref[mode][0])
        for d in range(3):
            assert np.array_equal(db[d], ref[mode][1][d])
        nf = 3 * box.nx * box.ny * box.nz
        assert (st.faces_hll, st.faces_hlld) == ((nf, 0) if mode == O.HLL else (0, nf))


def test_mask_mode_reproduces_the_learned_choices():
    cfg, box = _cfg_box(9, 22)
    vec = _net(5)
    cfg.riemann, cfg.mlp = O.LEARNED, vec
    z = O.switch_logits(cfg, box.cell, box.face)
    cfg.mlp_zt = float(np.median(z))        # about half the faces each way
    st = O.Stats()
    du, db = O.rhs(cfg, box.cell, box.face, st)
    choice = (z >= cfg.mlp_zt).astype(np.uint8)
    assert st.faces_hlld == int(choice.sum()) and st.faces_hll == choice.size - int(choice.sum())
    mcfg = O.Config(cfg.nx, cfg.ny, cfg.nz, cfg.dx, cfg.dy, cfg.dz, gamma=cfg.gamma, riemann=O.MASK,
                    choice=choice.reshape(-1))
    du2, db2 = O.rhs(mcfg, box.cell, box.face)
    assert np.array_equal(du, du2)
    for d in range(3):
        assert np.array_equal(db[d], db2[d])
    # and the mix differs from both pure solvers
    for mode in (O.HLL, O.HLLD):
        mcfg.riemann = mode
        assert not np.array_equal(O.rhs(mcfg, box.cell, box.face)[0], du)


def test_switch_logits_are_the_network_on_the_reconstructed_faces():
    # the logit of one face recomputed by hand from the oracle primitives
    cfg, box = _cfg_box(8, 23)
    vec = _net(6)
    cfg.riemann, cfg.mlp = O.LEARNED, vec
    z = O.switch_logits(cfg, box.cell, box.face)
    n = (box.nx, box.ny, box.nz)
    rho = box.cell[0]
    v = box.cell[1:4] / rho
    from paper_2606_12753_gb300 import inputs as I
    bc = I.cell_b(box.face, n, box.bc)
    p = (box.gamma - 1) * (box.cell[4] - 0.5 * rho * (v ** 2).sum(0) - 0.5 * sum(b * b for b in bc))
    prims = np.stack([rho, v[0], v[1], v[2], p, bc[0], bc[1], bc[2]])
    rng = np.random.default_rng(24)
    for _ in range(40):
        d = int(rng.integers(3))
        i, j, k = (int(rng.integers(m)) for m in n)
        t1, t2 = (d + 1) % 3, (d + 2) % 3
        cells = []
        for o in (-2, -1, 0, 1):
            c = [i, j, k]
            c[d] = (c[d] + o) % n[d]
            q = prims[:, c[2], c[1], c[0]]
            cells.append(np.array([q[0], q[1 + d], q[1 + t1], q[1 + t2], q[4], q[5 + t1], q[5 + t2]]))
        wl = np.array([cells[1][u] + 0.5 * O.mc_slope(cells[0][u], cells[1][u], cells[2][u]) for u in range(7)])
        wr = np.array([cells[2][u] - 0.5 * O.mc_slope(cells[1][u], cells[2][u], cells[3][u]) for u in range(7)])
        bn = box.face[d][k, j, i]
        zz, _ = M.forward(M.unflatten(vec), M.features(wl, wr, bn, box.gamma)[None, :], bf16_inputs=True)
        assert z[d, k, j, i] == pytest.approx(zz[0], rel=1e-10, abs=1e-10)
