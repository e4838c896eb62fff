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
