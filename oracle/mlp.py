"""FP64 reference of the learned HLL/HLLD face switch -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU leg use this module;
the CUDA library never does.  It defines, in plain numpy:

* the 16 face features, from the reconstructed states w_L, w_R (rho, v_n,
  v_t1, v_t2, p, B_t1, B_t2), the normal field B_n and the fast speeds, with
  rho_bar = (rho_L + rho_R)/2, p_bar likewise, c = max(c_fL, c_fR),
  b = sqrt(rho_bar) c:
      rho_L/rho_bar, rho_R/rho_bar, v_L/c (3), v_R/c (3), p_L/p_bar,
      p_R/p_bar, B_n/b, B_tL/b (2), B_tR/b (2), min(c_fL, c_fR)/c;
* the label: 1 when the HLLD and HLL fluxes differ by more than 1e-3 in some
  component, each component scaled by (rho c, rho c^2 x 3, rho c^3, b c, b c)
  (rho = rho_bar) -- i.e. when the cheap HLL flux is not good enough;
* the network 16 -> 32 -> 32 -> 1 with ReLU hidden layers and a sigmoid
  output, its binary cross-entropy loss, the gradients by backpropagation and
  one Adam step.
Optional bfloat16 rounding (round to nearest even) reproduces the inputs the
tensor-core kernels see: weights, features and hidden activations rounded to
bf16, products accumulated in higher precision.
"""
from __future__ import annotations

import numpy as np

from . import fast_speed, hll, hlld

NF, NH = 16, 32
LABEL_THRESHOLD = 1e-3


def bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    a = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(wl, wr, bn, gamma):
    wl = np.asarray(wl, dtype=np.float64)
    wr = np.asarray(wr, dtype=np.float64)
    cl = fast_speed(wl, bn, gamma)
    cr = fast_speed(wr, bn, gamma)
    rho = 0.5 * (wl[0] + wr[0])
    pbar = 0.5 * (wl[4] + wr[4])
    c = max(cl, cr)
    b = np.sqrt(rho) * c
    f = np.empty(NF)
    f[0], f[1] = wl[0] / rho, wr[0] / rho
    f[2:5] = wl[1:4] / c
    f[5:8] = wr[1:4] / c
    f[8], f[9] = wl[4] / pbar, wr[4] / pbar
    f[10] = bn / b
    f[11:13] = wl[5:7] / b
    f[13:15] = wr[5:7] / b
    f[15] = min(cl, cr) / c
    return f


def label(wl, wr, bn, gamma, threshold=LABEL_THRESHOLD):
    cl = fast_speed(wl, bn, gamma)
    cr = fast_speed(wr, bn, gamma)
    rho = 0.5 * (wl[0] + wr[0])
    c = max(cl, cr)
    b = np.sqrt(rho) * c
    scale = np.array([rho * c, rho * c * c, rho * c * c, rho * c * c, rho * c ** 3, b * c, b * c])
    d = np.abs(hlld(wl, wr, bn, gamma) - hll(wl, wr, bn, gamma)) / scale
    return 1.0 if d.max() > threshold else 0.0


# ----------------------------------------------------------------- network

def init_params(seed: int):
    """He-normal weights, zero biases; W1 (32,16), W2 (32,32), W3 (1,32)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((NH, NF)) * np.sqrt(2.0 / NF), "b1": np.zeros(NH),
        "W2": rng.standard_normal((NH, NH)) * np.sqrt(2.0 / NH), "b2": np.zeros(NH),
        "W3": rng.standard_normal((1, NH)) * np.sqrt(2.0 / NH), "b3": np.zeros(1),
    }


def forward(params, X, bf16_inputs=False):
    """Logits z (N,) and the cached activations.  With bf16_inputs, X, the
    weights and the hidden activations fed to the next layer are rounded to
    bfloat16 (the biases and all sums stay in FP64)."""
    r = bf16 if bf16_inputs else (lambda a: np.asarray(a, dtype=np.float64))
    X = r(X)
    W1, W2, W3 = r(params["W1"]), r(params["W2"]), r(params["W3"])
    a1 = X @ W1.T + params["b1"]
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + params["b2"]
    h2 = r(np.maximum(a2, 0.0))
    z = (h2 @ W3.T)[:, 0] + params["b3"][0]
    return z, {"X": X, "a1": a1, "h1": h1, "a2": a2, "h2": h2, "W1": W1, "W2": W2, "W3": W3}


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def bce_loss(z, y):
    """Mean binary cross-entropy of logits z against labels y."""
    z = np.asarray(z, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def backward(cache, z, y, bf16_deltas=False):
    """Gradients of the mean BCE loss with respect to every parameter.  With
    bf16_deltas the layer deltas are rounded to bfloat16 where they enter a
    matrix product (as tensor-core operands); bias sums use them unrounded."""
    r = bf16 if bf16_deltas else (lambda a: a)
    n = z.shape[0]
    dz = (sigmoid(z) - y) / n                       # (N,)
    g = {}
    g["W3"] = (dz @ cache["h2"])[None, :]
    g["b3"] = np.array([dz.sum()])
    dh2 = dz[:, None] * cache["W3"]                  # (N, 32)
    da2 = dh2 * (cache["a2"] > 0.0)
    g["W2"] = r(da2).T @ cache["h1"]
    g["b2"] = da2.sum(axis=0)
    dh1 = r(da2) @ cache["W2"]
    da1 = dh1 * (cache["a1"] > 0.0)
    g["W1"] = r(da1).T @ cache["X"]
    g["b1"] = da1.sum(axis=0)
    return g


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in place; state holds m, v and t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params


# flat parameter order shared with the C ABI: W1, b1, W2, b2, W3, b3
ORDER = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (1, NH)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in ORDER)


def flatten(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).reshape(-1) for k, _ in ORDER])


def unflatten(vec):
    out, o = {}, 0
    for k, s in ORDER:
        n = int(np.prod(s))
        out[k] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out
