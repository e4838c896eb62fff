"""Learned face switch on the GPU: the BF16 tensor-core forward/backward and
the Adam step against the FP64 reference in oracle/mlp.py (same bf16-rounded
weights, inputs and activations), the face sampler against the oracle's
reconstruction and solvers, and a short training run."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2606_12753_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _params(seed=1):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    p["b1"] = 0.1 * rng.standard_normal(32)
    p["b2"] = 0.1 * rng.standard_normal(32)
    p["b3"] = 0.1 * rng.standard_normal(1)
    return p


def _block(torch, params):
    from paper_2606_12753_gb300 import mhd
    blk = torch.zeros(mhd.mlp_param_bytes(), dtype=torch.uint8, device="cuda")
    mhd.mlp_init(blk.data_ptr(), M.flatten(params).astype(np.float32))
    return blk


def _x(n, seed=2):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, 16)) * np.array([1, 1, .5, .5, .5, .5, .5, .5, 1, 1, .7, .7, .7, .7, .7, .3])
            + np.array([1, 1, 0, 0, 0, 0, 0, 0, 1, 1, 0, 0, 0, 0, 0, .6])).astype(np.float32)


def test_forward_matches_reference():
    import torch
    from paper_2606_12753_gb300 import mhd
    params = _params()
    n = 3001
    X = _x(n)
    blk = _block(torch, params)
    xd = torch.from_numpy(X).cuda()
    zd = torch.empty(n, dtype=torch.float32, device="cuda")
    mhd.mlp_forward(blk.data_ptr(), xd.data_ptr(), n, zd.data_ptr())
    torch.cuda.synchronize()
    z = zd.cpu().numpy().astype(np.float64)
    params32 = M.unflatten(M.flatten(params).astype(np.float32).astype(np.float64))
    zr, _ = M.forward(params32, X.astype(np.float64), bf16_inputs=True)
    d = np.abs(z - zr)
    # FP32 accumulation vs FP64: a hidden activation can round to the other
    # neighbouring bf16 value; almost all rows agree to FP32 rounding
    assert np.quantile(d, 0.99) <= 1e-4 * (1 + np.abs(zr).max())
    assert d.max() <= 2e-2 * (1 + np.abs(zr).max())


def test_backward_matches_reference():
    import torch
    from paper_2606_12753_gb300 import mhd
    params = _params(3)
    n = 2048
    X = _x(n, 4)
    rng = np.random.default_rng(5)
    y = (rng.uniform(size=n) < 0.35).astype(np.float32)
    blk = _block(torch, params)
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    gd = torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda")
    mhd.mlp_backward(blk.data_ptr(), xd.data_ptr(), yd.data_ptr(), n, gd.data_ptr())
    torch.cuda.synchronize()
    g = gd.cpu().numpy().astype(np.float64)
    params32 = M.unflatten(M.flatten(params).astype(np.float32).astype(np.float64))
    zr, cache = M.forward(params32, X.astype(np.float64), bf16_inputs=True)
    gr = M.flatten(M.backward(cache, zr, y.astype(np.float64), bf16_deltas=True))
    assert np.linalg.norm(g - gr) <= 2e-3 * np.linalg.norm(gr), np.linalg.norm(g - gr) / np.linalg.norm(gr)
    for name, shape in M.ORDER:          # every parameter group, not just the norm
        a = M.unflatten(g)[name]
        b = M.unflatten(gr)[name]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-9, name


def test_adam_matches_reference():
    import torch
    from paper_2606_12753_gb300 import mhd
    params = _params(6)
    rng = np.random.default_rng(7)
    grad = rng.standard_normal(M.NPARAM).astype(np.float32) * 1e-2
    blk = _block(torch, params)
    md = torch.zeros(M.NPARAM, device="cuda")
    vd = torch.zeros(M.NPARAM, device="cuda")
    gd = torch.from_numpy(grad).cuda()
    state = {}
    ref = M.unflatten(M.flatten(params).astype(np.float32).astype(np.float64))
    for step in (1, 2, 3):
        mhd.mlp_adam(blk.data_ptr(), md.data_ptr(), vd.data_ptr(), gd.data_ptr(), step, lr=1e-3)
        ref = M.adam_step(ref, M.unflatten(grad.astype(np.float64)), state, lr=1e-3)
    torch.cuda.synchronize()
    got = blk[: M.NPARAM * 4].view(torch.float32).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, M.flatten(ref), rtol=1e-5, atol=1e-7)


def _oracle_face(prims, n, d, s, gamma, bfloor=1e-10):
    """Reconstructed states of the face below cell s along d (periodic)."""
    k, j, i = np.unravel_index(s, (n[2], n[1], n[0]))
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    cells = []
    for o in (-2, -1, 0, 1):
        c = [i, j, k]
        c[d] = (c[d] + o) % n[d]
        q = prims[:, c[2], c[1], c[0]]
        cells.append(np.array([q[0], q[1 + d], q[1 + t1], q[1 + t2], q[4], q[5 + t1], q[5 + t2]]))
    wl = np.array([cells[1][v] + 0.5 * O.mc_slope(cells[0][v], cells[1][v], cells[2][v]) for v in range(7)])
    wr = np.array([cells[2][v] - 0.5 * O.mc_slope(cells[1][v], cells[2][v], cells[3][v]) for v in range(7)])
    for w in (wl, wr):
        w[0] = max(w[0], bfloor)
        w[4] = max(w[4], bfloor)
    return wl, wr


def test_face_sampler_matches_oracle():
    import torch
    from paper_2606_12753_gb300 import mhd
    box = I.turbulence_3d(24, seed=11)
    s = mhd.Solver(box, precision="fp64")
    s.set_state(box.cell, box.face)
    s.step(-1.0, 2)
    cell, face = s.get_state()
    n = (box.nx, box.ny, box.nz)
    ncell = box.ncell
    rng = np.random.default_rng(12)
    ids = rng.integers(0, 3 * ncell, 300).astype(np.int64)
    idd = torch.from_numpy(ids).cuda()
    Xd = torch.empty((300, 16), device="cuda")
    yd = torch.empty(300, device="cuda")
    sd = torch.empty(300, device="cuda")
    mhd.mhd_dump_faces(s.h, idd.data_ptr(), 300, Xd.data_ptr(), yd.data_ptr(), sd.data_ptr())
    X, y, score = Xd.cpu().numpy(), yd.cpu().numpy(), sd.cpu().numpy()
    s.close()
    # oracle primitives of the same state (cell-centred field from the faces)
    rho = cell[0]
    v = cell[1:4] / rho
    bc = I.cell_b(face, n, box.bc)
    p = (box.gamma - 1) * (cell[4] - 0.5 * rho * (v ** 2).sum(0) - 0.5 * sum(b * b for b in bc))
    prims = np.stack([rho, v[0], v[1], v[2], p, bc[0], bc[1], bc[2]])
    agree = 0
    for q, fid in enumerate(ids):
        d, sidx = divmod(int(fid), ncell)
        wl, wr = _oracle_face(prims, n, d, sidx, box.gamma)
        bn = face[d].reshape(-1)[sidx]
        np.testing.assert_allclose(X[q], M.features(wl, wr, bn, box.gamma), rtol=2e-6, atol=2e-7)
        lab = M.label(wl, wr, bn, box.gamma)
        if abs(score[q] - 1e-3) > 1e-6:
            assert y[q] == lab, (q, score[q], lab)
            agree += 1
    assert agree >= 290
    assert 0.02 < y.mean() < 0.98     # both classes present


def test_training_lowers_the_loss():
    import torch
    from paper_2606_12753_gb300 import mhd
    box = I.turbulence_3d(32, seed=13)
    s = mhd.Solver(box, precision="fp64")
    s.set_state(box.cell, box.face)
    s.step(-1.0, 3)
    nfaces = 3 * box.ncell
    ids = torch.arange(nfaces, dtype=torch.int64, device="cuda")
    X = torch.empty((nfaces, 16), device="cuda")
    y = torch.empty(nfaces, device="cuda")
    mhd.mhd_dump_faces(s.h, ids.data_ptr(), nfaces, X.data_ptr(), y.data_ptr())
    s.close()
    blk = _block(torch, M.init_params(14))
    m = torch.zeros(M.NPARAM, device="cuda")
    v = torch.zeros(M.NPARAM, device="cuda")
    g = torch.zeros(M.NPARAM, device="cuda")
    z = torch.empty(nfaces, device="cuda")

    def loss():
        mhd.mlp_forward(blk.data_ptr(), X.data_ptr(), nfaces, z.data_ptr())
        return float(torch.nn.functional.binary_cross_entropy_with_logits(z, y))

    l0 = loss()
    gen = torch.Generator(device="cuda").manual_seed(15)
    bs = 4096
    for step in range(1, 301):
        idx = torch.randint(0, nfaces, (bs,), device="cuda", generator=gen)
        xb, yb = X[idx].contiguous(), y[idx].contiguous()
        g.zero_()
        mhd.mlp_backward(blk.data_ptr(), xb.data_ptr(), yb.data_ptr(), bs, g.data_ptr())
        mhd.mlp_adam(blk.data_ptr(), m.data_ptr(), v.data_ptr(), g.data_ptr(), step, lr=3e-3)
    l1 = loss()
    assert np.isfinite(l1) and l1 < 0.7 * l0, (l0, l1)


@pytest.mark.parametrize("n", [1, 5, 127, 128, 129, 300])
def test_forward_and_backward_on_partial_tiles(n):
    """The tensor-core kernels take 128 rows per tile; row counts below,
    at and just past a tile (rows past n are zero in the products and add
    nothing to the gradient) match the reference."""
    import torch
    from paper_2606_12753_gb300 import mhd
    params = _params(11)
    X = _x(n, 12)
    rng = np.random.default_rng(13)
    y = (rng.uniform(size=n) < 0.4).astype(np.float32)
    blk = _block(torch, params)
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    zd = torch.empty(n, dtype=torch.float32, device="cuda")
    gd = torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda")
    mhd.mlp_forward(blk.data_ptr(), xd.data_ptr(), n, zd.data_ptr())
    mhd.mlp_backward(blk.data_ptr(), xd.data_ptr(), yd.data_ptr(), n, gd.data_ptr())
    torch.cuda.synchronize()
    params32 = M.unflatten(M.flatten(params).astype(np.float32).astype(np.float64))
    zr, cache = M.forward(params32, X.astype(np.float64), bf16_inputs=True)
    z = zd.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(z))
    assert np.abs(z - zr).max() <= 2e-2 * (1 + np.abs(zr).max())
    gr = M.flatten(M.backward(cache, zr, y.astype(np.float64), bf16_deltas=True))
    g = gd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - gr) <= 5e-3 * np.linalg.norm(gr), np.linalg.norm(g - gr) / np.linalg.norm(gr)
