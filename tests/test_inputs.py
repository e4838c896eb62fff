"""The seeded synthetic input recipes have the statistics their documentation
states (density, pressure, sound speed, Mach number, plasma beta, spectrum,
solenoidal fields), and a seed fixes each of them."""
import math

import numpy as np
import pytest

from paper_2606_12753_gb300 import inputs as I


def _prims(box):
    n = (box.nx, box.ny, box.nz)
    rho = box.cell[0]
    v = box.cell[1:4] / rho
    b = I.cell_b(box.face, n, box.bc)
    p = (box.gamma - 1.0) * (box.cell[4] - 0.5 * rho * (v ** 2).sum(0) - 0.5 * sum(x * x for x in b))
    return rho, v, p, b


def _div_b(box):
    """Discrete divergence of the face field (the CT one), per cell."""
    n = (box.nx, box.ny, box.nz)
    Bx, By, Bz = box.face
    hi = [Bx[:, :, 1:n[0] + 1] if box.bc[0] == I.OUTFLOW else np.roll(Bx, -1, axis=2),
          By[:, 1:n[1] + 1, :] if box.bc[1] == I.OUTFLOW else np.roll(By, -1, axis=1),
          Bz[1:n[2] + 1, :, :] if box.bc[2] == I.OUTFLOW else np.roll(Bz, -1, axis=0)]
    lo = [Bx[:, :, :n[0]], By[:, :n[1], :], Bz[:n[2], :, :]]
    return sum((hi[d] - lo[d]) / (box.dx, box.dy, box.dz)[d] for d in range(3))


def test_turbulence_start():
    box = I.turbulence_3d(32, seed=7)
    rho, v, p, b = _prims(box)
    assert np.all(rho == 1.0)
    np.testing.assert_allclose(p, 0.6, rtol=1e-12)
    assert math.sqrt(box.gamma * 0.6 / 1.0) == pytest.approx(1.0)          # sound speed 1
    assert math.sqrt(float(np.mean((v ** 2).sum(0)))) == pytest.approx(1.0, rel=1e-12)   # rms Mach 1
    beta = 2.0 * p / sum(x * x for x in b)
    np.testing.assert_allclose(beta, 1.0, rtol=1e-12)
    assert np.abs(_div_b(box)).max() < 1e-12
    # solenoidal, band-limited velocity: k . v_hat = 0 and no power outside 1 <= |k| <= 8
    k1 = np.fft.fftfreq(32, d=1.0 / 32)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    vh = [np.fft.fftn(v[d]) for d in range(3)]
    div = KX * vh[0] + KY * vh[1] + KZ * vh[2]
    assert np.abs(div).max() < 1e-10 * max(np.abs(x).max() for x in vh)
    kmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    outside = (kmag < 1) | (kmag > 8)
    assert max(np.abs(x[outside]).max() for x in vh) < 1e-10 * max(np.abs(x).max() for x in vh)


def test_turbulence_seed_fixes_the_state():
    a, b, c = I.turbulence_3d(16, seed=5), I.turbulence_3d(16, seed=5), I.turbulence_3d(16, seed=6)
    np.testing.assert_array_equal(a.cell, b.cell)
    assert not np.array_equal(a.cell, c.cell)


def test_orszag_tang_3d_start():
    n = 24
    box = I.orszag_tang_3d(n, seed=3)
    rho, v, p, b = _prims(box)
    np.testing.assert_allclose(rho, box.gamma ** 2, rtol=1e-14)
    np.testing.assert_allclose(p, box.gamma, rtol=1e-10)
    assert np.abs(_div_b(box)).max() < 1e-10
    assert np.all(v[2] == 0.0)
    # each velocity component is the 2D vortex times (1 + 0.01 xi)
    y = (np.arange(n) + 0.5) / n
    base = -np.sin(2 * np.pi * y)[None, :, None] * np.ones((n, n, n))
    ok = np.abs(base) > 0.3
    ratio = v[0][ok] / base[ok] - 1.0
    assert abs(float(ratio.std()) - 0.01) < 0.002 and abs(float(ratio.mean())) < 0.002


def test_blast_batch_recipe():
    boxes = I.blast_batch(64, seed=64, size_scale=0.25)   # the 64-box recipe at a quarter of its size
    assert len(boxes) == 64
    for bx in boxes:
        assert bx.bc == (I.OUTFLOW,) * 3
        assert all(max(4, round(32 * 0.25)) - 1 <= d <= round(128 * 0.25) + 1 for d in (bx.nx, bx.ny, bx.nz))
        rho, v, p, b = _prims(bx)
        assert np.all(rho == 1.0) and np.all(v == 0.0)
        bmag2 = sum(x * x for x in b)
        np.testing.assert_allclose(bmag2, 100.0, rtol=1e-12)                # |B| = 10
        ratio = bx.meta["ratio"]
        assert 10.0 <= ratio <= 100.0
        # p_out = 0.1 outside the sphere (beta = 2 p / B^2 = 0.002), ratio x p_out inside
        assert np.all(np.isclose(p, 0.1, rtol=1e-12) | np.isclose(p, 0.1 * ratio, rtol=1e-12))
        assert np.abs(_div_b(bx)).max() < 1e-9
    sizes = np.log([d for bx in boxes for d in (bx.nx, bx.ny, bx.nz)])
    assert abs(float(sizes.mean()) - math.log(64 * 0.25)) < 0.15              # log-uniform in [32, 128] x 0.25


def test_riemann_2d_quadrants():
    n = 40
    box = I.riemann_2d(n, seed=8)
    rho, v, p, b = _prims(box)
    assert np.abs(_div_b(box)).max() < 1e-12
    half = n // 2
    for ys in (slice(0, half), slice(half, n)):
        for xs in (slice(0, half), slice(half, n)):
            for f in (rho, p, v[0], v[1], v[2], b[2]):
                q = f[0, ys, xs]
                assert np.all(q == q.flat[0])                               # one state per quadrant
    assert np.all(box.face[0][0, :half] == box.face[0][0, 0, 0])             # B_x by the y-half only
    assert np.all(box.face[1][0, :, :half] == box.face[1][0, 0, 0])          # B_y by the x-half only
