"""Multi-dimensional verification problems for the oracle's pins.

* Oblique linear waves (after Gardiner & Stone 2008, JCP 227:4123, Sec. 8.1):
  the 1D eigenmodes of the Gardiner-Stone background (rho = 1, p = 1/gamma,
  B = (1, sqrt 2, 1/2) in the wave frame, so the fast, Alfven and slow speeds
  are 2, 1 and 1/2) propagated along an oblique wave vector of a periodic box.
  The eigenvectors come from numpy's eigen-decomposition of the primitive
  Jacobian of 1D ideal MHD, written here from the equations of motion.
* Field-loop advection (Gardiner & Stone 2005, JCP 205:509, Sec. 5.1): a weak
  cylindrical current-free loop of field carried obliquely across a periodic
  box by a uniform flow.

Every face field is the discrete curl of an edge vector potential plus a
uniform part, so div B = 0 to rounding.  Nothing here is the method's
arithmetic; the states only feed the oracle.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2606_12753_gb300 import inputs as I

G = 5.0 / 3.0


def primitive_jacobian(rho, u, v, w, p, bx, by, bz, g):
    """A in dW/dt + A dW/dx = 0 for W = (rho, u, v, w, p, By, Bz), Bx constant."""
    A = np.zeros((7, 7))
    A[0, 0], A[0, 1] = u, rho
    A[1, 1], A[1, 4], A[1, 5], A[1, 6] = u, 1 / rho, by / rho, bz / rho
    A[2, 2], A[2, 5] = u, -bx / rho
    A[3, 3], A[3, 6] = u, -bx / rho
    A[4, 1], A[4, 4] = g * p, u
    A[5, 1], A[5, 2], A[5, 5] = by, -bx, u
    A[6, 1], A[6, 3], A[6, 6] = bz, -bx, u
    return A


def gs_eigenmode(wave):
    """(speed, right eigenvector scaled to max |r| = 1) of the Gardiner-Stone
    background for wave in ('fast', 'alfven', 'slow')."""
    A = primitive_jacobian(1.0, 0, 0, 0, 1.0 / G, 1.0, math.sqrt(2.0), 0.5, G)
    lam, R = np.linalg.eig(A)
    lam, R = lam.real, R.real
    target = {"fast": 2.0, "alfven": 1.0, "slow": 0.5}[wave]
    m = int(np.argmin(np.abs(lam - target)))
    assert abs(lam[m] - target) < 1e-10
    return lam[m], R[:, m] / np.abs(R[:, m]).max()


def wave_frame(kdir):
    """Orthonormal right-handed (n, e1, e2) with n along kdir."""
    n = np.asarray(kdir, dtype=np.float64)
    n = n / np.linalg.norm(n)
    e1 = np.cross(n, [0.0, 0.0, 1.0])
    if np.linalg.norm(e1) < 1e-12:
        e1 = np.cross(n, [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return n, e1, e2


def oblique_wave_box(dims, wave, amp=1e-6, sign=1.0):
    """Periodic box of dims = (nx, ny, nz) square cells of size h = 1/(the
    smallest cell count above 1), with a plane eigenmode of one period along each axis that has
    more than one cell: k = 2 pi (1/Lx, 1/Ly, 1/Lz).  The profile is
    sign * amp * cos(k.x).  Returns (Box, wave speed, |k|)."""
    nx, ny, nz = dims
    h = 1.0 / min(d for d in dims if d > 1)
    L = [nx * h, ny * h, nz * h]
    k = np.array([2 * np.pi / L[d] if dims[d] > 1 else 0.0 for d in range(3)])
    n, e1, e2 = wave_frame(k)
    speed, r = gs_eigenmode(wave)
    a = sign * amp
    B0 = 1.0 * n + math.sqrt(2.0) * e1 + 0.5 * e2
    kn = float(np.linalg.norm(k))
    # B = B0 + a (r5 e1 + r6 e2) cos(k.x): the perturbation is the curl of
    # a (r6 e1 - r5 e2) sin(k.x)/|k|
    avec = a * (r[6] * e1 - r[5] * e2) / kn

    def A(d, x, y, z):
        ph = k[0] * x * h + k[1] * y * h + k[2] * z * h
        return avec[d] * np.sin(ph)

    bc = (I.PERIODIC,) * 3
    fp = I.faces_from_potential(dims, bc, (h, h, h), A)
    face = [np.ascontiguousarray(fp[d] + B0[d]) for d in range(3)]
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    prof = np.cos(k[0] * x * h + k[1] * y * h + k[2] * z * h)
    rho = 1.0 + a * r[0] * prof
    p = 1.0 / G + a * r[4] * prof
    dv = r[1] * n + r[2] * e1 + r[3] * e2
    v = tuple(a * dv[d] * prof for d in range(3))
    cell = I.conserved(rho, v, p, face, dims, bc, G)
    return I.Box(nx, ny, nz, h, h, h, bc, G, cell, face, name=f"oblique_{wave}"), speed, kn


def field_loop_box(n, vz=0.0, amp=1e-3, radius=0.3, direction=1.0):
    """Field loop of Gardiner & Stone (2005, Sec. 5.1) on [-1, 1] x [-1/2, 1/2]
    with 2n x n cells: rho = 1, p = 1, v = direction (2, 1) + (0, 0, vz),
    A_z = amp (R - r) for r < R (0 outside), so |B| = amp inside the loop.
    The flow carries the loop once across the box in x and twice in y by
    t = 1; direction = -1 reverses it, so every mass flux changes sign."""
    dims = (2 * n, n, 1)
    h = 1.0 / n
    bc = (I.PERIODIC,) * 3

    def A(d, x, y, zz):
        if d != 2:
            return np.zeros_like(x)
        X = x * h - 1.0
        Y = y * h - 0.5
        r = np.sqrt(X * X + Y * Y)
        return np.where(r < radius, amp * (radius - r), 0.0)

    face = I.faces_from_potential(dims, bc, (h, h, h), A)
    shape = (1, n, 2 * n)
    cell = I.conserved(np.ones(shape), (np.full(shape, 2.0 * direction), np.full(shape, 1.0 * direction),
                                        np.full(shape, vz)),
                       np.ones(shape), face, dims, bc, G)
    return I.Box(2 * n, n, 1, h, h, h, bc, G, cell, face, name=f"field_loop_{n}")


def magnetic_energy(box_or_face, dims, h):
    """Sum over cells of |B_c|^2/2 times the cell volume."""
    face = box_or_face
    bx, by, bz = I.cell_b(face, dims, (I.PERIODIC,) * 3)
    return 0.5 * float((bx * bx + by * by + bz * bz).sum()) * h ** 3
