"""Seeded synthetic initial states for the MHD workloads.

This module only draws and lays out initial data.  It holds none of the
method's arithmetic (no reconstruction, Riemann solver, transport or time
integration) and imports neither the CUDA library nor the oracle, so the GPU
path and the CPU oracle can both be fed from it.

State convention: ``cell`` is float64 of shape (5, nz, ny, nx) holding
(rho, mx, my, mz, E); ``face`` is [Bx, By, Bz] with Bx of shape (nz, ny, nx+o),
By (nz, ny+o, nx), Bz (nz+o, ny, nx), o = 1 on an outflow axis else 0.  Face
index i along its normal sits at i-1/2.  Every face field is built as the
discrete curl of an edge-centred vector potential, so the discrete div B of
every generated state is zero up to rounding.

The recipes follow the workloads the method is measured on: the 2D and 3D
Orszag-Tang vortex (the paper's Sec. 3 test problem), 3D decaying turbulence,
batches of blast waves with outflow boundaries, plus the small verification
problems (linear waves, the Brio-Wu shock tube, smooth random states).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, OUTFLOW = 0, 1
GAMMA = 5.0 / 3.0


@dataclass
class Box:
    """One box: grid, boundary kinds, gamma and its initial state."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    bc: tuple
    gamma: float
    cell: np.ndarray
    face: list
    name: str = ""
    cfl: float = 0.4
    meta: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz


def _edge_coords(n, d, bc):
    """Coordinates (x, y, z) in cell units of the edge lattice of the vector
    potential component A_d, covering every face of the box: along d the edge
    sits at a cell centre, across it at a cell corner."""
    nx, ny, nz = n
    o = [1 if b == OUTFLOW else 0 for b in bc]
    cnt = []
    for e in range(3):
        if e == d:
            cnt.append(n[e])
        else:
            cnt.append(n[e] + 1)      # one corner more than faces on this axis
    ax = []
    for e in range(3):
        if e == d:
            ax.append(np.arange(cnt[e]) + 0.5)
        else:
            ax.append(np.arange(cnt[e]) + 0.0)
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x, y, z


def faces_from_potential(n, bc, delta, A):
    """Face B = curl A on the staggered grid.  ``A(d, x, y, z)`` evaluates the
    edge component d at cell-unit coordinates.  Returns [Bx, By, Bz]."""
    nx, ny, nz = n
    dx, dy, dz = delta
    Ae = []
    for d in range(3):
        x, y, z = _edge_coords(n, d, bc)
        Ae.append(A(d, x, y, z))
    o = [1 if b == OUTFLOW else 0 for b in bc]
    # A_x: shape (nz+1, ny+1, nx), A_y: (nz+1, ny, nx+1), A_z: (nz, ny+1, nx+1)
    Ax, Ay, Az = Ae
    nxf, nyf, nzf = nx + o[0], ny + o[1], nz + o[2]
    Bx = (Az[:, 1:ny + 1, :nxf] - Az[:, 0:ny, :nxf]) / dy - (Ay[1:nz + 1, :, :nxf] - Ay[0:nz, :, :nxf]) / dz
    By = (Ax[1:nz + 1, :nyf, :] - Ax[0:nz, :nyf, :]) / dz - (Az[:, :nyf, 1:nx + 1] - Az[:, :nyf, 0:nx]) / dx
    Bz = (Ay[:nzf, :, 1:nx + 1] - Ay[:nzf, :, 0:nx]) / dx - (Ax[:nzf, 1:ny + 1, :] - Ax[:nzf, 0:ny, :]) / dy
    return [np.ascontiguousarray(Bx), np.ascontiguousarray(By), np.ascontiguousarray(Bz)]


def cell_b(face, n, bc):
    """Cell-centred field as the mean of each cell's two faces (periodic axes
    wrap the upper face)."""
    nx, ny, nz = n
    Bx, By, Bz = face
    bx_hi = Bx[:, :, 1:nx + 1] if bc[0] == OUTFLOW else np.roll(Bx, -1, axis=2)
    by_hi = By[:, 1:ny + 1, :] if bc[1] == OUTFLOW else np.roll(By, -1, axis=1)
    bz_hi = Bz[1:nz + 1, :, :] if bc[2] == OUTFLOW else np.roll(Bz, -1, axis=0)
    return (0.5 * (Bx[:, :, :nx] + bx_hi), 0.5 * (By[:, :ny, :] + by_hi), 0.5 * (Bz[:nz, :, :] + bz_hi))


def conserved(rho, v, p, face, n, bc, gamma):
    """Cell array (rho, m, E) from primitive rho, v, p and the face field."""
    bcx, bcy, bcz = cell_b(face, n, bc)
    vx, vy, vz = v
    e = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bcx * bcx + bcy * bcy + bcz * bcz)
    cell = np.stack([rho, rho * vx, rho * vy, rho * vz, e]).astype(np.float64)
    return np.ascontiguousarray(cell)


def _centres(n):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    return x, y, z


# --------------------------------------------------------------------------
# Orszag-Tang vortex
# --------------------------------------------------------------------------

def orszag_tang_2d(n: int = 128, gamma: float = GAMMA) -> Box:
    """2D Orszag-Tang vortex on [0,1]^2, n x n x 1, periodic: rho = gamma^2,
    p = gamma, v = (-sin 2 pi y, sin 2 pi x), B = (-sin 2 pi y, sin 4 pi x)/sqrt(4 pi),
    the field taken as the curl of A_z = (cos 2 pi y/(2 pi) + cos 4 pi x/(4 pi))/sqrt(4 pi)."""
    dims = (n, n, 1)
    h = 1.0 / n
    bc = (PERIODIC, PERIODIC, PERIODIC)
    s4 = math.sqrt(4.0 * math.pi)

    def A(d, x, y, z):
        if d != 2:
            return np.zeros_like(x)
        X, Y = x * h, y * h
        return (np.cos(2 * np.pi * Y) / (2 * np.pi) + np.cos(4 * np.pi * X) / (4 * np.pi)) / s4

    face = faces_from_potential(dims, bc, (h, h, h), A)
    x, y, z = _centres(dims)
    X, Y = x * h, y * h
    rho = np.full(X.shape, gamma * gamma)
    p = np.full(X.shape, gamma)
    v = (-np.sin(2 * np.pi * Y), np.sin(2 * np.pi * X), np.zeros_like(X))
    cell = conserved(rho, v, p, face, dims, bc, gamma)
    return Box(n, n, 1, h, h, h, bc, gamma, cell, face, name=f"orszag_tang_2d_{n}")


def orszag_tang_3d(n: int = 512, seed: int = 12753, noise: float = 0.01, gamma: float = GAMMA) -> Box:
    """3D extension of Orszag-Tang: the 2D fields replicated along z on an
    n^3 periodic box, each velocity component multiplied by (1 + noise * xi),
    xi seeded standard-normal white noise."""
    dims = (n, n, n)
    h = 1.0 / n
    bc = (PERIODIC, PERIODIC, PERIODIC)
    s4 = math.sqrt(4.0 * math.pi)

    def A(d, x, y, z):
        if d != 2:
            return np.zeros_like(x)
        X, Y = x * h, y * h
        return (np.cos(2 * np.pi * Y) / (2 * np.pi) + np.cos(4 * np.pi * X) / (4 * np.pi)) / s4

    face = faces_from_potential(dims, bc, (h, h, h), A)
    x, y, z = _centres(dims)
    X, Y = x * h, y * h
    rng = np.random.default_rng(seed)
    rho = np.full(X.shape, gamma * gamma)
    p = np.full(X.shape, gamma)
    vx = -np.sin(2 * np.pi * Y) * (1.0 + noise * rng.standard_normal(X.shape))
    vy = np.sin(2 * np.pi * X) * (1.0 + noise * rng.standard_normal(X.shape))
    vz = np.zeros_like(X)
    cell = conserved(rho, (vx, vy, vz), p, face, dims, bc, gamma)
    return Box(n, n, n, h, h, h, bc, gamma, cell, face, name=f"orszag_tang_3d_{n}", meta={"seed": seed})


# --------------------------------------------------------------------------
# decaying turbulence
# --------------------------------------------------------------------------

def turbulence_3d(n: int = 256, seed: int = 2606, kmin: int = 1, kmax: int = 8,
                  rho0: float = 1.0, p0: float = 0.6, mach: float = 1.0, beta: float = 1.0,
                  gamma: float = GAMMA) -> Box:
    """3D decaying-turbulence start on [0,1]^3, periodic: rho = 1, p = 0.6
    (sound speed 1), a random-phase solenoidal velocity with integer
    wavenumbers kmin <= |k| <= kmax (units of 2 pi) and amplitude |k|^(-11/6)
    per mode (shell spectrum E(k) ~ k^(-5/3)), rescaled to rms |v| = mach, and
    a uniform B0 = sqrt(2 p / beta) along z."""
    dims = (n, n, n)
    h = 1.0 / n
    bc = (PERIODIC, PERIODIC, PERIODIC)
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    Kmag = np.sqrt(K2)
    amp = np.where((Kmag >= kmin) & (Kmag <= kmax), np.power(np.maximum(Kmag, 1e-30), -11.0 / 6.0), 0.0)
    vel = []
    xi = [rng.standard_normal(K2.shape) + 1j * rng.standard_normal(K2.shape) for _ in range(3)]
    kdotxi = (KX * xi[0] + KY * xi[1] + KZ * xi[2]) / np.where(K2 > 0, K2, 1.0)
    for d, Kd in enumerate((KX, KY, KZ)):
        spec = amp * (xi[d] - Kd * kdotxi)
        vel.append(np.real(np.fft.ifftn(spec)))
    del xi, kdotxi
    rms = math.sqrt(float(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)))
    vel = [np.ascontiguousarray(v * (mach / rms)) for v in vel]
    b0 = math.sqrt(2.0 * p0 / beta)
    face = [np.zeros((n, n, n)), np.zeros((n, n, n)), np.full((n, n, n), b0)]
    rho = np.full(dims[::-1], rho0)
    p = np.full(dims[::-1], p0)
    cell = conserved(rho, vel, p, face, dims, bc, gamma)
    return Box(n, n, n, h, h, h, bc, gamma, cell, face, name=f"turbulence_3d_{n}", meta={"seed": seed})


# --------------------------------------------------------------------------
# blast batch
# --------------------------------------------------------------------------

def blast_box(dims, seed_rng: np.random.Generator, h: float = 1.0 / 128, radius: float = 0.1,
              p_out: float = 0.1, b_mag: float = 10.0, gamma: float = GAMMA) -> Box:
    """One blast box with outflow boundaries: rho = 1, B = b_mag (1,1,0)/sqrt 2,
    p = p_out outside and ratio * p_out inside a sphere of ``radius`` whose
    centre is uniform in [0.3, 0.7] of each box length, ratio log-uniform in
    [10, 100]."""
    nx, ny, nz = dims
    bc = (OUTFLOW, OUTFLOW, OUTFLOW)
    L = (nx * h, ny * h, nz * h)
    centre = [seed_rng.uniform(0.3, 0.7) * L[d] for d in range(3)]
    ratio = math.exp(seed_rng.uniform(math.log(10.0), math.log(100.0)))
    b = b_mag / math.sqrt(2.0)

    def A(d, x, y, z):
        # uniform B = (b, b, 0) = curl A with A_z = b (y - x) in physical units
        if d != 2:
            return np.zeros_like(x)
        return b * (y * h - x * h)

    face = faces_from_potential(dims, bc, (h, h, h), A)
    x, y, z = _centres(dims)
    r2 = (x * h - centre[0]) ** 2 + (y * h - centre[1]) ** 2 + (z * h - centre[2]) ** 2
    p = np.where(r2 < radius * radius, ratio * p_out, p_out)
    rho = np.ones(p.shape)
    zero = np.zeros(p.shape)
    cell = conserved(rho, (zero, zero, zero), p, face, dims, bc, gamma)
    return Box(nx, ny, nz, h, h, h, bc, gamma, cell, face, name=f"blast_{nx}x{ny}x{nz}",
               meta={"centre": centre, "ratio": ratio})


def riemann_2d(n: int = 3200, seed: int = 3200, gamma: float = GAMMA) -> Box:
    """Seeded four-quadrant 2D MHD Riemann problem on [0,1]^2 (n x n x 1,
    outflow in x and y, periodic along the single z cell), quadrants split at
    x = 1/2 and y = 1/2.  Each quadrant has its own rho in [0.5, 2], p in
    [0.3, 1.5], v in [-0.5, 0.5]^2 x [-0.2, 0.2] and B_z in [-0.5, 0.5]; B_x
    takes one of two values by the y-half and B_y one of two by the x-half
    (|B| in [0.2, 0.8]), so the face field is divergence-free.  A stand-in of
    the paper's 2D Riemann workload, whose quadrant states it does not print."""
    rng = np.random.default_rng(seed)
    dims = (n, n, 1)
    h = 1.0 / n
    bc = (OUTFLOW, OUTFLOW, PERIODIC)
    q = {key: (rng.uniform(0.5, 2.0), rng.uniform(0.3, 1.5), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5),
               rng.uniform(-0.2, 0.2), rng.uniform(-0.5, 0.5)) for key in ("ll", "lr", "ul", "ur")}
    sgn = lambda: 1.0 if rng.uniform() < 0.5 else -1.0  # noqa: E731
    bx_half = (sgn() * rng.uniform(0.2, 0.8), sgn() * rng.uniform(0.2, 0.8))   # y < 1/2, y > 1/2
    by_half = (sgn() * rng.uniform(0.2, 0.8), sgn() * rng.uniform(0.2, 0.8))   # x < 1/2, x > 1/2
    xc = (np.arange(n) + 0.5) * h
    upper = xc > 0.5                       # by the cell centre
    X, Y = np.meshgrid(upper, upper, indexing="xy")   # X: x > 1/2, Y: y > 1/2, shape (ny, nx)
    key = np.where(Y, np.where(X, "ur", "ul"), np.where(X, "lr", "ll"))
    fields = np.zeros((6, n, n))
    for name, vals in q.items():
        m = key == name
        for v in range(6):
            fields[v][m] = vals[v]
    rho, p, vx, vy, vz, bz = [f[None] for f in fields]
    bx = np.where(upper, bx_half[1], bx_half[0])[None, :, None] * np.ones((1, n, n + 1))
    by = np.where(upper, by_half[1], by_half[0])[None, None, :] * np.ones((1, n + 1, n))
    face = [np.ascontiguousarray(bx), np.ascontiguousarray(by), np.ascontiguousarray(bz.copy())]
    cell = conserved(rho, (vx, vy, vz), p, face, dims, bc, gamma)
    return Box(n, n, 1, h, h, h, bc, gamma, cell, face, name=f"riemann2d_{n}",
               meta={"quadrants": {k: [float(x) for x in v] for k, v in q.items()}, "bx": bx_half, "by": by_half})


def blast_batch(nbox: int = 64, seed: int = 64, nmin: int = 32, nmax: int = 128,
                size_scale: float = 1.0) -> list:
    """``nbox`` independent blast boxes; each axis length is log-uniform in
    [nmin, nmax] cells (times ``size_scale``, for small test batches)."""
    rng = np.random.default_rng(seed)
    boxes = []
    for _ in range(nbox):
        dims = []
        for _d in range(3):
            nd = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
            dims.append(max(4, int(round(nd * size_scale))))
        boxes.append(blast_box(tuple(dims), rng))
    return boxes


# --------------------------------------------------------------------------
# verification problems
# --------------------------------------------------------------------------

def uniform_state(dims, bc=(PERIODIC,) * 3, rho=1.3, v=(0.3, -0.2, 0.1), p=0.7, B=(0.4, -0.5, 0.6),
                  gamma: float = GAMMA, h: float = None) -> Box:
    nx, ny, nz = dims
    h = h or 1.0 / max(dims)
    shapes = [(nz, ny, nx + (bc[0] == OUTFLOW)), (nz, ny + (bc[1] == OUTFLOW), nx), (nz + (bc[2] == OUTFLOW), ny, nx)]
    face = [np.full(shapes[d], float(B[d])) for d in range(3)]
    shape = (nz, ny, nx)
    cell = conserved(np.full(shape, rho), tuple(np.full(shape, vv) for vv in v), np.full(shape, p), face, dims, bc, gamma)
    return Box(nx, ny, nz, h, h, h, tuple(bc), gamma, cell, face, name="uniform")


def random_state(dims, seed: int, bc=(PERIODIC,) * 3, nmodes: int = 6, noise: float = 0.05,
                 vamp: float = 0.8, bamp: float = 0.6, b0=(0.3, -0.2, 0.4), gamma: float = GAMMA,
                 h: float = None) -> Box:
    """Smooth random state (a few random Fourier modes) plus seeded white
    noise, with a divergence-free face field from a random vector potential.
    Exercises every limiter branch and every HLLD region."""
    nx, ny, nz = dims
    h = h or 1.0 / max(dims)
    rng = np.random.default_rng(seed)
    L = np.array([nx, ny, nz], dtype=np.float64)

    def modes():
        k = rng.integers(-3, 4, size=(nmodes, 3)).astype(np.float64)
        for d in range(3):
            if dims[d] == 1:
                k[:, d] = 0.0
        ph = rng.uniform(0, 2 * np.pi, nmodes)
        a = rng.standard_normal(nmodes)
        return k, ph, a

    def field_at(md, x, y, z):
        k, ph, a = md
        out = np.zeros_like(x, dtype=np.float64)
        for m in range(len(a)):
            out += a[m] * np.sin(2 * np.pi * (k[m, 0] * x / L[0] + k[m, 1] * y / L[1] + k[m, 2] * z / L[2]) + ph[m])
        return out / math.sqrt(len(a))

    amods = [modes() for _ in range(3)]

    def A(d, x, y, z):
        # uniform part b0 = curl A0 with A0 = (b0_y z - b0_z y, b0_z x - b0_x z, b0_x y - b0_y x)/2 * h
        X, Y, Z = x * h, y * h, z * h
        lin = [0.5 * (b0[1] * Z - b0[2] * Y), 0.5 * (b0[2] * X - b0[0] * Z), 0.5 * (b0[0] * Y - b0[1] * X)][d]
        # only periodic-compatible part for the random modes
        return lin + bamp * h * max(dims) / (2 * np.pi) * field_at(amods[d], x, y, z)

    face = faces_from_potential(dims, bc, (h, h, h), A)
    if any(b == PERIODIC for b in bc):
        # the linear part of A is not periodic; rebuild the uniform field on
        # periodic axes exactly by removing the wrap jump
        Bl = [np.full(face[d].shape, float(b0[d])) for d in range(3)]
        face_r = faces_from_potential(dims, bc, (h, h, h),
                                      lambda d, x, y, z: bamp * h * max(dims) / (2 * np.pi) * field_at(amods[d], x, y, z))
        face = [np.ascontiguousarray(face_r[d] + Bl[d]) for d in range(3)]
    x, y, z = _centres(dims)
    m_r, m_p = modes(), modes()
    m_v = [modes() for _ in range(3)]
    rho = 1.0 + 0.3 * np.tanh(field_at(m_r, x, y, z)) + noise * rng.uniform(-1, 1, x.shape)
    p = 0.8 + 0.3 * np.tanh(field_at(m_p, x, y, z)) + noise * rng.uniform(-1, 1, x.shape)
    v = tuple(vamp * field_at(m_v[d], x, y, z) + noise * rng.uniform(-1, 1, x.shape) for d in range(3))
    cell = conserved(rho, v, p, face, dims, bc, gamma)
    return Box(nx, ny, nz, h, h, h, tuple(bc), gamma, cell, face, name=f"random_{nx}x{ny}x{nz}_{seed}")


def brio_wu(n: int = 256, axis: int = 0, gamma: float = 2.0) -> Box:
    """Brio-Wu shock tube along ``axis`` on [0,1]: (rho, p, B_t1) = (1, 1, 1)
    left, (0.125, 0.1, -1) right, B_n = 0.75, gamma = 2, outflow ends."""
    dims = [1, 1, 1]
    dims[axis] = n
    nx, ny, nz = dims
    h = 1.0 / n
    bc = [PERIODIC, PERIODIC, PERIODIC]
    bc[axis] = OUTFLOW
    shapes = [(nz, ny, nx + (bc[0] == OUTFLOW)), (nz, ny + (bc[1] == OUTFLOW), nx), (nz + (bc[2] == OUTFLOW), ny, nx)]
    t1 = (axis + 1) % 3
    face = [np.zeros(shapes[d]) for d in range(3)]
    face[axis][...] = 0.75
    pos = (np.arange(n) + 0.5) * h
    left = pos < 0.5
    bt = np.where(left, 1.0, -1.0)
    shape = (nz, ny, nx)
    face[t1][...] = bt.reshape([n if d == axis else 1 for d in (2, 1, 0)])
    rho = np.where(left, 1.0, 0.125).reshape([n if d == axis else 1 for d in (2, 1, 0)]) * np.ones(shape)
    p = np.where(left, 1.0, 0.1).reshape([n if d == axis else 1 for d in (2, 1, 0)]) * np.ones(shape)
    zero = np.zeros(shape)
    cell = conserved(rho, (zero, zero, zero), p, face, tuple(dims), tuple(bc), gamma)
    return Box(nx, ny, nz, h, h, h, tuple(bc), gamma, cell, face, name=f"brio_wu_{n}")


# --------------------------------------------------------------------------
# edge cases of the method (verification states)
# --------------------------------------------------------------------------

def _smooth_fields(dims, rng, count, nmodes=5):
    """`count` smooth periodic random fields on the cell centres, each of unit
    rms order, from a few seeded Fourier modes along the axes with >1 cell."""
    nx, ny, nz = dims
    x, y, z = _centres(dims)
    L = np.array([nx, ny, nz], dtype=np.float64)
    out = []
    for _ in range(count):
        f = np.zeros((nz, ny, nx))
        for _m in range(nmodes):
            k = rng.integers(-3, 4, size=3).astype(np.float64)
            for d in range(3):
                if dims[d] == 1:
                    k[d] = 0.0
            f += rng.standard_normal() * np.sin(2 * np.pi * (k[0] * x / L[0] + k[1] * y / L[1] + k[2] * z / L[2])
                                                 + rng.uniform(0, 2 * np.pi))
        out.append(f / math.sqrt(nmodes))
    return out


def supersonic_state(dims, seed: int, v0=(4.0, -4.0, 4.0), gamma: float = GAMMA) -> Box:
    """Smooth random state (rho ~ 1, p ~ 0.8, |B| ~ 0.5) moving with the
    uniform velocity v0, well above the fast speed (~1.3) along every axis:
    the x and z faces take the left outer state (S_L > 0), the y faces the
    right one (S_R < 0).  Periodic."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    h = 1.0 / max(dims)
    fr, fp, fvx, fvy, fvz = _smooth_fields(dims, rng, 5)
    rho = 1.0 + 0.2 * np.tanh(fr)
    p = 0.8 + 0.2 * np.tanh(fp)
    v = (v0[0] + 0.3 * fvx, v0[1] + 0.3 * fvy, v0[2] + 0.3 * fvz)
    bc = (PERIODIC,) * 3
    b0 = (0.3, -0.2, 0.4)
    face = [np.full((nz, ny, nx), b0[d]) for d in range(3)]
    cell = conserved(rho, v, p, face, dims, bc, gamma)
    return Box(nx, ny, nz, h, h, h, bc, gamma, cell, face, name=f"supersonic_{nx}x{ny}x{nz}_{seed}")


def transverse_field_state(dims, seed: int, gamma: float = GAMMA) -> Box:
    """State whose field is purely along z and varies only in x and y, with
    rho, p and v also independent of z: B_n = 0 on every x and y face (the
    HLLD double-star region collapses there), and B_x = B_y = 0 for all
    time.  Periodic."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    h = 1.0 / max(dims)
    d2 = (nx, ny, 1)
    fr, fp, fvx, fvy, fvz, fb = _smooth_fields(d2, rng, 6)
    rep = lambda a: np.ascontiguousarray(np.repeat(a, nz, axis=0))
    rho = rep(1.0 + 0.3 * np.tanh(fr))
    p = rep(0.7 + 0.3 * np.tanh(fp))
    v = (rep(0.8 * fvx), rep(0.8 * fvy), rep(0.5 * fvz))
    bz = rep(0.8 + 0.4 * np.tanh(fb))
    bc = (PERIODIC,) * 3
    face = [np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)), bz]
    cell = conserved(rho, v, p, face, dims, bc, gamma)
    return Box(nx, ny, nz, h, h, h, bc, gamma, cell, face, name=f"transverse_{nx}x{ny}x{nz}_{seed}")


def alfvenic_shear_state(dims, seed: int, b0: float = 1.0, p0: float = 0.1, gamma: float = GAMMA) -> Box:
    """Uniform rho = 1 and p = p0 at rest along x, field B = (b0, 0, 0) with
    the Alfven speed b0 above the sound speed, and transverse velocities
    v_y(x, z), v_z(x, y): every x face has equal outer states but for its
    tangential velocity, B_t = 0 and a fast speed equal to the Alfven speed,
    the degenerate star state of HLLD (den = 0 up to rounding).  The y and z
    faces have B_n = 0.  Periodic."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    h = 1.0 / max(dims)
    x, y, z = _centres(dims)
    L = np.array([nx, ny, nz], dtype=np.float64)
    f1, f2 = _smooth_fields((nx, 1, nz), rng, 1)[0], _smooth_fields((nx, ny, 1), rng, 1)[0]
    vy = 0.3 * np.broadcast_to(f1, (nz, ny, nx)) if ny > 1 or nz > 1 else 0.3 * f1
    vz = 0.3 * np.broadcast_to(f2, (nz, ny, nx))
    shape = (nz, ny, nx)
    bc = (PERIODIC,) * 3
    face = [np.full(shape, b0), np.zeros(shape), np.zeros(shape)]
    cell = conserved(np.ones(shape), (np.zeros(shape), np.ascontiguousarray(vy), np.ascontiguousarray(vz)),
                     np.full(shape, p0), face, dims, bc, gamma)
    return Box(nx, ny, nz, h, h, h, bc, gamma, cell, face, name=f"alfvenic_shear_{nx}x{ny}x{nz}_{seed}")


def near_floor_state(dims, seed: int, bc=(OUTFLOW,) * 3, gamma: float = GAMMA, floor_cells: int = 4) -> Box:
    """Density spanning 1e-8 .. 1 (log-smooth), temperature p/rho ~ 0.5, slow
    flow (|v| ~ 0.1) and a weak uniform field (|B| = 1e-5), so that thermal
    energy dominates even at the lowest densities; in `floor_cells` seeded
    cells of the lowest-density tenth the total energy is set to half the
    kinetic energy, so their recovered pressure is negative and takes the
    pressure floor."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    h = 1.0 / max(dims)
    fr, ft, fvx, fvy, fvz = _smooth_fields(dims, rng, 5)
    rho = 10.0 ** (-4.0 + 4.0 * np.tanh(1.5 * fr))
    p = rho * (0.5 + 0.2 * np.tanh(ft))
    v = (0.1 * fvx, 0.1 * fvy, 0.1 * fvz)
    b = (1e-5 * 0.6, -1e-5 * 0.64, 1e-5 * 0.48)
    shapes = [(nz, ny, nx + (bc[0] == OUTFLOW)), (nz, ny + (bc[1] == OUTFLOW), nx), (nz + (bc[2] == OUTFLOW), ny, nx)]
    face = [np.full(shapes[d], b[d]) for d in range(3)]
    cell = conserved(rho, v, p, face, dims, bc, gamma)
    low = np.flatnonzero(rho.ravel() <= np.quantile(rho, 0.1))
    for s in rng.choice(low, size=min(floor_cells, low.size), replace=False):
        k, j, i = np.unravel_index(s, rho.shape)
        ke = 0.5 * (cell[1, k, j, i] ** 2 + cell[2, k, j, i] ** 2 + cell[3, k, j, i] ** 2) / cell[0, k, j, i]
        cell[4, k, j, i] = 0.5 * ke
    return Box(nx, ny, nz, h, h, h, tuple(bc), gamma, cell, face, name=f"near_floor_{nx}x{ny}x{nz}_{seed}")
