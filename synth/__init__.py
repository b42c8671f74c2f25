"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only draws numbers: mesh vertex coordinates, per-element
coefficients and random vectors. It contains none of the solver's arithmetic,
so both the CUDA path and the CPU oracle can take their inputs from it.
All generators use numpy's PCG64 with an explicit seed (default 2304).
"""
import numpy as np

DEFAULT_SEED = 2304


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def lattice_vertices(nx, ny, nz, perturb=0.0, seed=DEFAULT_SEED, extent=(1.0, 1.0, 1.0)):
    """Vertex coordinates (SoA vx, vy, vz) of an nx x ny x nz hex mesh of the box
    [0,Lx]x[0,Ly]x[0,Lz]; vertex (i,j,k) is stored at i + (nx+1)(j + (ny+1)k).
    Each coordinate of every interior vertex (one not on the boundary of the box)
    is moved by U(-perturb*h, +perturb*h), h the element size along that axis;
    boundary vertices stay where they are."""
    Lx, Ly, Lz = extent
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    x = (i * hx).astype(np.float64).ravel()
    y = (j * hy).astype(np.float64).ravel()
    z = (k * hz).astype(np.float64).ravel()
    if perturb > 0:
        rng = _rng(seed)
        n = x.size
        d = rng.uniform(-perturb, perturb, size=(3, n))
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        inner = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
        x = x + np.where(inner, d[0] * hx, 0.0)
        y = y + np.where(inner, d[1] * hy, 0.0)
        z = z + np.where(inner, d[2] * hz, 0.0)
    return x, y, z


def lognormal(n, sigma, seed=DEFAULT_SEED, mu=0.0):
    """exp(mu + sigma Z), Z ~ N(0,1) i.i.d., one value per element."""
    return np.exp(mu + sigma * _rng(seed).standard_normal(n))


def uniform(n, seed=DEFAULT_SEED, lo=-1.0, hi=1.0):
    """i.i.d. U(lo, hi) vector (FP64)."""
    return _rng(seed).uniform(lo, hi, size=n)


def layered_permeability(nx, ny, nz, sigma=3.0, corr_len=10.0, seed=DEFAULT_SEED):
    """Per-element permeability of a layered reservoir: independently per z layer
    and y row, an AR(1) sequence along x with correlation exp(-1/corr_len),
    normalised to unit variance; permeability = exp(sigma Z). Element order
    ex + nx (ey + ny ez)."""
    rng = _rng(seed)
    rho = np.exp(-1.0 / corr_len)
    Z = np.zeros((nz, ny, nx))
    Z[:, :, 0] = rng.standard_normal((nz, ny))
    s = np.sqrt(1.0 - rho * rho)
    for ix in range(1, nx):
        Z[:, :, ix] = rho * Z[:, :, ix - 1] + s * rng.standard_normal((nz, ny))
    return np.exp(sigma * Z).ravel()


def bent_tube_mask(nx, ny, nz, radius=0.15, bend_radius=0.6, seed=DEFAULT_SEED):
    """Boolean per element of the unit-cube mesh: True where the element centroid
    lies within `radius` of a quarter-circle arc {(R cos t, R sin t, 0.5) + c},
    t in [0, pi/2], with a seeded offset c ~ U(-0.05, 0.05)^3."""
    rng = _rng(seed)
    c = rng.uniform(-0.05, 0.05, size=3)
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    px = (ex.ravel() + 0.5) / nx - c[0]
    py = (ey.ravel() + 0.5) / ny - c[1]
    pz = (ez.ravel() + 0.5) / nz - c[2]
    t = np.clip(np.arctan2(py, px), 0.0, np.pi / 2)
    ax, ay = bend_radius * np.cos(t), bend_radius * np.sin(t)
    d2 = (px - ax) ** 2 + (py - ay) ** 2 + (pz - 0.5) ** 2
    return d2 <= radius * radius
