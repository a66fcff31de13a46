"""Seeded synthetic inputs for PW advection (fields, grids, densities, layouts).

This module holds input generation only: random numbers, analytic wind
patterns, vertical grid spacings, densities and the padded storage layout.
It contains none of the advection arithmetic, so both the GPU library's
tests and the CPU oracle can draw the same inputs from it.

Layout: a field of an nx x ny x nz domain is a float array of shape
``(nz, ny + 2, sy)`` indexed ``[k, j, i]`` (x fastest). ``i = 0`` and
``i = nx + 1`` (likewise ``j``) are the one-cell halo; columns ``i > nx + 1``
are row padding so that every row starts on a 32-byte boundary.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
used as a counter-based generator: value n of stream s under seed q is
``mix64(key(q, s) + (n + 1) * 0x9E3779B97F4A7C15)``, turned into a double in
[0, 1) from its top 53 bits.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    base = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1 + 0x632BE59BD9B4E019) & (2**64 - 1)],
                    dtype=np.uint64)
    return _mix64(base)[0]


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream ``stream`` of seed ``seed``."""
    with np.errstate(over="ignore"):
        ctr = (np.arange(1, n + 1, dtype=np.uint64) * GOLDEN_GAMMA) + _key(seed, stream)
        bits = _mix64(ctr)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, stream: int, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, n)


def randint(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in [lo, hi] inclusive."""
    return lo + np.floor(uniform01(seed, stream, n) * (hi - lo + 1)).astype(np.int64)


# ----------------------------------------------------------------------------
# Layout


def row_stride(nx: int, elem_bytes: int) -> int:
    """Padded row length (elements) for nx interior points: nx + 2 rounded up
    so that a row is a whole number of 32-byte sectors."""
    per = 32 // elem_bytes
    return ((nx + 2 + per - 1) // per) * per


def empty_field(nx: int, ny: int, nz: int, dtype=np.float64) -> np.ndarray:
    sy = row_stride(nx, np.dtype(dtype).itemsize)
    return np.zeros((nz, ny + 2, sy), dtype=dtype)


def fill_periodic_halo(f: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Copy the interior's opposite edges into the halo (x first, then y, so
    corners are filled too). Works in place and returns f."""
    f[:, :, 0] = f[:, :, nx]
    f[:, :, nx + 1] = f[:, :, 1]
    f[:, 0, :] = f[:, ny, :]
    f[:, ny + 1, :] = f[:, 1, :]
    return f


def interior(f: np.ndarray, nx: int, ny: int) -> np.ndarray:
    return f[:, 1:ny + 1, 1:nx + 1]


# ----------------------------------------------------------------------------
# Vertical grids and densities


def dz_uniform(nz: int, dz: float) -> np.ndarray:
    """Cell thicknesses; entry 0 (below the first w level) is unused."""
    return np.full(nz, float(dz))


def dz_stretched(nz: int, dz0: float = 10.0, ratio: float = 1.03) -> np.ndarray:
    """dz(k) = dz0 * ratio**(k-2) for paper levels k = 2..nz (index k-1)."""
    d = np.empty(nz)
    d[0] = dz0
    for k in range(1, nz):
        d[k] = dz0 * ratio ** (k - 1)
    return d


def level_heights(dz: np.ndarray):
    """(z_w, z_n): heights of the w levels (z_w[0] = 0) and of the u/v levels
    (midpoints, with a mirrored ghost level below the ground)."""
    nz = dz.shape[0]
    zw = np.zeros(nz)
    for k in range(1, nz):
        zw[k] = zw[k - 1] + dz[k]
    zn = np.zeros(nz)
    for k in range(1, nz):
        zn[k] = 0.5 * (zw[k - 1] + zw[k])
    if nz > 1:
        zn[0] = -zn[1]
    return zw, zn


def density_exponential(dz: np.ndarray, rho0: float = 1.2, scale_height: float = 8000.0):
    """(rho_w, rho_n): an isothermal-atmosphere density at the w and u levels."""
    zw, zn = level_heights(dz)
    return rho0 * np.exp(-zw / scale_height), rho0 * np.exp(-zn / scale_height)


# ----------------------------------------------------------------------------
# Wind fields


def fields_iid(nx, ny, nz, seed=1, lo=-10.0, hi=10.0, dtype=np.float64):
    """u, v, w i.i.d. uniform in [lo, hi] on the interior (streams 0, 1, 2),
    periodic halo in x and y."""
    out = []
    for s in range(3):
        f = empty_field(nx, ny, nz, dtype)
        vals = uniform(seed, s, nx * ny * nz, lo, hi).reshape(nz, ny, nx)
        f[:, 1:ny + 1, 1:nx + 1] = vals
        out.append(fill_periodic_halo(f, nx, ny))
    return tuple(out)


def fields_integer(nx, ny, nz, seed=3, lo=-8, hi=8, rigid=False):
    """u, v, w with small integer values (exact in every format used)."""
    out = []
    for s in range(3):
        f = empty_field(nx, ny, nz)
        vals = randint(seed, s, nx * ny * nz, lo, hi).astype(np.float64).reshape(nz, ny, nx)
        f[:, 1:ny + 1, 1:nx + 1] = vals
        out.append(fill_periodic_halo(f, nx, ny))
    if rigid:
        out[2][0] = 0.0
        out[2][nz - 1] = 0.0
    return tuple(out)


def fields_modes(nx, ny, nz, dx, dy, dz, seed=2, n_modes=8, mean_u=5.0, noise=0.01):
    """Smooth periodic winds: each field is a sum of n_modes travelling
    sinusoids A sin(2 pi (kx x/Lx + ky y/Ly) + kz pi z/Lz + phi) with integer
    kx, ky in [1, 4], kz in [1, 3], A ~ U[0.5, 2], phi ~ U[0, 2 pi), plus
    uniform noise of +-noise * max|field|. u gets mean mean_u, v and w mean 0;
    w is zero on the bottom and top w levels.

    Positions follow the C-grid: u at x = i*dx (cell faces), v at y = j*dy,
    others at cell centres (i - 1/2)*dx; u, v at the u-level heights, w at
    the w-level heights.
    """
    zw, zn = level_heights(dz)
    Lx, Ly, Lz = nx * dx, ny * dy, max(zw[-1], 1.0)
    xc = (np.arange(1, nx + 1) - 0.5) * dx
    xf = np.arange(1, nx + 1) * dx
    yc = (np.arange(1, ny + 1) - 0.5) * dy
    yf = np.arange(1, ny + 1) * dy
    pos = {0: (xf, yc, zn), 1: (xc, yf, zn), 2: (xc, yc, zw)}
    means = (mean_u, 0.0, 0.0)
    out = []
    for s in range(3):
        x, y, z = pos[s]
        base = 16 * s
        kx = randint(seed, base + 0, n_modes, 1, 4)
        ky = randint(seed, base + 1, n_modes, 1, 4)
        kz = randint(seed, base + 2, n_modes, 1, 3)
        amp = uniform(seed, base + 3, n_modes, 0.5, 2.0)
        phi = uniform(seed, base + 4, n_modes, 0.0, 2.0 * math.pi)
        val = np.zeros((nz, ny, nx))
        for m in range(n_modes):
            ex = np.exp(1j * (2.0 * math.pi * kx[m] * x / Lx))
            ey = np.exp(1j * (2.0 * math.pi * ky[m] * y / Ly))
            ez = np.exp(1j * (math.pi * kz[m] * z / Lz + phi[m]))
            eyx = ey[:, None] * ex[None, :]
            for k in range(nz):
                val[k] += amp[m] * (ez[k] * eyx).imag
        mx = float(np.max(np.abs(val))) if val.size else 0.0
        val += uniform(seed, base + 5, nx * ny * nz, -noise * mx, noise * mx).reshape(nz, ny, nx)
        val += means[s]
        if s == 2:
            val[0] = 0.0
            val[nz - 1] = 0.0
        f = empty_field(nx, ny, nz)
        f[:, 1:ny + 1, 1:nx + 1] = val
        out.append(fill_periodic_halo(f, nx, ny))
    return tuple(out)


# ----------------------------------------------------------------------------
# Named workloads (the five configurations the library is measured on)


def config_small_iid(seed=1):
    """64 x 64 x 64, periodic, i.i.d. U[-10, 10] winds, dx = dy = 50 m,
    uniform dz = 20 m."""
    nx = ny = nz = 64
    return dict(nx=nx, ny=ny, nz=nz, dx=50.0, dy=50.0, dz=dz_uniform(nz, 20.0),
                fields=lambda: fields_iid(nx, ny, nz, seed=seed))


def config_16m_modes(seed=2):
    """512 x 512 x 64 (16.8M points), smooth 8-mode winds with a 5 m/s mean
    wind, dx = dy = 50 m, dz growing from 10 m by 3 % per level."""
    nx, ny, nz = 512, 512, 64
    dz = dz_stretched(nz, 10.0, 1.03)
    return dict(nx=nx, ny=ny, nz=nz, dx=50.0, dy=50.0, dz=dz,
                fields=lambda: fields_modes(nx, ny, nz, 50.0, 50.0, dz, seed=seed))


def config_134m_iid(seed=1):
    """1024 x 1024 x 128 (134M points) with the winds and grid of the small
    configuration."""
    nx, ny, nz = 1024, 1024, 128
    return dict(nx=nx, ny=ny, nz=nz, dx=50.0, dy=50.0, dz=dz_uniform(nz, 20.0),
                fields=lambda: fields_iid(nx, ny, nz, seed=seed))


def batched_domain_sizes(n=96, seed=4):
    """Uneven domain sizes: x, y uniform in [32, 384], z uniform in [32, 128]."""
    nx = randint(seed, 0, n, 32, 384)
    ny = randint(seed, 1, n, 32, 384)
    nz = randint(seed, 2, n, 32, 128)
    return [(int(a), int(b), int(c)) for a, b, c in zip(nx, ny, nz)]
