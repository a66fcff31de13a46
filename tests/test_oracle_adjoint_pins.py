"""Pins of the oracle's scatter-form adjoint.

The forward map F(x) = (su, sv, sw) is a quadratic form B(x, x), so its
Jacobian is J(x) d = B(x, d) + B(d, x) = F(x + d) - F(x) - F(d), computed
here with the forward oracle alone (independent of the adjoint code). On
integer winds with dyadic coefficients every operation is exact, so the
identities below hold bit for bit:
  dot-product test   <J(x) d, y> = <d, J(x)^T y>
  Euler identity     <J(x)^T y, x> = <y, J(x) x> = 2 <y, F(x)>
"""
import numpy as np
import pytest

from paper_2107_13500_gb300 import synth


def _raw_integer(nx, ny, nz, seed, stream, lo=-6, hi=6):
    """Integer values on every cell, halo included (no periodicity), zero padding."""
    f = synth.empty_field(nx, ny, nz)
    f[:, :, : nx + 2] = synth.randint(seed, stream, nz * (ny + 2) * (nx + 2), lo, hi).reshape(
        nz, ny + 2, nx + 2).astype(np.float64)
    return f


def _mask_interior(f, nx, ny):
    g = np.zeros_like(f)
    g[:, 1:ny + 1, 1:nx + 1] = f[:, 1:ny + 1, 1:nx + 1]
    return g


@pytest.mark.parametrize("shape", [(5, 4, 6), (3, 7, 2), (6, 6, 3)])
def test_dot_product_exact(oracle_lib, shape):
    nx, ny, nz = shape
    c = oracle_lib.coeffs(nz, 0.25, 0.5, synth.dz_uniform(nz, 0.5))
    x = [_raw_integer(nx, ny, nz, 21, s) for s in range(3)]
    d = [_raw_integer(nx, ny, nz, 22, s) for s in range(3)]
    y = [_mask_interior(_raw_integer(nx, ny, nz, 23, s), nx, ny) for s in range(3)]
    fx = oracle_lib.advect(*x, c, nx, ny)
    fd = oracle_lib.advect(*d, c, nx, ny)
    fxd = oracle_lib.advect(*[a + b for a, b in zip(x, d)], c, nx, ny)
    jd = [a - b - e for a, b, e in zip(fxd, fx, fd)]
    lhs = sum(float(np.sum(_mask_interior(j, nx, ny) * yy)) for j, yy in zip(jd, y))
    g = oracle_lib.advect_adjoint(*x, c, nx, ny, *y)
    rhs = sum(float(np.sum(gg * dd)) for gg, dd in zip(g, d))
    assert lhs == rhs
    # Euler identity for a quadratic form
    euler = sum(float(np.sum(gg * xx)) for gg, xx in zip(g, x))
    two_f = 2.0 * sum(float(np.sum(_mask_interior(f, nx, ny) * yy)) for f, yy in zip(fx, y))
    assert euler == two_f


def test_dot_product_random_stretched(oracle_lib):
    """Same identity on real-valued winds with density and a stretched grid,
    to rounding."""
    nx, ny, nz = 9, 8, 12
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    c = oracle_lib.coeffs(nz, 50.0, 40.0, dz, rho, rhon)
    x = list(synth.fields_iid(nx, ny, nz, seed=31))
    d = [f.copy() for f in synth.fields_iid(nx, ny, nz, seed=32)]
    y = [_mask_interior(f, nx, ny) for f in synth.fields_iid(nx, ny, nz, seed=33)]
    h = 2.0 ** -10
    fp = oracle_lib.advect(*[a + h * b for a, b in zip(x, d)], c, nx, ny)
    fm = oracle_lib.advect(*[a - h * b for a, b in zip(x, d)], c, nx, ny)
    jd = [(p - m) / (2 * h) for p, m in zip(fp, fm)]   # exact for a quadratic up to rounding
    lhs = sum(float(np.sum(_mask_interior(j, nx, ny) * yy)) for j, yy in zip(jd, y))
    g = oracle_lib.advect_adjoint(*x, c, nx, ny, *y)
    rhs = sum(float(np.sum(gg * dd)) for gg, dd in zip(g, d))
    scale = sum(float(np.sum(np.abs(gg * dd))) for gg, dd in zip(g, d))
    assert abs(lhs - rhs) <= 1e-11 * scale


def test_adjoint_touches_only_read_cells(oracle_lib):
    """Padding columns beyond the halo are never read, so get no gradient."""
    nx, ny, nz = 5, 4, 4
    c = oracle_lib.coeffs(nz, 0.25, 0.5, synth.dz_uniform(nz, 0.5))
    x = [_raw_integer(nx, ny, nz, 41, s) for s in range(3)]
    y = [_mask_interior(_raw_integer(nx, ny, nz, 42, s), nx, ny) for s in range(3)]
    g = oracle_lib.advect_adjoint(*x, c, nx, ny, *y)
    for gg in g:
        assert np.all(gg[:, :, nx + 2:] == 0)
