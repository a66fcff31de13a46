"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
tendencies of linear winds, exact zeros, the x<->y transpose identity that
ties sv to Listing 1's su, discrete energy conservation (which any sign or
index slip in a flux breaks), second-order convergence to the continuous
tendency -(u.grad)q - q div(u)/2, exact homogeneity, the paper's printed
operation counts, and closed forms of the stretched-grid coefficients.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2107_13500_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _coeffs(oracle, nz, dx, dy, dz, rho=None, rhon=None):
    return oracle.coeffs(nz, dx, dy, dz, rho, rhon)


def _field_from(fn, nx, ny, nz, dx, dy, zlev):
    """Fill every cell (halo included) from fn(x_index, y_index, k) arrays."""
    f = synth.empty_field(nx, ny, nz)
    ii = np.arange(0, nx + 2)
    jj = np.arange(0, ny + 2)
    for k in range(nz):
        f[k, :, : nx + 2] = fn(ii[None, :], jj[:, None], k)
    return f


def _interior(f, nx, ny, k0=0, k1=None):
    return f[k0:k1, 1:ny + 1, 1:nx + 1]


# ---------------------------------------------------------------- coefficients

def test_coeffs_uniform_grid(oracle_lib):
    nz = 12
    c = _coeffs(oracle_lib, nz, 50.0, 40.0, synth.dz_uniform(nz, 20.0))
    assert c["tcx"] == 0.25 / 50.0 and c["tcy"] == 0.25 / 40.0
    assert c["tzc1"][0] == 0 and c["tzc2"][0] == 0
    np.testing.assert_array_equal(c["tzc1"][1:], 0.25 / 20.0)
    np.testing.assert_array_equal(c["tzc2"][1:], 0.25 / 20.0)
    np.testing.assert_array_equal(c["tzd1"][1:nz - 1], 0.25 / 20.0)
    np.testing.assert_array_equal(c["tzd2"][1:nz - 1], 0.25 / 20.0)
    assert c["tzd1"][0] == c["tzd2"][0] == c["tzd1"][nz - 1] == c["tzd2"][nz - 1] == 0


def test_coeffs_stretched_closed_form(oracle_lib):
    """dz(k) = 10 * 1.03**(k-2): the spacing around w level k is the mean of
    the two adjacent thicknesses, so tzd = 0.5/(dz(k) + dz(k+1)); tzc = 0.25/dz(k)."""
    nz = 64
    r = 1.03
    dz = synth.dz_stretched(nz, 10.0, r)
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, dz)
    k = np.arange(1, nz)
    dzk = 10.0 * r ** (k - 1)
    np.testing.assert_allclose(c["tzc1"][1:], 0.25 / dzk, rtol=1e-14)
    np.testing.assert_allclose(c["tzc2"][1:], 0.25 / dzk, rtol=1e-14)
    k = np.arange(1, nz - 1)
    np.testing.assert_allclose(c["tzd1"][1:nz - 1],
                               0.5 / (10.0 * r ** (k - 1) + 10.0 * r ** k), rtol=1e-12)


def test_coeffs_density_ratio(oracle_lib):
    """With rho = exp(-z/H): tzc1/tzc2 = rho(k-1)/rho(k) = exp(dz(k)/H) and
    tzd2/tzd1 = rhon(k+1)/rhon(k) = exp(-(zn(k+1)-zn(k))/H)."""
    nz, H = 40, 8000.0
    dz = synth.dz_stretched(nz, 10.0, 1.03)
    rho, rhon = synth.density_exponential(dz, 1.2, H)
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, dz, rho, rhon)
    k = np.arange(1, nz)
    np.testing.assert_allclose(c["tzc1"][k] / c["tzc2"][k], np.exp(dz[k] / H), rtol=1e-13)
    k = np.arange(1, nz - 1)
    dzn = 0.5 * (dz[k] + dz[k + 1])
    np.testing.assert_allclose(c["tzd2"][k] / c["tzd1"][k], np.exp(-dzn / H), rtol=1e-12)


def test_coeffs_rejects_bad_input(oracle_lib):
    with pytest.raises(ValueError):
        _coeffs(oracle_lib, 8, 0.0, 1.0, synth.dz_uniform(8, 1.0))
    bad = synth.dz_uniform(8, 1.0)
    bad[3] = -1.0
    with pytest.raises(ValueError):
        _coeffs(oracle_lib, 8, 1.0, 1.0, bad)


# ---------------------------------------------------------------- exact zeros

@pytest.mark.parametrize("stretched", [False, True])
def test_level_constant_winds_give_zero(oracle_lib, stretched):
    """u = U(k), v = V(k), w = 0: every flux difference cancels exactly."""
    nx, ny, nz = 9, 7, 10
    dz = synth.dz_stretched(nz) if stretched else synth.dz_uniform(nz, 20.0)
    rho, rhon = synth.density_exponential(dz) if stretched else (None, None)
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, dz, rho, rhon)
    U = synth.uniform(7, 0, nz, -10, 10)
    V = synth.uniform(7, 1, nz, -10, 10)
    u = synth.empty_field(nx, ny, nz)
    v = synth.empty_field(nx, ny, nz)
    w = synth.empty_field(nx, ny, nz)
    u[:] = U[:, None, None]
    v[:] = V[:, None, None]
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    for s in (su, sv, sw):
        assert np.all(_interior(s, nx, ny) == 0.0)


def test_error_scale_bounds_result(oracle_lib):
    """The per-point error scale (sum of |monomials|) bounds |result| by the
    triangle inequality, equals it when every monomial has one sign (all
    winds positive, only x self terms), and scales with degree two."""
    nx, ny, nz = 9, 8, 7
    c = oracle_lib.coeffs(nz, 50.0, 40.0, synth.dz_stretched(nz))
    u, v, w = synth.fields_iid(nx, ny, nz, seed=13)
    s, a = oracle_lib.advect(u, v, w, c, nx, ny, want_abs=True)
    for si, ai in zip(s, a):
        assert np.all(np.abs(si) <= ai * (1 + 1e-15))
    s2, a2 = oracle_lib.advect(2 * u, 2 * v, 2 * w, c, nx, ny, want_abs=True)
    for ai, bi in zip(a, a2):
        np.testing.assert_array_equal(4 * ai, bi)


def test_error_scales_closed_form_and_order(oracle_lib):
    """The two error scales on a field whose face sums cancel exactly: u
    alternating +1/-1 along x, v = w = 0. Every face of su then carries
    a + b = 0, so su = 0 and the strict scale (|c||q||a+b| per face) is 0,
    while the monomial scale (|c||q|(|a|+|b|)) is tcx (1*2 + 1*2) = 4 tcx.
    On all-positive winds the two scales are equal bit for bit, and on any
    winds strict <= monomial."""
    nx, ny, nz = 8, 5, 4
    dz = synth.dz_uniform(nz, 20.0)
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, dz)
    u = _field_from(lambda i, j, k: np.where(i % 2 == 0, 1.0, -1.0) + 0.0 * j, nx, ny, nz, 50.0, 50.0, None)
    v = synth.empty_field(nx, ny, nz)
    w = synth.empty_field(nx, ny, nz)
    (su, _, _), (a, _, _) = oracle_lib.advect(u, v, w, c, nx, ny, want_abs=True)
    m, _, _ = oracle_lib.monomial_scale(u, v, w, c, nx, ny)
    assert np.all(_interior(su, nx, ny) == 0.0)
    assert np.all(_interior(a, nx, ny) == 0.0)
    np.testing.assert_array_equal(_interior(m, nx, ny, 1), 4 * c["tcx"])
    assert np.all(_interior(m, nx, ny, 0, 1) == 0.0)  # level 1 is not computed
    up = [np.abs(f) + 1.0 for f in synth.fields_iid(nx, ny, nz, seed=14)]
    _, ap = oracle_lib.advect(*up, c, nx, ny, want_abs=True)
    mp = oracle_lib.monomial_scale(*up, c, nx, ny)
    for x, y in zip(ap, mp):
        np.testing.assert_array_equal(x, y)
    f = synth.fields_iid(nx, ny, nz, seed=15)
    _, af = oracle_lib.advect(*f, c, nx, ny, want_abs=True)
    mf = oracle_lib.monomial_scale(*f, c, nx, ny)
    for x, y in zip(af, mf):
        assert np.all(x <= y)
        assert np.any(x < y)


def test_level_one_is_not_computed(oracle_lib):
    nx, ny, nz = 6, 5, 6
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0))
    u, v, w = synth.fields_iid(nx, ny, nz, seed=11)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    for s in (su, sv, sw):
        assert np.all(s[0] == 0.0)
    assert np.all(sw[nz - 1] == 0.0)
    assert np.any(su[nz - 1] != 0.0) and np.any(sv[nz - 1] != 0.0)


# ---------------------------------------------------------------- closed forms

DX, DY, DZ = 0.5, 0.25, 0.5      # dyadic, so every intermediate below is exact


def _setup_closed(oracle_lib, nx=10, ny=8, nz=9):
    c = _coeffs(oracle_lib, nz, DX, DY, synth.dz_uniform(nz, DZ))
    zn = (np.arange(nz) - 0.5) * DZ         # u-level heights; zn[0] = -zn[1]
    zw = np.arange(nz) * DZ                  # w-level heights
    return nx, ny, nz, c, zn, zw


def _const(nx, ny, nz, val):
    f = synth.empty_field(nx, ny, nz)
    f[:] = val
    return f


def test_closed_form_su_self_term(oracle_lib):
    """u = a x (u points at x = i dx), v = w = 0: su = -3/2 a^2 x exactly."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    a = 0.75
    u = _field_from(lambda i, j, k: a * i * DX + 0 * j, nx, ny, nz, DX, DY, zn)
    v, w = _const(nx, ny, nz, 0.0), _const(nx, ny, nz, 0.0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    x = np.arange(1, nx + 1) * DX
    expect = np.broadcast_to(-1.5 * a * a * x, (nz - 1, ny, nx))
    np.testing.assert_array_equal(_interior(su, nx, ny, 1), expect)
    assert np.all(_interior(sv, nx, ny) == 0) and np.all(_interior(sw, nx, ny) == 0)


def test_closed_form_sv_self_term(oracle_lib):
    """v = b y (v points at y = j dy), u = w = 0: sv = -3/2 b^2 y exactly."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    b = -1.25
    v = _field_from(lambda i, j, k: b * j * DY + 0 * i, nx, ny, nz, DX, DY, zn)
    u, w = _const(nx, ny, nz, 0.0), _const(nx, ny, nz, 0.0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    y = np.arange(1, ny + 1) * DY
    expect = np.broadcast_to((-1.5 * b * b * y)[:, None], (nz - 1, ny, nx))
    np.testing.assert_array_equal(_interior(sv, nx, ny, 1), expect)
    assert np.all(_interior(su, nx, ny) == 0) and np.all(_interior(sw, nx, ny) == 0)


def test_closed_form_sw_self_term(oracle_lib):
    """w = g z (w levels, w = 0 on the ground), u = v = 0:
    sw = -3/2 g^2 z on levels 2..nz-1, 0 on the top level."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    g = 0.5
    w = _field_from(lambda i, j, k: g * zw[k] + 0 * i + 0 * j, nx, ny, nz, DX, DY, zw)
    u, v = _const(nx, ny, nz, 0.0), _const(nx, ny, nz, 0.0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    expect = np.broadcast_to((-1.5 * g * g * zw[1:nz - 1])[:, None, None], (nz - 2, ny, nx))
    np.testing.assert_array_equal(_interior(sw, nx, ny, 1, nz - 1), expect)
    assert np.all(_interior(su, nx, ny) == 0) and np.all(_interior(sv, nx, ny) == 0)


def test_closed_form_su_cross_y(oracle_lib):
    """u = a y, v = V0: su = -V0 a (the -v du/dy advection), sv = sw = 0."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    a, V0 = 1.5, -2.0
    u = _field_from(lambda i, j, k: a * (j - 0.5) * DY + 0 * i, nx, ny, nz, DX, DY, zn)
    v, w = _const(nx, ny, nz, V0), _const(nx, ny, nz, 0.0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    np.testing.assert_array_equal(_interior(su, nx, ny, 1), -V0 * a)
    assert np.all(_interior(sv, nx, ny) == 0) and np.all(_interior(sw, nx, ny) == 0)


def test_closed_form_sv_cross_x(oracle_lib):
    """v = b x, u = U0: sv = -U0 b, su = sw = 0."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    b, U0 = -0.75, 3.0
    v = _field_from(lambda i, j, k: b * (i - 0.5) * DX + 0 * j, nx, ny, nz, DX, DY, zn)
    u, w = _const(nx, ny, nz, U0), _const(nx, ny, nz, 0.0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    np.testing.assert_array_equal(_interior(sv, nx, ny, 1), -U0 * b)
    assert np.all(_interior(su, nx, ny) == 0) and np.all(_interior(sw, nx, ny) == 0)


def test_closed_form_su_cross_z(oracle_lib):
    """u = a zn, w = W0: su = -W0 a below the top level; sw = 0."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    a, W0 = 0.25, 1.5
    u = _field_from(lambda i, j, k: a * zn[k] + 0 * i + 0 * j, nx, ny, nz, DX, DY, zn)
    v, w = _const(nx, ny, nz, 0.0), _const(nx, ny, nz, W0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    np.testing.assert_array_equal(_interior(su, nx, ny, 1, nz - 1), -W0 * a)
    assert np.all(_interior(sw, nx, ny) == 0) and np.all(_interior(sv, nx, ny) == 0)


def test_closed_form_sv_cross_z(oracle_lib):
    """v = b zn, w = W0: sv = -W0 b below the top level."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    b, W0 = -0.5, 2.0
    v = _field_from(lambda i, j, k: b * zn[k] + 0 * i + 0 * j, nx, ny, nz, DX, DY, zn)
    u, w = _const(nx, ny, nz, 0.0), _const(nx, ny, nz, W0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    np.testing.assert_array_equal(_interior(sv, nx, ny, 1, nz - 1), -W0 * b)
    assert np.all(_interior(su, nx, ny) == 0)


def test_closed_form_sw_cross_x_and_y(oracle_lib):
    """w = g x + h y, u = U0, v = V0: sw = -(U0 g + V0 h) on levels 2..nz-1,
    and su = sv = 0 below the top level."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    g, h, U0, V0 = 0.5, -0.25, 2.0, 4.0
    w = _field_from(lambda i, j, k: g * (i - 0.5) * DX + h * (j - 0.5) * DY, nx, ny, nz, DX, DY, zw)
    u, v = _const(nx, ny, nz, U0), _const(nx, ny, nz, V0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    np.testing.assert_array_equal(_interior(sw, nx, ny, 1, nz - 1), -(U0 * g + V0 * h))
    assert np.all(_interior(su, nx, ny, 1, nz - 1) == 0)
    assert np.all(_interior(sv, nx, ny, 1, nz - 1) == 0)


def test_top_level_keeps_only_lower_flux(oracle_lib):
    """Listing 1's else branch: at k = nz only tzc1(k) u(k-1)(w(k-1,i)+w(k-1,i+1))
    remains. With u = U0 and w = W0 that is 2 tzc1 U0 W0 (su) and likewise sv."""
    nx, ny, nz, c, zn, zw = _setup_closed(oracle_lib)
    U0, V0, W0 = 1.5, -0.5, 2.0
    u, v, w = _const(nx, ny, nz, U0), _const(nx, ny, nz, V0), _const(nx, ny, nz, W0)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    t = c["tzc1"][nz - 1]
    np.testing.assert_array_equal(_interior(su, nx, ny, nz - 1), 2 * t * U0 * W0)
    np.testing.assert_array_equal(_interior(sv, nx, ny, nz - 1), 2 * t * V0 * W0)
    np.testing.assert_array_equal(_interior(su, nx, ny, 1, nz - 1), 0.0)


# ---------------------------------------------------------------- symmetry

def _transpose(f, nx, ny):
    """Swap x and y of a field (nz, ny+2, sy) -> (nz, nx+2, sy')."""
    t = synth.empty_field(ny, nx, f.shape[0])
    t[:, :, : ny + 2] = np.transpose(f[:, : ny + 2, : nx + 2], (0, 2, 1))
    return t


def test_transpose_identity_sv_from_su(oracle_lib):
    """sv(u, v, w; tcx, tcy) == T su(Tv, Tu, Tw; tcy, tcx) bit for bit, and
    the same with su and sv exchanged (T swaps x and y)."""
    nx, ny, nz = 11, 7, 8
    dz = synth.dz_stretched(nz)
    c = _coeffs(oracle_lib, nz, 50.0, 30.0, dz)
    ct = dict(c, tcx=c["tcy"], tcy=c["tcx"])
    u, v, w = synth.fields_iid(nx, ny, nz, seed=5)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    tu, tv, tw = _transpose(v, nx, ny), _transpose(u, nx, ny), _transpose(w, nx, ny)
    su_t, sv_t, sw_t = oracle_lib.advect(tu, tv, tw, ct, ny, nx)
    np.testing.assert_array_equal(_interior(sv, nx, ny), _interior(_transpose(su_t, ny, nx), nx, ny))
    np.testing.assert_array_equal(_interior(su, nx, ny), _interior(_transpose(sv_t, ny, nx), nx, ny))
    # sw adds its x and y terms in the other order after the swap: rounding only.
    np.testing.assert_allclose(_interior(sw, nx, ny), _interior(_transpose(sw_t, ny, nx), nx, ny),
                               rtol=0, atol=1e-12)


def test_homogeneity_degree_two(oracle_lib):
    """The map is a quadratic form: F(2x) = 4 F(x) exactly in binary FP."""
    nx, ny, nz = 8, 9, 7
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, synth.dz_stretched(nz))
    u, v, w = synth.fields_iid(nx, ny, nz, seed=6)
    a = oracle_lib.advect(u, v, w, c, nx, ny)
    b = oracle_lib.advect(2 * u, 2 * v, 2 * w, c, nx, ny)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(4 * x, y)


# ---------------------------------------------------------------- conservation

def test_discrete_energy_conservation(oracle_lib):
    """Periodic in x and y, w = 0 on the ground and at the lid, stretched grid
    with density: sum dz rhon u su = sum dz rhon v sv = sum dzn rho w sw = 0,
    to rounding relative to the sum of the absolute summands."""
    nx, ny, nz = 16, 12, 20
    dz = synth.dz_stretched(nz, 10.0, 1.03)
    rho, rhon = synth.density_exponential(dz, 1.2, 8000.0)
    c = _coeffs(oracle_lib, nz, 50.0, 40.0, dz, rho, rhon)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=9)
    w[0] = 0.0
    w[nz - 1] = 0.0
    (su, sv, sw), (au, av, aw) = oracle_lib.advect(u, v, w, c, nx, ny, want_abs=True)
    zw, zn = synth.level_heights(dz)
    wu = (dz * rhon)[1:, None, None]
    dzn = np.zeros(nz)
    dzn[:nz - 1] = zn[1:] - zn[:nz - 1]
    ww = (dzn * rho)[1:, None, None]
    for f, s, a, wt in ((u, su, au, wu), (v, sv, av, wu), (w, sw, aw, ww)):
        terms = wt * _interior(f, nx, ny, 1) * _interior(s, nx, ny, 1)
        scale = np.sum(wt * np.abs(_interior(f, nx, ny, 1)) * _interior(a, nx, ny, 1))
        assert abs(terms.sum()) <= 1e-14 * scale, (terms.sum(), scale)


def test_energy_weights_closed_form(oracle_lib):
    """Uniform 20 m levels, no density: every u/v cell weighs dz = 20 and
    every computed w cell dzn = 20. Geometric levels: the w cell around
    level k spans half of each adjacent layer, dzn = (dz(k) + dz(k+1)) / 2;
    density multiplies in the level's own value."""
    nz = 10
    wu, ww = oracle_lib.energy_weights(nz, synth.dz_uniform(nz, 20.0))
    assert wu[0] == 0.0 and np.all(wu[1:] == 20.0)
    assert ww[0] == 0.0 and ww[nz - 1] == 0.0 and np.all(ww[1:nz - 1] == 20.0)
    dz = synth.dz_stretched(nz, 10.0, 1.5)
    rho, rhon = synth.density_exponential(dz, 1.2, 2000.0)
    wu, ww = oracle_lib.energy_weights(nz, dz, rho, rhon)
    k = np.arange(1, nz - 1)
    np.testing.assert_allclose(wu[1:], dz[1:] * rhon[1:], rtol=1e-15)
    np.testing.assert_allclose(ww[k], 0.5 * (dz[k] + dz[k + 1]) * rho[k], rtol=1e-14)


def test_energy_budget_sums(oracle_lib):
    """pwo_energy_budget on fields whose sums are known: u = su = 1 gives
    nx ny sum(wu); v = 2, sv = -3 gives -6 nx ny sum(wu) with absolute sum
    +6 nx ny sum(wu); w = sw = 0 gives 0. Halo cells never count."""
    nx, ny, nz = 7, 5, 6
    dz = synth.dz_stretched(nz)
    wu, ww = oracle_lib.energy_weights(nz, dz)
    one = synth.empty_field(nx, ny, nz) + 1.0
    two, m3 = 2.0 * one, -3.0 * one
    zero = synth.empty_field(nx, ny, nz)
    for f in (one, two, m3):
        f[:, 0, :] = 1e30  # halo rows: must not enter the sums
        f[:, :, 0] = 1e30
    out = oracle_lib.energy_budget(one, two, zero, one, m3, zero, wu, ww, nx, ny)
    tot = nx * ny * float(np.sum(wu))
    np.testing.assert_allclose(out, [tot, -6 * tot, 0.0, tot, 6 * tot, 0.0], rtol=1e-14)


def test_energy_budget_of_oracle_output_conserves(oracle_lib):
    """The oracle's own source terms on a periodic domain with w = 0 on the
    ground and the lid: each weighted sum vanishes to rounding relative to
    the sum of |mass x wind x error scale| (stretched grid with density)."""
    nx, ny, nz = 14, 10, 18
    dz = synth.dz_stretched(nz, 10.0, 1.03)
    rho, rhon = synth.density_exponential(dz, 1.2, 8000.0)
    c = _coeffs(oracle_lib, nz, 50.0, 40.0, dz, rho, rhon)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=19)
    w[0] = 0.0
    w[nz - 1] = 0.0
    s, a = oracle_lib.advect(u, v, w, c, nx, ny, want_abs=True)
    wu, ww = oracle_lib.energy_weights(nz, dz, rho, rhon)
    out = oracle_lib.energy_budget(u, v, w, *s, wu, ww, nx, ny)
    for n, (f, ai, wt) in enumerate(zip((u, v, w), a, (wu, wu, ww))):
        scale = np.sum(wt[:, None, None] * np.abs(_interior(f, nx, ny)) * _interior(ai, nx, ny))
        assert abs(out[n]) <= 1e-14 * scale, (n, out[n], scale)
        assert out[3 + n] > 0


def test_energy_conservation_detects_flux_swap(oracle_lib):
    """Sanity of the invariant above: exchanging tzc1 and tzc2 (a plausible
    slip) breaks it by many orders of magnitude."""
    nx, ny, nz = 8, 8, 16
    dz = synth.dz_stretched(nz, 10.0, 1.03)
    rho, rhon = synth.density_exponential(dz, 1.2, 2000.0)
    c = _coeffs(oracle_lib, nz, 50.0, 50.0, dz, rho, rhon)
    bad = dict(c, tzc1=c["tzc2"].copy(), tzc2=c["tzc1"].copy())
    u, v, w = synth.fields_iid(nx, ny, nz, seed=10)
    w[0] = 0.0
    w[nz - 1] = 0.0
    (su, _, _), (au, _, _) = oracle_lib.advect(u, v, w, bad, nx, ny, want_abs=True)
    wu = (dz * rhon)[1:, None, None]
    tot = np.sum(wu * _interior(u, nx, ny, 1) * _interior(su, nx, ny, 1))
    scale = np.sum(wu * np.abs(_interior(u, nx, ny, 1)) * _interior(au, nx, ny, 1))
    assert abs(tot) > 1e-6 * scale


# ---------------------------------------------------------------- convergence

def _analytic_case(N):
    """Smooth winds on [0,L]^2 x [0,H], w = 0 at z = 0 and z = H. Returns
    fields on the C grid and the continuous tendency -(u.grad)q - q div(u)/2
    at each variable's own points."""
    L, H = 1000.0, 500.0
    nx = ny = N
    nz = N // 2 + 1
    dx, dy, dzv = L / nx, L / ny, H / (nz - 1)
    kx = 2 * math.pi / L
    kz = math.pi / H
    U0, V0 = 1.0, 0.5
    A, B, C = 1.0, 0.7, 0.3

    def fu(x, y, z):
        return U0 + A * np.sin(kx * x) * np.cos(kx * y) * np.cos(kz * z)

    def fv(x, y, z):
        return V0 + B * np.cos(kx * x) * np.sin(kx * y) * np.cos(kz * z)

    def fw(x, y, z):
        return C * np.sin(kx * x) * np.sin(kx * y) * np.sin(kz * z)

    def grad(f, x, y, z, h=1e-4):
        # fourth-order central differences of the analytic functions
        def d(g):
            return (-g(2 * h) + 8 * g(h) - 8 * g(-h) + g(-2 * h)) / (12 * h)
        fx = d(lambda e: f(x + e * L, y, z)) / L
        fy = d(lambda e: f(x, y + e * L, z)) / L
        fz = d(lambda e: f(x, y, z + e * L)) / L
        return fx, fy, fz

    def tendency(f, x, y, z):
        fx, fy, fz = grad(f, x, y, z)
        ux = grad(fu, x, y, z)[0]
        vy = grad(fv, x, y, z)[1]
        wz = grad(fw, x, y, z)[2]
        q = f(x, y, z)
        return -(fu(x, y, z) * fx + fv(x, y, z) * fy + fw(x, y, z) * fz) - 0.5 * q * (ux + vy + wz)

    zw = np.arange(nz) * dzv
    zn = (np.arange(nz) - 0.5) * dzv
    i = np.arange(0, nx + 2)[None, None, :]
    j = np.arange(0, ny + 2)[None, :, None]
    xc, xf = (i - 0.5) * dx, i * dx
    yc, yf = (j - 0.5) * dy, j * dy
    Zn, Zw = zn[:, None, None], zw[:, None, None]
    out = []
    for f, x, y, z in ((fu, xf, yc, Zn), (fv, xc, yf, Zn), (fw, xc, yc, Zw)):
        a = synth.empty_field(nx, ny, nz)
        a[:, :, : nx + 2] = f(x, y, z)
        out.append(a)
    tends = [tendency(fu, xf, yc, Zn), tendency(fv, xc, yf, Zn), tendency(fw, xc, yc, Zw)]
    return nx, ny, nz, dx, dy, synth.dz_uniform(nz, dzv), out, tends


def test_second_order_convergence(oracle_lib):
    """Error against the continuous tendency falls by ~4x per halving of the
    grid spacing for su, sv and sw (observed order >= 1.9 on the finest pair)."""
    errs = []
    for N in (16, 32, 64):
        nx, ny, nz, dx, dy, dz, (u, v, w), tends = _analytic_case(N)
        c = _coeffs(oracle_lib, nz, dx, dy, dz)
        s = oracle_lib.advect(u, v, w, c, nx, ny)
        e = []
        for idx, (si, ti) in enumerate(zip(s, tends)):
            k1 = nz - 1 if idx == 2 else nz
            ti = np.broadcast_to(ti, (nz, ny + 2, nx + 2))
            e.append(np.max(np.abs(si[1:k1, 1:ny + 1, 1:nx + 1] - ti[1:k1, 1:ny + 1, 1:nx + 1])))
        errs.append(e)
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    # pre-asymptotic on the coarsest pair; a first-order slip would give ~1
    assert np.all(order >= 1.85) and np.all(order[-1] >= 1.9), (errs, order)


# ---------------------------------------------------------------- exactness

def test_integer_inputs_are_exact(oracle_lib):
    """On integer winds and dyadic coefficients no FP64 operation rounds, so
    the oracle equals an exact rational evaluation of the same sums. (This
    checks exactness, which the GPU bit-exact test relies on; the formulas
    themselves are pinned by the tests above.)"""
    nx = ny = nz = 4
    dz = synth.dz_uniform(nz, 0.5)
    c = _coeffs(oracle_lib, nz, 0.25, 0.25, dz)
    u, v, w = synth.fields_integer(nx, ny, nz, seed=3)
    su, sv, sw = oracle_lib.advect(u, v, w, c, nx, ny)
    F = Fraction
    tcx, tcy = F(c["tcx"]), F(c["tcy"])
    for k in range(1, nz):
        tz1, tz2 = F(c["tzc1"][k]), F(c["tzc2"][k])
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                U = lambda kk, jj, ii: F(u[kk, jj, ii])
                V = lambda kk, jj, ii: F(v[kk, jj, ii])
                W = lambda kk, jj, ii: F(w[kk, jj, ii])
                s = tcx * (U(k, j, i - 1) * (U(k, j, i) + U(k, j, i - 1)) - U(k, j, i + 1) * (U(k, j, i) + U(k, j, i + 1)))
                s += tcy * (U(k, j - 1, i) * (V(k, j - 1, i) + V(k, j - 1, i + 1)) - U(k, j + 1, i) * (V(k, j, i) + V(k, j, i + 1)))
                s += tz1 * U(k - 1, j, i) * (W(k - 1, j, i) + W(k - 1, j, i + 1))
                if k < nz - 1:
                    s -= tz2 * U(k + 1, j, i) * (W(k, j, i) + W(k, j, i + 1))
                assert F(su[k, j, i]) == s


# ---------------------------------------------------------------- paper figures

def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    vals = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                key, val = line.split("=")
                vals[key.strip()] = float(val)
    return vals


def test_paper_operation_counts(oracle_lib):
    """Sec. III: 63 operations per cell, 55 at the column top, and the
    theoretical 18.86 GFLOPS at 300 MHz / 25.02 at 398 MHz for 64 levels."""
    g = _golden("paper_figures.txt")
    nz = int(g["column_levels"])
    per_col = oracle_lib.flops_per_column(nz)
    assert per_col == (nz - 2) * g["ops_per_cell"] + g["ops_column_top"]
    per_cell = per_col / (nz - 1)
    assert round(g["clock_u280_mhz"] * 1e6 * per_cell / 1e9, 2) == g["theoretical_gflops_u280"]
    assert round(g["clock_s10_mhz"] * 1e6 * per_cell / 1e9, 2) == g["theoretical_gflops_s10"]


def test_paper_traffic_volumes_match_bytes_per_point():
    """Sec. IV's host<->device volumes for 16M, 67M, 268M and 536M grid
    cells are the algorithmic 48 bytes per point of the FP64 path (read u,
    v, w, write su, sv, sw: 6 x 8 B), the volume every HBM fraction of the
    benchmark counts. The printed cell counts are power-of-two domains
    (2^24 .. 2^29 cells) truncated to whole millions; for those domains the
    48 B/pt volumes agree with the printed ones to the paper's rounding
    (within 1 %)."""
    from paper_2107_13500_gb300 import pw
    g = _golden("paper_figures.txt")
    bpp = pw.BYTES_PER_POINT["f64"]
    assert bpp == 6 * 8
    assert pw.BYTES_PER_POINT["paired"] == bpp
    assert pw.BYTES_PER_POINT["split"] == pw.BYTES_PER_POINT["f32"] == 6 * 4
    for tag in ("16m", "67m", "268m", "536m"):
        pts, vol = g[f"points_{tag}"], g[f"transfer_{tag}_bytes"]
        n2 = 2 ** math.ceil(math.log2(pts))
        assert int(n2 // 1e6) == int(pts // 1e6), tag  # the printed count: that power of two, truncated
        assert abs(bpp * n2 - vol) / vol < 0.01, (tag, bpp * n2, vol)
        assert abs(bpp * pts - vol) / vol < 0.05, (tag, bpp * pts, vol)
