"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every declared symbol, validates arguments with the
documented error codes before touching the device, and its host coefficient
tables agree with the independent oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2107_13500_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_13500_gb300 import build, pw
    build.build()
    return pw.load_library()


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(pw_[a-z0-9_]+)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "pw_advect" in names and "pw_make_coeffs" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_version_and_error_text(lib):
    from paper_2107_13500_gb300 import pw
    assert "sm_103a" in pw.version()


def test_make_coeffs_agrees_with_oracle(lib, oracle_lib):
    from paper_2107_13500_gb300 import pw
    for nz, dz, dens in ((64, synth.dz_stretched(64), True), (16, synth.dz_uniform(16, 20.0), False),
                         (1, synth.dz_uniform(1, 5.0), False), (2, synth.dz_stretched(2), True)):
        rho, rhon = synth.density_exponential(dz) if dens else (None, None)
        a = pw.make_coeffs(nz, 50.0, 35.0, dz, rho, rhon)
        b = oracle_lib.coeffs(nz, 50.0, 35.0, dz, rho, rhon)
        assert a.tcx == b["tcx"] and a.tcy == b["tcy"]
        for row, key in enumerate(("tzc1", "tzc2", "tzd1", "tzd2")):
            np.testing.assert_allclose(a.tz4[row], b[key], rtol=4e-16, atol=0)


def test_make_coeffs_validation(lib):
    from paper_2107_13500_gb300 import pw
    with pytest.raises(pw.PWError) as e:
        pw.make_coeffs(8, -1.0, 1.0, synth.dz_uniform(8, 1.0))
    assert e.value.code == pw.PW_EINVAL
    bad = synth.dz_uniform(8, 1.0)
    bad[5] = 0.0
    with pytest.raises(pw.PWError) as e:
        pw.make_coeffs(8, 1.0, 1.0, bad)
    assert e.value.code == pw.PW_EINVAL


def _call_advect(lib, dtype, ptrs, dims, split=None, coeffs=True):
    from paper_2107_13500_gb300 import pw
    c = pw.Coeffs(0.005, 0.005, 0x1000, 0x2000, 0x3000, 0x4000)
    vp = ctypes.c_void_p
    return lib.pw_advect(dtype, vp(ptrs[0]), vp(ptrs[1]), vp(ptrs[2]), ctypes.byref(c) if coeffs else None,
                         ctypes.byref(dims) if dims is not None else None, vp(split) if split else None,
                         vp(ptrs[3]), vp(ptrs[4]), vp(ptrs[5]), None)


def test_advect_validation_codes_without_device(lib):
    """Fake, never-dereferenced addresses: every case fails validation
    before any CUDA call, so no GPU is needed."""
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 30, 20, 5
    sy = pw.row_stride(nx, 8)
    sz = sy * (ny + 2)
    ext = nz * sz * 8
    base = 1 << 40
    ptrs = [base + n * ext for n in range(6)]
    good = pw.Dims(nx, ny, nz, 1, sy, sz)
    assert _call_advect(lib, pw.PW_F64, ptrs, None) == pw.PW_ENULL
    assert _call_advect(lib, pw.PW_F64, ptrs, good, coeffs=False) == pw.PW_ENULL
    assert _call_advect(lib, pw.PW_F64, [0] + ptrs[1:], good) == pw.PW_ENULL
    assert _call_advect(lib, 7, ptrs, good) == pw.PW_EINVAL
    assert _call_advect(lib, pw.PW_F64, ptrs, pw.Dims(nx, ny, nz, 2, sy, sz)) == pw.PW_EINVAL
    assert _call_advect(lib, pw.PW_F64, ptrs, pw.Dims(0, ny, nz, 1, sy, sz)) == pw.PW_EINVAL
    assert _call_advect(lib, pw.PW_F64, ptrs, pw.Dims(nx, ny, nz, 1, nx + 1, sz)) == pw.PW_EINVAL
    assert _call_advect(lib, pw.PW_F64, ptrs, pw.Dims(nx, ny, nz, 1, sy, sy)) == pw.PW_EINVAL
    assert _call_advect(lib, pw.PW_F64, ptrs, pw.Dims(nx, ny, nz, 1, sy + 1, (sy + 1) * (ny + 2))) == pw.PW_EINVAL
    assert _call_advect(lib, pw.PW_F64, [ptrs[0] + 8] + ptrs[1:], good) == pw.PW_EINVAL
    # an output overlapping an input, or another output
    assert _call_advect(lib, pw.PW_F64, ptrs[:3] + [ptrs[1] + 64, ptrs[4], ptrs[5]], good) == pw.PW_EALIAS
    assert _call_advect(lib, pw.PW_F64, ptrs[:4] + [ptrs[3], ptrs[5]], good) == pw.PW_EALIAS
    # split table only with PW_F32_SPLIT, and required there
    assert _call_advect(lib, pw.PW_F64, ptrs, good, split=0x5000) == pw.PW_EINVAL
    sy4 = pw.row_stride(nx, 4)
    d4 = pw.Dims(nx, ny, nz, 1, sy4, sy4 * (ny + 2))
    assert _call_advect(lib, pw.PW_F32_SPLIT, ptrs, d4) == pw.PW_ENULL
    assert b"pw_advect" in lib.pw_last_error()


def test_split_table_algebra(lib, oracle_lib):
    """Evaluating the mean/perturbation expansion with the table's entries
    (in FP64 here) reproduces the oracle on the full fields up to the float
    rounding of the table entries: the algebra loses no term."""
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 12, 10, 9
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    c = pw.make_coeffs(nz, 50.0, 40.0, dz, rho, rhon)
    co = oracle_lib.coeffs(nz, 50.0, 40.0, dz, rho, rhon)
    fu, fv, fw = synth.fields_iid(nx, ny, nz, seed=17, lo=-3, hi=3)
    means = [synth.uniform(18, s, nz, -8, 8) for s in range(3)]
    full = [f + m[:, None, None] for f, m in zip((fu, fv, fw), means)]
    ref = oracle_lib.advect(*full, co, nx, ny)
    T = pw.make_split_table(c, *means).astype(np.float64)
    u, v, w = fu, fv, fw
    su = np.zeros_like(u); sv = np.zeros_like(u); sw = np.zeros_like(u)
    for k in range(1, nz):
        t = T[k]
        top = k == nz - 1
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                a, b, cc = u[k, j, i - 1], u[k, j, i], u[k, j, i + 1]
                s = t[26] * (a - cc) * (t[0] + a + b + cc)
                a, cc = u[k, j - 1, i], u[k, j + 1, i]
                p = v[k, j - 1, i] + v[k, j - 1, i + 1]
                q = v[k, j, i] + v[k, j, i + 1]
                s += t[27] * (t[1] * (a - cc) + t[2] * (p - q) + a * p - cc * q)
                P = w[k - 1, j, i] + w[k - 1, j, i + 1]
                a = u[k - 1, j, i]
                s += t[3] + t[4] * (t[5] * P + t[6] * a + a * P)
                if not top:
                    Q = w[k, j, i] + w[k, j, i + 1]
                    cc = u[k + 1, j, i]
                    s -= t[7] * (t[8] * Q + t[9] * cc + cc * Q)
                su[k, j, i] = s
                a, b, cc = v[k, j - 1, i], v[k, j, i], v[k, j + 1, i]
                s = t[27] * (a - cc) * (t[10] + a + b + cc)
                a, cc = v[k, j, i - 1], v[k, j, i + 1]
                p = u[k, j, i - 1] + u[k, j + 1, i - 1]
                q = u[k, j, i] + u[k, j + 1, i]
                s += t[26] * (t[11] * (a - cc) + t[12] * (p - q) + a * p - cc * q)
                P = w[k - 1, j, i] + w[k - 1, j + 1, i]
                a = v[k - 1, j, i]
                s += t[13] + t[4] * (t[14] * P + t[6] * a + a * P)
                if not top:
                    Q = w[k, j, i] + w[k, j + 1, i]
                    cc = v[k + 1, j, i]
                    s -= t[7] * (t[15] * Q + t[9] * cc + cc * Q)
                sv[k, j, i] = s
                if not top:
                    a, cc = w[k, j, i - 1], w[k, j, i + 1]
                    p = u[k, j, i - 1] + u[k + 1, j, i - 1]
                    q = u[k, j, i] + u[k + 1, j, i]
                    s = t[26] * (t[16] * (p - q) + t[17] * (a - cc) + a * p - cc * q)
                    a, cc = w[k, j - 1, i], w[k, j + 1, i]
                    p = v[k, j - 1, i] + v[k + 1, j - 1, i]
                    q = v[k, j, i] + v[k + 1, j, i]
                    s += t[27] * (t[16] * (p - q) + t[18] * (a - cc) + a * p - cc * q)
                    a, b, cc = w[k - 1, j, i], w[k, j, i], w[k + 1, j, i]
                    s += t[19] + t[20] * ((a + b) * (t[21] + a) + t[22] * a)
                    s -= t[23] * ((b + cc) * (t[24] + cc) + t[25] * cc)
                    sw[k, j, i] = s
    for got, want in zip((su, sv, sw), ref):
        gi, wi = got[1:, 1:ny + 1, 1:nx + 1], want[1:, 1:ny + 1, 1:nx + 1]
        assert np.max(np.abs(gi - wi)) <= 1e-5 * np.max(np.abs(wi))


def test_batch_plan_validation_without_device(lib):
    """pw_make_batch_plan rejects bad requests before encoding anything."""
    import ctypes
    from paper_2107_13500_gb300 import pw
    assert lib.pw_batch_plan_bytes(96) > lib.pw_batch_plan_bytes(1) > 0
    assert lib.pw_variant_count(pw.PW_F32) == 8 and lib.pw_variant_count(pw.PW_F64_PAIRED) == 4
    assert lib.pw_variant_count(pw.PW_F64) == 2
    nbytes = lib.pw_batch_plan_bytes(2)
    raw = np.zeros(nbytes + 128, dtype=np.uint8)
    off = (-raw.ctypes.data) % 64
    plan = ctypes.c_void_p(raw.ctypes.data + off)
    doms = (pw.Domain * 2)()
    n = ctypes.c_longlong(0)
    assert lib.pw_make_batch_plan(pw.PW_F64, 2, doms, 2, plan, nbytes, ctypes.byref(n)) == pw.PW_EINVAL
    assert lib.pw_make_batch_plan(99, 2, doms, 0, plan, nbytes, ctypes.byref(n)) == pw.PW_EINVAL
    assert lib.pw_make_batch_plan(pw.PW_F32, 0, doms, 0, plan, nbytes, ctypes.byref(n)) == pw.PW_EINVAL
    assert lib.pw_make_batch_plan(pw.PW_F32, 2, doms, 7, plan, nbytes, ctypes.byref(n)) == pw.PW_EINVAL
    assert lib.pw_make_batch_plan(pw.PW_F32, 2, doms, 0, plan, nbytes - 1, ctypes.byref(n)) == pw.PW_EINVAL
    mis = ctypes.c_void_p(raw.ctypes.data + off + 8)
    assert lib.pw_make_batch_plan(pw.PW_F32, 2, doms, 0, mis, nbytes, ctypes.byref(n)) == pw.PW_EINVAL
    # zeroed domains: dims fail validation, naming the domain
    assert lib.pw_make_batch_plan(pw.PW_F32, 2, doms, 0, plan, nbytes, ctypes.byref(n)) == pw.PW_EINVAL
    assert b"domain" in lib.pw_last_error()
    assert lib.pw_advect_batched(pw.PW_F32, 0, None, 1, None) == pw.PW_ENULL
    assert lib.pw_advect_batched(pw.PW_F64, 2, plan, 1, None) == pw.PW_EINVAL
    assert lib.pw_advect_batched(99, 0, plan, 1, None) == pw.PW_EINVAL


def test_adjoint_validation_without_device(lib):
    import ctypes
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 12, 6, 4
    sy = pw.row_stride(nx, 8)
    d = pw.Dims(nx, ny, nz, 1, sy, sy * (ny + 2))
    c = pw.Coeffs(0.005, 0.005, 0x1000, 0x2000, 0x3000, 0x4000)
    ext = nz * sy * (ny + 2) * 8
    p = [ctypes.c_void_p((1 << 40) + k * ext) for k in range(9)]
    # the mean+perturbation form has no adjoint
    assert lib.pw_advect_adjoint(pw.PW_F32_SPLIT, *p[:3], ctypes.byref(c), ctypes.byref(d), *p[3:], 0,
                                 None) == pw.PW_EUNSUPPORTED
    alias = p[:6] + [p[0]] + p[7:]
    assert lib.pw_advect_adjoint(pw.PW_F64, *alias[:3], ctypes.byref(c), ctypes.byref(d), *alias[3:], 0,
                                 None) == pw.PW_EALIAS
    assert lib.pw_fold_periodic_halo(pw.PW_F64, None, ctypes.byref(d), None) == pw.PW_ENULL


def test_energy_weights_agree_with_oracle(lib, oracle_lib):
    """pw_make_energy_weights (host, library) against the oracle's own
    computation of the cell masses, on uniform, stretched and density grids."""
    from paper_2107_13500_gb300 import pw
    for nz, dz, dens in ((64, synth.dz_stretched(64), True), (16, synth.dz_uniform(16, 20.0), False),
                         (1, synth.dz_uniform(1, 5.0), False), (3, synth.dz_stretched(3), True)):
        rho, rhon = synth.density_exponential(dz) if dens else (None, None)
        a = pw.make_energy_weights(nz, dz, rho, rhon)
        b = oracle_lib.energy_weights(nz, dz, rho, rhon)
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=4e-16, atol=0)
    with pytest.raises(pw.PWError) as e:
        pw.make_energy_weights(4, np.array([0.0, 1.0, -1.0, 1.0]))
    assert e.value.code == pw.PW_EINVAL


def test_energy_budget_validation_without_device(lib):
    """pw_energy_budget rejects bad element sizes, mismatched domains, NULL
    and misaligned pointers and overlapping results before any launch."""
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 12, 6, 4
    sy8, sy4 = pw.row_stride(nx, 8), pw.row_stride(nx, 4)
    d8 = pw.Dims(nx, ny, nz, 1, sy8, sy8 * (ny + 2))
    d4 = pw.Dims(nx, ny, nz, 1, sy4, sy4 * (ny + 2))
    dbad = pw.Dims(nx + 1, ny, nz, 1, sy8, sy8 * (ny + 2))
    p = [ctypes.c_void_p((1 << 40) + k * (1 << 24)) for k in range(10)]
    wu, ww, lev, tot = p[6:10]
    B = ctypes.byref
    assert lib.pw_energy_budget(*p[:3], 2, B(d8), *p[3:6], 8, B(d8), wu, ww, lev, tot, None) == pw.PW_EINVAL
    assert lib.pw_energy_budget(*p[:3], 8, B(d8), *p[3:6], 4, B(dbad), wu, ww, lev, tot, None) == pw.PW_EINVAL
    assert lib.pw_energy_budget(*p[:3], 8, B(d8), *p[3:6], 4, B(d4), None, ww, lev, tot, None) == pw.PW_ENULL
    assert lib.pw_energy_budget(None, *p[1:3], 8, B(d8), *p[3:6], 8, B(d8), wu, ww, lev, tot, None) == pw.PW_ENULL
    mis = ctypes.c_void_p((1 << 40) + 4)
    assert lib.pw_energy_budget(mis, *p[1:3], 8, B(d8), *p[3:6], 8, B(d8), wu, ww, lev, tot, None) == pw.PW_EINVAL
    assert lib.pw_energy_budget(*p[:3], 8, B(d8), *p[3:6], 8, B(d8), wu, ww, lev,
                                ctypes.c_void_p(lev.value + 8), None) == pw.PW_EALIAS
