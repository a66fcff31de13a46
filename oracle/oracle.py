"""ctypes wrapper and build step for the C oracle in ``pw_oracle.c``.

TEST INFRASTRUCTURE ONLY (see ``pw_oracle.h``). Arrays are numpy float64 in
the layout ``f[k, j, i]`` of shape ``(nz, ny + 2, sy)`` (x fastest, one halo
cell in x and y, rows possibly padded to ``sy >= nx + 2``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pw_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libpw_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    deps = [_SRC, os.path.join(_HERE, "pw_oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            lib.pwo_coeffs.restype = ctypes.c_int
            lib.pwo_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp,
                                       _dp, _dp, _dp, _dp, _dp, _dp]
            lib.pwo_advect.restype = None
            lib.pwo_advect.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_longlong] * 2 + [_dp] * 3
                                       + [ctypes.c_double] * 2 + [_dp] * 4 + [_dp] * 6 + [ctypes.c_int])
            lib.pwo_advect_adjoint.restype = None
            lib.pwo_advect_adjoint.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_longlong] * 2 + [_dp] * 3
                                               + [ctypes.c_double] * 2 + [_dp] * 4 + [_dp] * 6)
            lib.pwo_monomial_scale.restype = None
            lib.pwo_monomial_scale.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_longlong] * 2 + [_dp] * 3
                                               + [ctypes.c_double] * 2 + [_dp] * 4 + [_dp] * 3 + [ctypes.c_int])
            lib.pwo_energy_weights.restype = ctypes.c_int
            lib.pwo_energy_weights.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.pwo_energy_budget.restype = None
            lib.pwo_energy_budget.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_longlong] * 2 + [_dp] * 6
                                              + [_dp] * 3)
            lib.pwo_flops_per_column.restype = ctypes.c_longlong
            lib.pwo_flops_per_column.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def coeffs(nz, dx, dy, dz, rho=None, rhon=None):
    """Return dict(tcx, tcy, tzc1, tzc2, tzd1, tzd2) (numpy float64, length nz)."""
    lib = _load()
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    assert dz.shape == (nz,)
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    rhon = None if rhon is None else np.ascontiguousarray(rhon, dtype=np.float64)
    tcx = ctypes.c_double()
    tcy = ctypes.c_double()
    out = [np.zeros(nz) for _ in range(4)]
    rc = lib.pwo_coeffs(nz, dx, dy, _ptr(dz), _ptr(rho), _ptr(rhon), ctypes.byref(tcx),
                        ctypes.byref(tcy), *[_ptr(o) for o in out])
    if rc != 0:
        raise ValueError("pwo_coeffs: bad arguments")
    return dict(tcx=tcx.value, tcy=tcy.value, tzc1=out[0], tzc2=out[1], tzd1=out[2], tzd2=out[3])


def _dims(u, nx, ny):
    nz, nyh, sy = u.shape
    assert nyh == ny + 2 and sy >= nx + 2
    return nz, sy, sy * nyh


def advect(u, v, w, c, nx, ny, want_abs=False, nthreads=1, out=None):
    """Source terms (su, sv, sw) [, (asu, asv, asw)] for fields u, v, w.

    With want_abs the second triple is the per-point error scale: the sum of
    |c||q||a+b| over the face terms c*q*(a+b) of each output. Outputs have
    the inputs' shape; only the interior is written, the halo of freshly
    allocated outputs is zero.
    """
    lib = _load()
    nz, sy, sz = _dims(u, nx, ny)
    for f in (u, v, w):
        assert f.shape == u.shape and f.dtype == np.float64 and f.flags.c_contiguous
    if out is None:
        su, sv, sw = (np.zeros_like(u) for _ in range(3))
    else:
        su, sv, sw = out
    ab = [np.zeros_like(u) for _ in range(3)] if want_abs else [None] * 3
    lib.pwo_advect(nx, ny, nz, sy, sz, _ptr(u), _ptr(v), _ptr(w), c["tcx"], c["tcy"],
                   _ptr(c["tzc1"]), _ptr(c["tzc2"]), _ptr(c["tzd1"]), _ptr(c["tzd2"]),
                   _ptr(su), _ptr(sv), _ptr(sw), _ptr(ab[0]), _ptr(ab[1]), _ptr(ab[2]), int(nthreads))
    if want_abs:
        return (su, sv, sw), tuple(ab)
    return su, sv, sw


def monomial_scale(u, v, w, c, nx, ny, nthreads=1):
    """Per-point monomial error scale (msu, msv, msw): each face term
    c*q*(a+b) counted as |c||q|(|a|+|b|) (interior; halo zero)."""
    lib = _load()
    nz, sy, sz = _dims(u, nx, ny)
    out = [np.zeros_like(u) for _ in range(3)]
    lib.pwo_monomial_scale(nx, ny, nz, sy, sz, _ptr(u), _ptr(v), _ptr(w), c["tcx"], c["tcy"],
                           _ptr(c["tzc1"]), _ptr(c["tzc2"]), _ptr(c["tzd1"]), _ptr(c["tzd2"]),
                           _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), int(nthreads))
    return tuple(out)


def energy_weights(nz, dz, rho=None, rhon=None):
    """(wu, ww): mass of the u/v cells and of the w cells per level."""
    lib = _load()
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    rhon = None if rhon is None else np.ascontiguousarray(rhon, dtype=np.float64)
    wu, ww = np.zeros(nz), np.zeros(nz)
    if lib.pwo_energy_weights(nz, _ptr(dz), _ptr(rho), _ptr(rhon), _ptr(wu), _ptr(ww)) != 0:
        raise ValueError("pwo_energy_weights: bad arguments")
    return wu, ww


def energy_budget(u, v, w, su, sv, sw, wu, ww, nx, ny):
    """[sum wu u su, sum wu v sv, sum ww w sw, and the three sums of the
    absolute summands] over the interior."""
    lib = _load()
    nz, sy, sz = _dims(u, nx, ny)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, w, su, sv, sw)]
    for a in arrs:
        assert a.shape == u.shape
    out = np.zeros(6)
    lib.pwo_energy_budget(nx, ny, nz, sy, sz, *[_ptr(a) for a in arrs], _ptr(np.ascontiguousarray(wu)),
                          _ptr(np.ascontiguousarray(ww)), _ptr(out))
    return out


def advect_adjoint(u, v, w, c, nx, ny, gsu, gsv, gsw):
    """Return (gu, gv, gw) = J(u,v,w)^T (gsu, gsv, gsw); halo cells included."""
    lib = _load()
    nz, sy, sz = _dims(u, nx, ny)
    gu, gv, gw = (np.zeros_like(u) for _ in range(3))
    lib.pwo_advect_adjoint(nx, ny, nz, sy, sz, _ptr(u), _ptr(v), _ptr(w), c["tcx"], c["tcy"],
                           _ptr(c["tzc1"]), _ptr(c["tzc2"]), _ptr(c["tzd1"]), _ptr(c["tzd2"]),
                           _ptr(np.ascontiguousarray(gsu)), _ptr(np.ascontiguousarray(gsv)),
                           _ptr(np.ascontiguousarray(gsw)), _ptr(gu), _ptr(gv), _ptr(gw))
    return gu, gv, gw


def flops_per_column(nz: int) -> int:
    return int(_load().pwo_flops_per_column(nz))
