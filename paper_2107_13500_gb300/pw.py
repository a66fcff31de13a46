"""Python binding of the C ABI in include/pw.h (argument marshalling only).

Every computation runs in ``libpw.so``'s CUDA kernels; this module only
turns torch tensors into pointers, sizes and a stream handle. PyTorch
supplies device memory and streams. There is no CPU fallback: if the
library is not built, or no GPU is present, calls raise.

Fields are torch tensors of shape ``(nz, ny + 2, sy)`` indexed ``[k, j, i]``
(x fastest, one halo cell in x and y, rows padded so that each starts on a
32-byte boundary); :func:`empty_field` allocates that layout.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

PW_OK = 0
PW_EINVAL = -1
PW_ENULL = -2
PW_EALIAS = -3
PW_EUNSUPPORTED = -4
PW_ECUDA = -5
PW_ETIMEOUT = -6

PW_F64 = 0
PW_F32_SPLIT = 1
PW_F64_PAIRED = 2
PW_F32 = 3
PW_SPLIT_NCOEF = 32

MODES = {"f64": PW_F64, "paired": PW_F64_PAIRED, "split": PW_F32_SPLIT, "f32": PW_F32}

# Algorithmic HBM traffic per point: read u, v, w once, write su, sv, sw once.
BYTES_PER_POINT = {"f64": 48, "paired": 48, "split": 24, "f32": 24}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpw.so")


class PWError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Dims(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("halo", ctypes.c_int),
                ("sy", ctypes.c_longlong), ("sz", ctypes.c_longlong)]


class Coeffs(ctypes.Structure):
    _fields_ = [("tcx", ctypes.c_double), ("tcy", ctypes.c_double),
                ("tzc1", ctypes.c_void_p), ("tzc2", ctypes.c_void_p),
                ("tzd1", ctypes.c_void_p), ("tzd2", ctypes.c_void_p)]


class Domain(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("su", ctypes.c_void_p), ("sv", ctypes.c_void_p), ("sw", ctypes.c_void_p),
                ("dims", Dims), ("coeffs", Coeffs), ("split", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def load_library(path: str | None = None):
    """Load libpw.so (built by ``build.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libpw.so not found at {p}: run paper_2107_13500_gb300.build.build() "
                               "(nvcc, sm_103a) first; there is no CPU fallback")
        lib = ctypes.CDLL(p)
        vp = ctypes.c_void_p
        lib.pw_last_error.restype = ctypes.c_char_p
        lib.pw_version.restype = ctypes.c_char_p
        lib.pw_make_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
        lib.pw_fill_periodic_halo.argtypes = [ctypes.c_int, vp, ctypes.POINTER(Dims), vp]
        lib.pw_advect.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.POINTER(Coeffs), ctypes.POINTER(Dims), vp,
                                  vp, vp, vp, vp]
        lib.pw_make_split_table.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp,
                                            _fp]
        lib.pw_split_field.argtypes = [vp, ctypes.POINTER(Dims), vp, ctypes.POINTER(Dims), vp, vp]
        lib.pw_device_status.argtypes = [ctypes.POINTER(ctypes.c_int), vp]
        for name in ("pw_make_coeffs", "pw_fill_periodic_halo", "pw_advect", "pw_make_split_table",
                     "pw_split_field", "pw_device_status"):
            getattr(lib, name).restype = ctypes.c_int
        lib.pw_advect_adjoint.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.POINTER(Coeffs),
                                          ctypes.POINTER(Dims), vp, vp, vp, vp, vp, vp, ctypes.c_int, vp]
        lib.pw_advect_adjoint.restype = ctypes.c_int
        lib.pw_fold_periodic_halo.argtypes = [ctypes.c_int, vp, ctypes.POINTER(Dims), vp]
        lib.pw_fold_periodic_halo.restype = ctypes.c_int
        lib.pw_batch_plan_bytes.argtypes = [ctypes.c_int]
        lib.pw_batch_plan_bytes.restype = ctypes.c_size_t
        lib.pw_variant_count.argtypes = [ctypes.c_int]
        lib.pw_variant_count.restype = ctypes.c_int
        lib.pw_make_batch_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Domain), ctypes.c_int, vp,
                                           ctypes.c_size_t, ctypes.POINTER(ctypes.c_longlong)]
        lib.pw_make_batch_plan.restype = ctypes.c_int
        lib.pw_advect_batched.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_longlong, vp]
        lib.pw_advect_batched.restype = ctypes.c_int
        lib.pw_advect_host_chunked.argtypes = [ctypes.c_int] + [vp] * 12 + [ctypes.POINTER(Coeffs),
                                                                          ctypes.POINTER(Dims), vp, ctypes.c_int,
                                                                          vp, vp, vp]
        lib.pw_advect_host_chunked.restype = ctypes.c_int
        lib.pw_selftest_bounded_wait.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_int), vp]
        lib.pw_selftest_bounded_wait.restype = ctypes.c_int
        lib.pw_make_energy_weights.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.pw_make_energy_weights.restype = ctypes.c_int
        lib.pw_energy_budget.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(Dims), vp, vp, vp, ctypes.c_int,
                                         ctypes.POINTER(Dims), vp, vp, vp, vp, vp]
        lib.pw_energy_budget.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc):
    if rc != PW_OK:
        raise PWError(rc, load_library().pw_last_error().decode())


def version() -> str:
    return load_library().pw_version().decode()


# ---------------------------------------------------------------- layouts

def row_stride(nx: int, elem_bytes: int) -> int:
    per = 32 // elem_bytes
    return ((nx + 2 + per - 1) // per) * per


def _aligned_zeros(shape, dtype, device, lead):
    """Zeros of `shape` (C order) whose first element sits `lead` elements
    past a 16-byte boundary (torch's allocator returns 512-byte blocks)."""
    import torch
    n = 1
    for d in shape:
        n *= d
    flat = torch.zeros(n + lead, dtype=dtype, device=device)
    return flat[lead:].view(shape)


def interior_lead(elem_bytes: int) -> int:
    """Elements between a 16-byte boundary and the halo cell i = 0 that put
    the first interior cell (i = 1) on the boundary: 1 double, 3 floats."""
    return 16 // elem_bytes - 1


def empty_field(nx, ny, nz, dtype=None, device="cuda", aligned=True):
    """Zeroed field in the library's layout. aligned=True places i = 1 of
    every row on a 16-byte boundary, which selects the vectorised kernels."""
    import torch
    dtype = dtype or torch.float64
    es = torch.empty((), dtype=dtype).element_size()
    shape = (nz, ny + 2, row_stride(nx, es))
    return _aligned_zeros(shape, dtype, device, interior_lead(es) if aligned else 0)


def field_like(t):
    """Zeroed tensor with t's shape, dtype, device and 16-byte phase."""
    es = t.element_size()
    return _aligned_zeros(tuple(t.shape), t.dtype, t.device, (t.data_ptr() % 16) // es)


def field_from_numpy(a, nx, dtype=None, device="cuda", aligned=True):
    """Copy a numpy field [nz][ny+2][>= nx+2] into a new device field."""
    import torch
    dtype = dtype or torch.float64
    t = empty_field(nx, a.shape[1] - 2, a.shape[0], dtype, device, aligned)
    src = torch.from_numpy(np.ascontiguousarray(a[:, :, : nx + 2]))
    t[:, :, : nx + 2].copy_(src.to(dtype))
    return t


def dims_of(t, nx: int, ny: int) -> Dims:
    if t.dim() != 3 or t.stride(2) != 1:
        raise ValueError("fields must be 3-D (nz, ny+2, sy) tensors with x contiguous")
    nz = t.shape[0]
    if t.shape[1] != ny + 2 or t.shape[2] < nx + 2:
        raise ValueError(f"field shape {tuple(t.shape)} does not hold a {nx}x{ny} interior with halo")
    return Dims(nx, ny, nz, 1, t.stride(1), t.stride(0))


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- coefficients

@dataclass
class Coefficients:
    """Host FP64 coefficients (from pw_make_coeffs) and their device copies."""
    nz: int
    tcx: float
    tcy: float
    tz4: np.ndarray          # (4, nz): tzc1, tzc2, tzd1, tzd2
    dev: object = None        # torch (4, nz) float64 on the GPU
    f32_table: object = None  # device table for PW_F32 (all means 0)

    def zero_mean_table(self, device="cuda"):
        """Device table for PW_F32: the split table with every mean 0."""
        import torch
        if self.f32_table is None or str(self.f32_table.device) != str(torch.device(device)):
            z = np.zeros(self.nz)
            self.f32_table = torch.from_numpy(make_split_table(self, z, z, z)).to(device)
        return self.f32_table

    def to_device(self, device="cuda"):
        import torch
        if self.dev is None or str(self.dev.device) != str(torch.device(device)):
            self.dev = torch.from_numpy(self.tz4.copy()).to(device)
        return self

    def c_struct(self) -> Coeffs:
        if self.dev is None:
            self.to_device()
        d = self.dev
        return Coeffs(self.tcx, self.tcy, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr())

    def as_dict(self):
        return dict(tcx=self.tcx, tcy=self.tcy, tzc1=self.tz4[0], tzc2=self.tz4[1], tzd1=self.tz4[2],
                    tzd2=self.tz4[3])


def make_coeffs(nz, dx, dy, dz, rho=None, rhon=None) -> Coefficients:
    lib = load_library()
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    if dz.shape != (nz,):
        raise ValueError("dz must have nz entries")
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    rhon = None if rhon is None else np.ascontiguousarray(rhon, dtype=np.float64)
    tc = np.zeros(2)
    tz = np.zeros((4, nz))
    _check(lib.pw_make_coeffs(nz, float(dx), float(dy), dz.ctypes.data_as(_dp),
                              None if rho is None else rho.ctypes.data_as(_dp),
                              None if rhon is None else rhon.ctypes.data_as(_dp),
                              tc.ctypes.data_as(_dp), tz.ctypes.data_as(_dp)))
    return Coefficients(nz, float(tc[0]), float(tc[1]), tz)


def make_split_table(coeffs: Coefficients, ubar, vbar, wbar) -> np.ndarray:
    lib = load_library()
    nz = coeffs.nz
    ub, vb, wb = (np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(nz)) for m in (ubar, vbar, wbar))
    tz = np.ascontiguousarray(coeffs.tz4)
    out = np.zeros((nz, PW_SPLIT_NCOEF), dtype=np.float32)
    _check(lib.pw_make_split_table(nz, coeffs.tcx, coeffs.tcy, tz.ctypes.data_as(_dp), ub.ctypes.data_as(_dp),
                                   vb.ctypes.data_as(_dp), wb.ctypes.data_as(_dp), out.ctypes.data_as(_fp)))
    return out


# ---------------------------------------------------------------- compute calls

def fill_periodic_halo(f, nx, ny, stream=None):
    import torch
    dt = PW_F32_SPLIT if f.dtype == torch.float32 else PW_F64
    d = dims_of(f, nx, ny)
    _check(load_library().pw_fill_periodic_halo(dt, ctypes.c_void_p(f.data_ptr()), ctypes.byref(d),
                                                _stream_handle(stream)))
    return f


def advect(u, v, w, coeffs: Coefficients, nx, ny, mode="paired", split_table=None, out=None, stream=None):
    """Source terms (su, sv, sw) of u, v, w.

    mode: "f64" (native FP64), "paired" (FP64 in/out, paired-FP32
    arithmetic), "split" (float perturbations; ``split_table`` is the
    device table from :func:`make_split_table`) or "f32" (float full fields).
    """
    lib = load_library()
    dt = MODES[mode]
    if mode == "f32" and split_table is None:
        split_table = coeffs.zero_mean_table(u.device)
    d = dims_of(u, nx, ny)
    for t in (v, w):
        if t.shape != u.shape or t.stride() != u.stride() or t.dtype != u.dtype:
            raise ValueError("u, v, w must share shape, strides and dtype")
    if out is None:
        out = tuple(field_like(u) for _ in range(3))
    su, sv, sw = out
    for t in out:
        if t.shape != u.shape or t.stride() != u.stride() or t.dtype != u.dtype:
            raise ValueError("outputs must match the inputs' layout")
    c = coeffs.c_struct()
    sp = None if split_table is None else ctypes.c_void_p(split_table.data_ptr())
    _check(lib.pw_advect(dt, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                         ctypes.c_void_p(w.data_ptr()), ctypes.byref(c), ctypes.byref(d), sp,
                         ctypes.c_void_p(su.data_ptr()), ctypes.c_void_p(sv.data_ptr()),
                         ctypes.c_void_p(sw.data_ptr()), _stream_handle(stream)))
    return su, sv, sw


class HostPipeline:
    """Device staging buffers and three streams (host->device, compute,
    device->host) for advect_host: reuse one across calls on same-shaped
    fields. It holds `depth` sets of the six staging fields and uses them in
    turn, so that consecutive calls overlap: a call's input copies wait only
    until the kernels of the call that last used its set have finished, and
    its kernels only until that call's outputs have left the device. With two
    sets, one call's outputs stream out while the next call's inputs stream in
    and its slabs compute."""

    def __init__(self, nx, ny, nz, dtype=None, device="cuda", depth=2):
        import torch
        dtype = dtype or torch.float64
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.sets = [[empty_field(nx, ny, nz, dtype, device) for _ in range(6)] for _ in range(depth)]
        self.dev = self.sets[0]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(3)]
        self.compute_done = [None] * depth  # per set: the last call's kernels done (its inputs are free)
        self.d2h_done = [None] * depth      # per set: the last call's outputs copied out (its outputs are free)
        self.done = None                     # the latest call's outputs are in host memory
        self.calls = 0

    def wait(self, stream=None):
        """Order `stream` (default: the current stream) after the latest
        call's outputs reaching host memory."""
        import torch
        if self.done is not None:
            (stream or torch.cuda.current_stream()).wait_event(self.done)

    def synchronize(self):
        """Block the host until the latest call's outputs are in host memory."""
        if self.done is not None:
            self.done.synchronize()


def pinned_field(nx, ny, nz, dtype=None):
    """Pinned host tensor in the library's layout (for advect_host)."""
    import torch
    dtype = dtype or torch.float64
    es = torch.empty((), dtype=dtype).element_size()
    return torch.zeros((nz, ny + 2, row_stride(nx, es)), dtype=dtype).pin_memory()


def advect_host(u_h, v_h, w_h, coeffs: Coefficients, nx, ny, mode="paired", out_host=None, pipeline=None,
                nchunks=8, split_table=None, wait=True):
    """pw_advect on pinned host fields with chunked, overlapped transfers
    (pw_advect_host_chunked). Returns the host outputs. The call's kernels
    are ordered after the caller's current stream (coefficients, tables).
    With wait=True it returns once the outputs have arrived. With
    wait=False it returns after enqueueing: on a caller's `pipeline`, the
    outputs are in host memory once pipeline.done has completed
    (pipeline.wait(stream), pipeline.synchronize()), and later calls on the
    pipeline overlap this one; without one, the caller's current stream is
    ordered after their arrival. The host inputs are read when the input
    copies run, which may be before earlier work on the caller's stream: they
    must be complete in host memory when the call is made."""
    import torch
    lib = load_library()
    dt = MODES[mode]
    nz = u_h.shape[0]
    d = dims_of(u_h, nx, ny)
    own = pipeline is None
    if own:
        pipeline = HostPipeline(nx, ny, nz, u_h.dtype, depth=1)
    if out_host is None:
        out_host = tuple(torch.zeros_like(u_h).pin_memory() for _ in range(3))
    if mode == "f32" and split_table is None:
        split_table = coeffs.zero_mean_table()
    k = pipeline.calls % len(pipeline.sets)
    dev = pipeline.sets[k]
    for t in dev:
        if t.stride() != u_h.stride():
            raise ValueError("host and device fields must share strides")
    c = coeffs.c_struct()
    vp = ctypes.c_void_p
    sh, sc, sd = pipeline.streams
    cur = torch.cuda.current_stream()
    # input copies: this set's staging inputs must be free (its last kernels done)
    if pipeline.compute_done[k] is not None:
        sh.wait_event(pipeline.compute_done[k])
    # kernels: the caller's device work (coefficients, tables), and this
    # set's staging outputs drained by its last call
    sc.wait_stream(cur)
    if pipeline.d2h_done[k] is not None:
        sc.wait_event(pipeline.d2h_done[k])
    sd.wait_stream(cur)
    _check(lib.pw_advect_host_chunked(dt, *(vp(t.data_ptr()) for t in (u_h, v_h, w_h) + tuple(out_host)),
                                      *(vp(t.data_ptr()) for t in dev), ctypes.byref(c), ctypes.byref(d),
                                      None if split_table is None else vp(split_table.data_ptr()), int(nchunks),
                                      vp(sh.cuda_stream), vp(sc.cuda_stream), vp(sd.cuda_stream)))
    pipeline.compute_done[k] = torch.cuda.Event()
    pipeline.compute_done[k].record(sc)
    pipeline.d2h_done[k] = torch.cuda.Event()
    pipeline.d2h_done[k].record(sd)
    # the output copies follow every kernel and input copy of the call
    pipeline.done = pipeline.d2h_done[k]
    pipeline.calls += 1
    if wait:
        sd.synchronize()
    elif own:
        cur.wait_event(pipeline.done)
    return out_host


def split_field(f, nx, ny, out=None, mean=None, stream=None):
    """(fp, mean): float perturbation field and per-level FP64 means of f."""
    import torch
    lib = load_library()
    df = dims_of(f, nx, ny)
    fp = out if out is not None else empty_field(nx, ny, f.shape[0], torch.float32, f.device)
    dp = dims_of(fp, nx, ny)
    m = mean if mean is not None else torch.empty(f.shape[0], dtype=torch.float64, device=f.device)
    _check(lib.pw_split_field(ctypes.c_void_p(f.data_ptr()), ctypes.byref(df), ctypes.c_void_p(fp.data_ptr()),
                              ctypes.byref(dp), ctypes.c_void_p(m.data_ptr()), _stream_handle(stream)))
    return fp, m


def selftest_bounded_wait(limit_us=20000, stream=None) -> int:
    """Run the bounded-wait self-test; returns the status it left
    (PW_ETIMEOUT when waits are bounded)."""
    st = ctypes.c_int(0)
    _check(load_library().pw_selftest_bounded_wait(int(limit_us), ctypes.byref(st), _stream_handle(stream)))
    return st.value


def device_status(stream=None) -> int:
    st = ctypes.c_int(0)
    _check(load_library().pw_device_status(ctypes.byref(st), _stream_handle(stream)))
    return st.value


def advect_adjoint(u, v, w, coeffs: Coefficients, nx, ny, gsu, gsv, gsw, mode="f64", out=None, accumulate=False,
                   stream=None):
    """(gu, gv, gw) = J(u, v, w)^T (gsu, gsv, gsw) on every cell the forward
    reads (halo included). mode "f64" (double, native FP64), "paired"
    (double, paired-FP32 arithmetic) or "f32" (float). Cotangents must share
    u's layout (shape, strides, 16-byte phase)."""
    lib = load_library()
    dt = {"f64": PW_F64, "paired": PW_F64_PAIRED, "f32": PW_F32}[mode]
    d = dims_of(u, nx, ny)
    ins = (u, v, w, gsu, gsv, gsw)
    for t in ins[1:]:
        if t.shape != u.shape or t.stride() != u.stride() or t.dtype != u.dtype:
            raise ValueError("u, v, w and the cotangents must share shape, strides and dtype")
    if out is None:
        out = tuple(field_like(u) for _ in range(3))
    gu, gv, gw = out
    c = coeffs.c_struct()
    vp = ctypes.c_void_p
    _check(lib.pw_advect_adjoint(dt, *(vp(t.data_ptr()) for t in ins[:3]), ctypes.byref(c), ctypes.byref(d),
                                 *(vp(t.data_ptr()) for t in ins[3:]), vp(gu.data_ptr()), vp(gv.data_ptr()),
                                 vp(gw.data_ptr()), 1 if accumulate else 0, _stream_handle(stream)))
    return gu, gv, gw


def make_energy_weights(nz, dz, rho=None, rhon=None):
    """(wu, ww): host masses of the u/v cells and of the w cells per level
    (pw_make_energy_weights)."""
    lib = load_library()
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    if dz.shape != (nz,):
        raise ValueError("dz must have nz entries")
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    rhon = None if rhon is None else np.ascontiguousarray(rhon, dtype=np.float64)
    wu, ww = np.zeros(nz), np.zeros(nz)
    _check(lib.pw_make_energy_weights(nz, dz.ctypes.data_as(_dp), None if rho is None else rho.ctypes.data_as(_dp),
                                      None if rhon is None else rhon.ctypes.data_as(_dp), wu.ctypes.data_as(_dp),
                                      ww.ctypes.data_as(_dp)))
    return wu, ww


def energy_budget(u, v, w, su, sv, sw, nx, ny, wu, ww, stream=None):
    """(totals, level_sums) of pw_energy_budget as device float64 tensors:
    totals = [sum wu u su, sum wu v sv, sum ww w sw, and the same sums of
    |summands|]; level_sums (nz, 6) the unweighted per-level sums. wu, ww
    are device float64 tensors of nz entries. Winds and tendencies may each
    be float or double."""
    import torch
    lib = load_library()
    dw, ds = dims_of(u, nx, ny), dims_of(su, nx, ny)
    for t in (v, w):
        if t.stride() != u.stride() or t.dtype != u.dtype:
            raise ValueError("u, v, w must share strides and dtype")
    for t in (sv, sw):
        if t.stride() != su.stride() or t.dtype != su.dtype:
            raise ValueError("su, sv, sw must share strides and dtype")
    nz = u.shape[0]
    level = torch.empty((nz, 6), dtype=torch.float64, device=u.device)
    totals = torch.empty(6, dtype=torch.float64, device=u.device)
    vp = ctypes.c_void_p
    _check(lib.pw_energy_budget(vp(u.data_ptr()), vp(v.data_ptr()), vp(w.data_ptr()), u.element_size(),
                                ctypes.byref(dw), vp(su.data_ptr()), vp(sv.data_ptr()), vp(sw.data_ptr()),
                                su.element_size(), ctypes.byref(ds), vp(wu.data_ptr()), vp(ww.data_ptr()),
                                vp(level.data_ptr()), vp(totals.data_ptr()), _stream_handle(stream)))
    return totals, level


def fold_periodic_halo(g, nx, ny, stream=None):
    """Transpose of fill_periodic_halo, in place: halo gradients are added to
    the interior cells they were copied from, and the halo is zeroed."""
    import torch
    dt = PW_F32 if g.dtype == torch.float32 else PW_F64
    d = dims_of(g, nx, ny)
    _check(load_library().pw_fold_periodic_halo(dt, ctypes.c_void_p(g.data_ptr()), ctypes.byref(d),
                                                _stream_handle(stream)))
    return g


# ---------------------------------------------------------------- batches

def variant_count(mode) -> int:
    return int(load_library().pw_variant_count(MODES[mode]))


class Batch:
    """Many independent domains evaluated by one persistent launch.

    domains: sequence of dicts with keys u, v, w (inputs), su, sv, sw
    (outputs; allocated with field_like(u) if absent), nx, ny, coeffs
    (Coefficients) and, for "split", split_table. mode "f64", "paired",
    "f32" or "split". The plan (TMA descriptors, work table and work-queue counter) is
    built on the host and copied once into a device buffer owned here.
    """

    def __init__(self, domains, mode="paired", variant=0):
        import torch
        lib = load_library()
        self.mode, self.variant = mode, int(variant)
        self.dt = MODES[mode]
        self.domains = []
        cs = (Domain * len(domains))()
        for n, d in enumerate(domains):
            u = d["u"]
            outs = tuple(d.get(k) if d.get(k) is not None else field_like(u) for k in ("su", "sv", "sw"))
            dd = dict(d, su=outs[0], sv=outs[1], sw=outs[2])
            split = d.get("split_table")
            if mode == "f32" and split is None:
                split = d["coeffs"].zero_mean_table(u.device)
                dd["split_table"] = split
            self.domains.append(dd)
            cstruct = d["coeffs"].c_struct()
            cs[n] = Domain(u.data_ptr(), d["v"].data_ptr(), d["w"].data_ptr(), outs[0].data_ptr(),
                           outs[1].data_ptr(), outs[2].data_ptr(), dims_of(u, d["nx"], d["ny"]), cstruct,
                           split.data_ptr() if split is not None else None)
        nbytes = int(lib.pw_batch_plan_bytes(len(domains)))
        raw = np.zeros(nbytes + 64, dtype=np.uint8)
        off = (-raw.ctypes.data) % 64
        host = raw[off:off + nbytes]
        n_items = ctypes.c_longlong(0)
        _check(lib.pw_make_batch_plan(self.dt, len(domains), cs, self.variant, ctypes.c_void_p(host.ctypes.data),
                                      nbytes, ctypes.byref(n_items)))
        self.n_items = int(n_items.value)
        self.plan_host = host
        self.plan_dev = torch.from_numpy(host.copy()).to(domains[0]["u"].device)
        self.points = sum(d["u"].shape[0] * d["nx"] * d["ny"] for d in domains)

    def run(self, stream=None):
        _check(load_library().pw_advect_batched(self.dt, self.variant, ctypes.c_void_p(self.plan_dev.data_ptr()),
                                                self.n_items, _stream_handle(stream)))

    def outputs(self):
        return [(d["su"], d["sv"], d["sw"]) for d in self.domains]
