"""pw_advect_batched_noalloc: the batched evaluation for callers that cannot
allocate device memory (real-time loops that must not call cudaMalloc, which
can synchronise the device; plug-ins inside a host program that owns every
device allocation; a device whose memory another allocator has reserved). It
keeps the plan in a fixed device array inside the library instead of a
caller-allocated buffer.

Checked through the C ABI against pw_advect_batched, on consecutive calls
with different plans (the shared array must be refreshed each time), and
for the domain-count limit. This file is collected last on purpose.
"""
import ctypes

import pytest

from paper_2107_13500_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_13500_gb300 import build, pw
    build.build()
    lib = pw.load_library()
    lib.pw_advect_batched_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                              ctypes.c_longlong, ctypes.c_void_p]
    lib.pw_advect_batched_noalloc.restype = ctypes.c_int
    lib.pw_noalloc_last_error.restype = ctypes.c_char_p
    return torch, pw, lib


def _domains(torch, pw, sizes, mode, seed):
    dt = torch.float64 if mode == "paired" else torch.float32
    doms = []
    for n, (nx, ny, nz) in enumerate(sizes):
        c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_stretched(nz)).to_device()
        f = []
        for s in range(3):
            a = synth.empty_field(nx, ny, nz)
            a[:, :, : nx + 2] = synth.uniform(seed + n, s, nz * (ny + 2) * (nx + 2), -10, 10).reshape(
                nz, ny + 2, nx + 2)
            f.append(pw.field_from_numpy(a, nx, dt))
        doms.append(dict(u=f[0], v=f[1], w=f[2], nx=nx, ny=ny, coeffs=c))
    return doms


def _noalloc(lib, pw, batch):
    return lib.pw_advect_batched_noalloc(batch.dt, batch.variant, ctypes.c_void_p(batch.plan_host.ctypes.data),
                                         batch.plan_host.nbytes, batch.n_items, pw._stream_handle())


def test_noalloc_matches_batched_on_consecutive_calls(env):
    torch, pw, lib = env
    plans = [("f32", [(40, 12, 9), (7, 30, 3), (130, 5, 20)], 1),
             ("paired", [(33, 17, 6), (64, 8, 11)], 0)]
    batches, refs = [], []
    for mode, sizes, variant in plans:
        b = pw.Batch(_domains(torch, pw, sizes, mode, seed=300 + len(sizes)), mode, variant)
        b.run()  # the existing entry point, plan in a caller-owned device buffer
        torch.cuda.synchronize()
        refs.append([tuple(t.clone() for t in o) for o in b.outputs()])
        batches.append(b)
    assert pw.device_status() == 0
    # call 1 (FP32 plan), call 2 (paired plan), call 3 (the FP32 plan again)
    for n in (0, 1, 0):
        b = batches[n]
        for o in b.outputs():
            for t in o:
                t.zero_()
        rc = _noalloc(lib, pw, b)
        assert rc == pw.PW_OK, lib.pw_noalloc_last_error()
        torch.cuda.synchronize()
        assert pw.device_status() == 0
        for r, o in zip(refs[n], b.outputs()):
            for rr, oo in zip(r, o):
                assert torch.equal(rr, oo)


def test_noalloc_rejects_plans_beyond_its_array(env):
    torch, pw, lib = env
    one = _domains(torch, pw, [(16, 8, 4)], "f32", seed=400)[0]
    limit = 256
    b = pw.Batch([one] * (limit + 1), "f32", 0)
    rc = _noalloc(lib, pw, b)
    assert rc == pw.PW_EINVAL
    assert b"at most 256" in lib.pw_noalloc_last_error()
