"""GPU checks of the batched persistent launch (pw_advect_batched): every
domain of a batch equals its own pw_advect call bit for bit (same per-point
arithmetic, any tile variant), the 96-domain uneven workload, a CUDA graph of
50 batched evaluations, plan/variant mismatch detection, and the autotuner.
"""
import numpy as np
import pytest

from helpers import TOL_F32_ELEM, TOL_F64, TOL_PAIRED, TOL_SPLIT_ELEM, to_device
from paper_2107_13500_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_13500_gb300 import build, pw
    build.build()
    pw.load_library()
    return torch


def _domains(torch, sizes, mode, seed=10, aligned=True, mixed=False):
    """One domain per (nx, ny, nz): stretched grid, smooth winds; FP32 modes
    get float fields (split: perturbations and the level table). `mixed`
    gives every third domain dy = 40 m and every third, from the second, a
    density profile, so one batch holds domains on both arithmetic forms of
    the kernels (shared coefficient products, or each term on its own)."""
    from paper_2107_13500_gb300 import pw
    doms = []
    for n, (nx, ny, nz) in enumerate(sizes):
        dz = synth.dz_stretched(nz)
        dy = 40.0 if mixed and n % 3 == 0 else 50.0
        rho, rhon = synth.density_exponential(dz) if mixed and n % 3 == 1 else (None, None)
        c = pw.make_coeffs(nz, 50.0, dy, dz, rho, rhon).to_device()
        u, v, w = synth.fields_modes(nx, ny, nz, 50.0, dy, dz, seed=seed + n, n_modes=3)
        if mode in ("paired", "f64"):
            f = [to_device(a, nx, torch.float64, aligned=aligned) for a in (u, v, w)]
            d = dict(u=f[0], v=f[1], w=f[2], nx=nx, ny=ny, coeffs=c)
        elif mode == "f32":
            f = [to_device(a, nx, torch.float32, aligned=aligned) for a in (u, v, w)]
            d = dict(u=f[0], v=f[1], w=f[2], nx=nx, ny=ny, coeffs=c)
        else:
            f64 = [to_device(a, nx, torch.float64) for a in (u, v, w)]
            fp, means = zip(*(pw.split_field(t, nx, ny, out=pw.empty_field(nx, ny, nz, torch.float32,
                                                                           aligned=aligned)) for t in f64))
            table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
            d = dict(u=fp[0], v=fp[1], w=fp[2], nx=nx, ny=ny, coeffs=c, split_table=table)
        doms.append(d)
    return doms


def _one_by_one(pw, doms, mode):
    return [pw.advect(d["u"], d["v"], d["w"], d["coeffs"], d["nx"], d["ny"], mode=mode,
                      split_table=d.get("split_table")) for d in doms]


SMALL = [(37, 13, 5), (64, 8, 3), (130, 33, 17), (5, 70, 2), (96, 96, 40), (1, 1, 1), (200, 9, 9)]


@pytest.mark.parametrize("mode", ["f64", "paired", "f32", "split"])
@pytest.mark.parametrize("aligned", [True, False])
def test_batched_equals_single(gpu, mode, aligned):
    from paper_2107_13500_gb300 import pw
    torch = gpu
    doms = _domains(torch, SMALL, mode, aligned=aligned, mixed=True)
    ref = _one_by_one(pw, doms, mode)
    for v in range(pw.variant_count(mode)):
        b = pw.Batch(doms, mode, v)
        b.run()
        torch.cuda.synchronize()
        assert pw.device_status() == 0
        for (nx, ny, nz), r, o in zip(SMALL, ref, b.outputs()):
            for rr, oo in zip(r, o):
                assert torch.equal(rr[:, 1:ny + 1, 1:nx + 1], oo[:, 1:ny + 1, 1:nx + 1]), (mode, v, nx, ny, nz)


@pytest.mark.parametrize("mode", ["f64", "paired", "f32", "split"])
def test_batched_96_uneven_domains(gpu, oracle_lib, mode):
    """The batched workload: 96 domains, x, y uniform in 32..384, z in 32..128
    (seed 4), stretched grids. Every domain equals its single launch; four of
    them are also checked against the oracle, at the tolerance of the mode
    (native FP64: the strict scale A; paired: the monomial scale M; FP32:
    32 * 2^-24 * M; split: 64 * 2^-24 * A on the mean + perturbation
    magnitudes)."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    sizes = synth.batched_domain_sizes(96, seed=4)
    doms = _domains(torch, sizes, mode, seed=100)
    b = pw.Batch(doms, mode, 0)
    b.run()
    ref = _one_by_one(pw, doms, mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    for (nx, ny, nz), r, o in zip(sizes, ref, b.outputs()):
        for rr, oo in zip(r, o):
            assert torch.equal(rr[:, 1:ny + 1, 1:nx + 1], oo[:, 1:ny + 1, 1:nx + 1])
    worst = 0.0
    for n in (0, 17, 50, 95):
        nx, ny, nz = sizes[n]
        dz = synth.dz_stretched(nz)
        u, v, w = synth.fields_modes(nx, ny, nz, 50.0, 50.0, dz, seed=100 + n, n_modes=3)
        co = oracle_lib.coeffs(nz, 50.0, 50.0, dz)
        want, ab = oracle_lib.advect(u, v, w, co, nx, ny, want_abs=True, nthreads=8)
        if mode == "split":
            means = [f[:, 1:ny + 1, 1:nx + 1].mean(axis=(1, 2)) for f in (u, v, w)]
            mags = [np.abs(m)[:, None, None] + np.abs(f - m[:, None, None]) for f, m in zip((u, v, w), means)]
            _, ab = oracle_lib.advect(*mags, co, nx, ny, want_abs=True, nthreads=8)
            tol = TOL_SPLIT_ELEM
        elif mode == "f64":
            tol = TOL_F64
        else:
            ab = oracle_lib.monomial_scale(u, v, w, co, nx, ny, nthreads=8)
            tol = TOL_PAIRED if mode == "paired" else TOL_F32_ELEM
        for got, wn, a in zip(b.outputs()[n], want, ab):
            g = got.double().cpu().numpy()[:, 1:ny + 1, 1:nx + 1]
            wi, ai = wn[:, 1:ny + 1, 1:nx + 1], a[:, 1:ny + 1, 1:nx + 1]
            err = np.abs(g - wi)
            assert np.all(err <= tol * ai)
            worst = max(worst, float(np.max(err / np.maximum(ai, 1e-300))))
    print(f"{mode}: worst err/scale {worst:.3e} (tolerance {tol:.3e})")


def test_batched_cuda_graph_50_evaluations(gpu):
    """50 batched tendency evaluations captured in one CUDA graph and
    replayed: each replay leaves the same outputs as a plain launch."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    doms = _domains(torch, SMALL, "f32")
    b = pw.Batch(doms, "f32", 0)
    b.run()
    torch.cuda.synchronize()
    ref = [tuple(t.clone() for t in o) for o in b.outputs()]
    for o in b.outputs():
        for t in o:
            t.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        b.run(stream=s)  # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            for _ in range(50):
                b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for o in b.outputs():
        for t in o:
            t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    for r, o in zip(ref, b.outputs()):
        for rr, oo in zip(r, o):
            assert torch.equal(rr, oo)


def test_batched_plan_variant_mismatch_reported(gpu):
    """A plan launched with another variant than it was built for is refused
    by the kernel (status PW_EINVAL), without touching outputs."""
    import ctypes
    from paper_2107_13500_gb300 import pw
    torch = gpu
    doms = _domains(torch, SMALL[:3], "f32")
    b = pw.Batch(doms, "f32", 1)
    rc = pw.load_library().pw_advect_batched(pw.PW_F32, 2, ctypes.c_void_p(b.plan_dev.data_ptr()), b.n_items,
                                             pw._stream_handle())
    assert rc == pw.PW_OK
    torch.cuda.synchronize()
    assert pw.device_status() == pw.PW_EINVAL
    for o in b.outputs():
        for t in o:
            assert float(t.abs().sum()) == 0.0


def test_autotuner_caches_per_shape_class(gpu, tmp_path):
    from paper_2107_13500_gb300 import autotune, pw
    torch = gpu
    doms = _domains(torch, SMALL[:4], "split")
    path = str(tmp_path / "tune.json")
    v, rec = autotune.tune(doms, "split", cache_path=path, reps=2)
    nv = pw.variant_count("split")
    assert nv == 8
    assert 0 <= v < nv and len(rec["ms"]) == nv
    v2, rec2 = autotune.tune(doms, "split", cache_path=path, reps=2)
    assert v2 == v and rec2 == rec
