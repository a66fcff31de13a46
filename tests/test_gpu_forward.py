"""GPU parity of pw_advect against the FP64 CPU oracle, through the C ABI.

Inputs come from the shared seeded generators; the oracle runs on the same
numpy arrays the GPU receives. Sizes span several tiles with ragged edges,
the edge cases of the method (nz = 1, 2, 3; one-column domains), the full
16.8M-point workload, and guard-band canaries around every output.
"""
import numpy as np
import pytest

from helpers import check_mode, compare_f32, compare_paired, interior, to_device, to_numpy_f64
from paper_2107_13500_gb300 import synth

pytestmark = pytest.mark.gpu

F64_MODES = ["f64", "paired"]


@pytest.fixture(scope="module")
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_13500_gb300 import build, pw
    build.build()
    pw.load_library()
    return torch


def _run(gpu, mode, u, v, w, nx, ny, nz, dx, dy, dz, rho=None, rhon=None, oracle_lib=None, aligned=True):
    from paper_2107_13500_gb300 import pw
    torch = gpu
    co = oracle_lib.coeffs(nz, dx, dy, dz, rho, rhon)
    (so, ab) = oracle_lib.advect(u, v, w, co, nx, ny, want_abs=True, nthreads=8)
    mb = oracle_lib.monomial_scale(u, v, w, co, nx, ny, nthreads=8) if mode == "paired" else None
    c = pw.make_coeffs(nz, dx, dy, dz, rho, rhon).to_device()
    du, dv, dw = (to_device(f, nx, torch.float64, aligned=aligned) for f in (u, v, w))
    out = pw.advect(du, dv, dw, c, nx, ny, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    g = [to_numpy_f64(t, u.shape[2], nx) for t in out]
    return g, so, (ab, mb)


@pytest.mark.parametrize("mode", F64_MODES)
def test_small_iid_config(gpu, oracle_lib, mode):
    """64^3 periodic, i.i.d. U[-10,10] winds, dx = dy = 50 m, dz = 20 m."""
    cfg = synth.config_small_iid()
    u, v, w = cfg["fields"]()
    g, o, a = _run(gpu, mode, u, v, w, cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"],
                   oracle_lib=oracle_lib)
    check_mode(mode, g, o, *a, cfg["nx"], cfg["ny"])


@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("mode", F64_MODES)
@pytest.mark.parametrize("shape", [(37, 13, 5), (33, 9, 7), (100, 17, 11), (31, 7, 3)])
def test_ragged_stretched_density(gpu, oracle_lib, mode, shape, aligned):
    """Sizes that leave partial tiles in x and y; stretched grid with density;
    both the 16-byte-aligned interior layout and the general one."""
    nx, ny, nz = shape
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=nx * 7 + ny)
    g, o, a = _run(gpu, mode, u, v, w, nx, ny, nz, 40.0, 60.0, dz, rho, rhon, oracle_lib, aligned)
    check_mode(mode, g, o, *a, nx, ny)


@pytest.mark.parametrize("dy", [50.0, 45.0])
@pytest.mark.parametrize("case", ["equal", "density", "one_level_differs"])
@pytest.mark.parametrize("mode", F64_MODES)
def test_f64_vertical_coefficient_paths(gpu, oracle_lib, mode, case, dy):
    """Both FP64-class kernels share one coefficient product between a
    level's two vertical face terms when every level's lower and upper
    coefficients are equal (no density stratification), and scale each face
    sum on its own otherwise; the paired kernel shares that form only where
    tcx = tcy as well (dx = dy), and then also takes one coefficient product
    for an output's x and y parts. Every combination, and a grid equal on
    every level but one (which must take the general form), against the
    oracle on the same coefficients at the mode's own scale."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 70, 19, 13
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz) if case == "density" else (None, None)
    c = pw.make_coeffs(nz, 50.0, dy, dz, rho, rhon)
    if case == "one_level_differs":
        c.tz4[1, 6] *= 1.5  # tzc2 of one level
        c.tz4[3, 4] *= 0.5  # tzd2 of another
    lv = slice(1, nz - 1)  # levels with an upper flux
    pairs_equal = np.array_equal(c.tz4[0, lv], c.tz4[1, lv]) and np.array_equal(c.tz4[2, lv], c.tz4[3, lv])
    assert pairs_equal == (case == "equal")
    co = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in c.as_dict().items()}
    c.to_device()
    u, v, w = synth.fields_iid(nx, ny, nz, seed=91)
    (so, ab) = oracle_lib.advect(u, v, w, co, nx, ny, want_abs=True, nthreads=8)
    mb = oracle_lib.monomial_scale(u, v, w, co, nx, ny, nthreads=8) if mode == "paired" else None
    du, dv, dw = (to_device(f, nx, torch.float64) for f in (u, v, w))
    out = pw.advect(du, dv, dw, c, nx, ny, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    g = [to_numpy_f64(t, u.shape[2], nx) for t in out]
    check_mode(mode, g, so, ab, mb, nx, ny)


@pytest.mark.parametrize("mode", F64_MODES)
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 1), (5, 4, 2), (1, 9, 4), (9, 1, 4), (64, 8, 3)])
def test_degenerate_shapes(gpu, oracle_lib, mode, shape):
    """nz = 1 (nothing computed), nz = 2 (only the top level), one-column
    domains in x or y."""
    nx, ny, nz = shape
    dz = synth.dz_uniform(nz, 20.0)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=99)
    g, o, a = _run(gpu, mode, u, v, w, nx, ny, nz, 50.0, 50.0, dz, oracle_lib=oracle_lib)
    check_mode(mode, g, o, *a, nx, ny)
    if nz == 1:
        for s in g:
            assert np.all(interior(s, nx, ny) == 0.0)


@pytest.mark.parametrize("mode", F64_MODES)
@pytest.mark.parametrize("shape", [(40, 8, 300), (17, 5, 129)])
def test_tall_columns_many_level_chunks(gpu, oracle_lib, mode, shape):
    """Few tiles and many levels: the launch cuts each column into many short
    level chunks (up to 64), so most chunk boundaries, with their re-read
    neighbour levels, fall inside the domain."""
    nx, ny, nz = shape
    dz = synth.dz_stretched(nz, 10.0, 1.01)
    rho, rhon = synth.density_exponential(dz)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=nz)
    g, o, a = _run(gpu, mode, u, v, w, nx, ny, nz, 50.0, 50.0, dz, rho, rhon, oracle_lib=oracle_lib)
    check_mode(mode, g, o, *a, nx, ny)


@pytest.mark.parametrize("mode", F64_MODES)
def test_integer_inputs_bit_exact(gpu, oracle_lib, mode):
    """Integer winds, dyadic coefficients: no operation of either side
    rounds, so the GPU must equal the oracle bit for bit."""
    nx, ny, nz = 45, 21, 9
    u, v, w = synth.fields_integer(nx, ny, nz, seed=3)
    g, o, a = _run(gpu, mode, u, v, w, nx, ny, nz, 0.25, 0.5, synth.dz_uniform(nz, 0.5), oracle_lib=oracle_lib)
    for gi, oi in zip(g, o):
        np.testing.assert_array_equal(interior(gi, nx, ny), interior(oi, nx, ny))


@pytest.mark.parametrize("mode", F64_MODES)
def test_full_16m_modes_config(gpu, oracle_lib, mode):
    """The 512 x 512 x 64 workload (smooth winds, mean 5 m/s, stretched grid)
    in the launch configuration the benchmark times, compared point by point."""
    cfg = synth.config_16m_modes()
    u, v, w = cfg["fields"]()
    g, o, a = _run(gpu, mode, u, v, w, cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"],
                   oracle_lib=oracle_lib)
    worst = check_mode(mode, g, o, *a, cfg["nx"], cfg["ny"])
    print("worst:", worst)


@pytest.mark.parametrize("mode", F64_MODES)
def test_full_134m_iid_config(gpu, oracle_lib, mode):
    """1024 x 1024 x 128 with i.i.d. U[-10,10] winds (134M points, 1.1 GB per
    field), compared point by point."""
    cfg = synth.config_134m_iid()
    u, v, w = cfg["fields"]()
    g, o, a = _run(gpu, mode, u, v, w, cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"],
                   oracle_lib=oracle_lib)
    del u, v, w
    print("worst:", check_mode(mode, g, o, *a, cfg["nx"], cfg["ny"]))


@pytest.mark.parametrize("e", [40, -40])
def test_paired_inputs_scaled_by_powers_of_two(gpu, oracle_lib, e):
    """The paired path carries FP32's exponent range. Winds scaled by 2^40
    and 2^-40 (magnitudes up to 2^43.4 and down to the smallest i.i.d.
    values near 2^-50) on a stretched grid with density, ragged tiles:
    every point stays within the paired tolerance of the oracle evaluated
    on the same scaled winds."""
    nx, ny, nz = 53, 19, 14
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    u, v, w = (f * 2.0 ** e for f in synth.fields_iid(nx, ny, nz, seed=40 + e))
    g, o, a = _run(gpu, "paired", u, v, w, nx, ny, nz, 50.0, 50.0, dz, rho, rhon, oracle_lib)
    print("worst (err/M, err/A, normwise):", compare_paired(g, o, *a, nx, ny))


def _run_f32(gpu, oracle_lib, u, v, w, nx, ny, nz, dx, dy, dz, rho=None, rhon=None, aligned=True):
    """PW_F32 on float copies of u, v, w; the oracle on the double fields."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    co = oracle_lib.coeffs(nz, dx, dy, dz, rho, rhon)
    so = oracle_lib.advect(u, v, w, co, nx, ny, nthreads=8)
    mb = oracle_lib.monomial_scale(u, v, w, co, nx, ny, nthreads=8)
    c = pw.make_coeffs(nz, dx, dy, dz, rho, rhon).to_device()
    du, dv, dw = (to_device(f, nx, torch.float32, aligned=aligned) for f in (u, v, w))
    out = pw.advect(du, dv, dw, c, nx, ny, mode="f32")
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    g = [to_numpy_f64(t.double(), u.shape[2], nx) for t in out]
    return compare_f32(g, so, mb, nx, ny)


@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("shape", [(37, 13, 5), (100, 17, 11), (131, 9, 7), (5, 4, 2)])
def test_f32_full_fields_ragged(gpu, oracle_lib, shape, aligned):
    """Plain FP32 (float winds, float arithmetic) against the FP64 oracle on
    the original double winds: ragged tiles, stretched grid with density,
    both interior alignments."""
    nx, ny, nz = shape
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=nx + 3 * ny)
    print("worst (err/M, max rel, rms rel):",
          _run_f32(gpu, oracle_lib, u, v, w, nx, ny, nz, 40.0, 60.0, dz, rho, rhon, aligned))


@pytest.mark.parametrize("cfg_name", ["config_small_iid", "config_16m_modes"])
def test_f32_full_fields_configs(gpu, oracle_lib, cfg_name):
    """Plain FP32 on the 64^3 i.i.d. and the 512 x 512 x 64 smooth-wind
    workloads, point by point against the oracle."""
    cfg = getattr(synth, cfg_name)()
    u, v, w = cfg["fields"]()
    print("worst (err/M, max rel, rms rel):",
          _run_f32(gpu, oracle_lib, u, v, w, cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"]))


@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("mode", F64_MODES)
def test_guard_bands_and_halo_untouched(gpu, oracle_lib, mode, aligned):
    """Outputs live inside a larger buffer filled with a NaN canary: after the
    call every cell outside the interior (halo, row padding, guard bands
    before and after) still holds the canary bit pattern."""
    import torch
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 35, 10, 6
    u, v, w = synth.fields_iid(nx, ny, nz, seed=12)
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    du, dv, dw = (to_device(f, nx, torch.float64, aligned=aligned) for f in (u, v, w))
    shape = du.shape
    n = du.numel()
    guard = 4096 + (1 if aligned else 0)
    canary = torch.tensor([0x7FF4DEADBEEF0001], dtype=torch.int64).view(torch.float64)
    bufs, outs = [], []
    for _ in range(3):
        b = torch.empty(n + 2 * guard, dtype=torch.float64, device="cuda")
        b.view(torch.int64).fill_(int(canary.view(torch.int64)))
        bufs.append(b)
        outs.append(b[guard:guard + n].view(shape))
    pw.advect(du, dv, dw, c, nx, ny, mode=mode, out=tuple(outs))
    torch.cuda.synchronize()
    for b in bufs:
        bits = b.view(torch.int64).cpu().numpy()
        mask = np.ones(bits.shape, dtype=bool)
        inner = mask[guard:guard + n].reshape(shape)
        inner[:, 1:ny + 1, 1:nx + 1] = False
        assert np.all(bits[mask] == int(canary.view(torch.int64))), "a cell outside the interior was written"


def test_host_chunked_back_to_back_calls(gpu):
    """Consecutive asynchronous advect_host calls on one pipeline overlap
    (two staging sets in turn: the next call's input copies and kernels run
    while the previous call's outputs drain); each call's outputs must still
    equal a device call on its own inputs once pipeline.synchronize() has
    returned."""
    import torch
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 96, 40, 24
    dz = synth.dz_stretched(nz)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz).to_device()
    pipe = pw.HostPipeline(nx, ny, nz)
    calls = []
    for seed in (31, 32, 33, 34, 35):
        fields = synth.fields_modes(nx, ny, nz, 50.0, 50.0, dz, seed=seed)
        host = [pw.pinned_field(nx, ny, nz) for _ in range(3)]
        for h, a in zip(host, fields):
            h[:, :, : nx + 2] = torch.from_numpy(a[:, :, : nx + 2])
        out = tuple(pw.pinned_field(nx, ny, nz) for _ in range(3))
        pw.advect_host(*host, c, nx, ny, mode="paired", out_host=out, pipeline=pipe, nchunks=6, wait=False)
        calls.append((fields, out))
    pipe.synchronize()
    for fields, out in calls:
        want = pw.advect(*[pw.field_from_numpy(a, nx) for a in fields], c, nx, ny, mode="paired")
        torch.cuda.synchronize()
        for g, w_ in zip(out, want):
            assert torch.equal(g[:, 1:ny + 1, 1:nx + 1], w_.cpu()[:, 1:ny + 1, 1:nx + 1])


def test_periodic_halo_fill_matches_numpy(gpu):
    """pw_fill_periodic_halo against numpy's wrap padding of the interior."""
    import torch
    from paper_2107_13500_gb300 import pw
    for dt, npdt in ((torch.float64, np.float64), (torch.float32, np.float32)):
        nx, ny, nz = 29, 11, 4
        f = synth.empty_field(nx, ny, nz, npdt)
        f[:, 1:ny + 1, 1:nx + 1] = synth.uniform(5, 0, nx * ny * nz, -1, 1).reshape(nz, ny, nx)
        t = pw.empty_field(nx, ny, nz, dt)
        t[:, :, : f.shape[2]] = torch.from_numpy(f)[:, :, : t.shape[2]]
        pw.fill_periodic_halo(t, nx, ny)
        torch.cuda.synchronize()
        got = t.cpu().numpy()[:, :, : nx + 2]
        want = np.pad(f[:, 1:ny + 1, 1:nx + 1], ((0, 0), (1, 1), (1, 1)), mode="wrap")
        np.testing.assert_array_equal(got, want)


def test_api_rejects_bad_arguments_on_device(gpu):
    """Aliased outputs, misaligned pointers and bad strides fail validation
    with the documented codes, and nothing is launched."""
    import torch
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 16, 8, 4
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    u, v, w = (pw.empty_field(nx, ny, nz) for _ in range(3))
    su, sv, sw = (pw.empty_field(nx, ny, nz) for _ in range(3))
    with pytest.raises(pw.PWError) as e:
        pw.advect(u, v, w, c, nx, ny, mode="f64", out=(u, sv, sw))
    assert e.value.code == pw.PW_EALIAS
    with pytest.raises(pw.PWError) as e:
        pw.advect(u, v, w, c, nx, ny, mode="f64", out=(su, su, sw))
    assert e.value.code == pw.PW_EALIAS
    # u, v, w share one set of TMA box coordinates: a u at another address
    # phase (mod 16 bytes) than v and w is rejected
    other = pw.empty_field(nx, ny, nz, aligned=False)
    assert other.data_ptr() % 16 != v.data_ptr() % 16
    with pytest.raises(pw.PWError) as e:
        pw.advect(other, v, w, c, nx, ny, mode="f64", out=(su, sv, sw))
    assert e.value.code == pw.PW_EINVAL
    assert pw.device_status() == 0


def test_bounded_wait_gives_up_and_device_stays_usable(gpu, oracle_lib):
    """A kernel waiting on a barrier nothing completes returns after its
    limit with a timeout status; the device then still runs pw_advect
    correctly and the status word is clear again."""
    from paper_2107_13500_gb300 import pw
    import time
    t0 = time.perf_counter()
    assert pw.selftest_bounded_wait(20000) == pw.PW_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert pw.device_status() == 0
    nx, ny, nz = 20, 9, 5
    u, v, w = synth.fields_iid(nx, ny, nz, seed=5)
    g, o, a = _run(gpu, "paired", u, v, w, nx, ny, nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0),
                   oracle_lib=oracle_lib)
    check_mode("paired", g, o, *a, nx, ny)


@pytest.mark.parametrize("mode", ["paired", "f32", "f64"])
@pytest.mark.parametrize("nchunks", [1, 3, 8, 1000])
def test_host_chunked_matches_device_call(gpu, mode, nchunks):
    """pw_advect_host_chunked (slabs of levels, transfers overlapped with
    compute) gives exactly what pw_advect gives on the same data already on
    the device; the host outputs' halo rows stay untouched."""
    import torch
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 70, 37, 9
    dt = torch.float32 if mode == "f32" else torch.float64
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_stretched(nz)).to_device()
    fields = synth.fields_modes(nx, ny, nz, 50.0, 50.0, synth.dz_stretched(nz), seed=21)
    host = [pw.pinned_field(nx, ny, nz, dt) for _ in range(3)]
    for h, a in zip(host, fields):
        h[:, :, : nx + 2] = torch.from_numpy(a[:, :, : nx + 2]).to(dt)
    out = tuple(pw.pinned_field(nx, ny, nz, dt).fill_(7.0) for _ in range(3))
    got = pw.advect_host(*host, c, nx, ny, mode=mode, out_host=out, nchunks=nchunks)
    dev = [pw.field_from_numpy(a, nx, dt) for a in fields]
    want = pw.advect(*dev, c, nx, ny, mode=mode)
    torch.cuda.synchronize()
    for g, w_ in zip(got, want):
        assert torch.equal(g[:, 1:ny + 1, 1:nx + 1], w_.cpu()[:, 1:ny + 1, 1:nx + 1])
        assert float((g[:, 0, :] - 7.0).abs().sum()) == 0.0 and float((g[:, ny + 1, :] - 7.0).abs().sum()) == 0.0


@pytest.mark.parametrize("mode", ["f64", "paired", "f32", "split"])
def test_homogeneity_bit_exact(gpu, mode):
    """The map is a quadratic form, so F(2x) = 4 F(x). Scaling by a power of
    two is exact through every product, FMA, pair split and join, level mean
    and split-table constant, so each mode must give 4 F(x) bit for bit
    (stretched grid with density, ragged tiles, several k-chunks)."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 77, 29, 23
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz, rho, rhon).to_device()
    fields = synth.fields_modes(nx, ny, nz, 50.0, 50.0, dz, seed=13)

    def evaluate(scale):
        if mode in ("f64", "paired"):
            x = [to_device(scale * f, nx, torch.float64) for f in fields]
            return pw.advect(*x, c, nx, ny, mode=mode)
        if mode == "f32":
            x = [to_device(scale * f, nx, torch.float32) for f in fields]
            return pw.advect(*x, c, nx, ny, mode="f32")
        x = [to_device(scale * f, nx, torch.float64) for f in fields]
        fp, means = zip(*(pw.split_field(t, nx, ny) for t in x))
        table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
        return pw.advect(*fp, c, nx, ny, mode="split", split_table=table)

    one, two = evaluate(1.0), evaluate(2.0)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    for a, b in zip(one, two):
        a, b = a[:, :, : nx + 2], b[:, :, : nx + 2]
        assert torch.isfinite(a).all()
        assert torch.equal(4 * a, b)
