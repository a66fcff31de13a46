"""GPU checks of the FP32 mean+perturbation path (PW_F32_SPLIT) against the
FP64 oracle on the original FP64 fields, and of pw_split_field.

Tolerance (derived): every float operation of the split form rounds a
quantity built from the level means and the perturbations, so its error is
at most 2^-24 of a product of |U(k)| + |u'|-type magnitudes. Summing over
the terms, |gpu - oracle| <= 64 * 2^-24 * A' per point, where A' is the
oracle's sum of absolute product terms evaluated on the nonnegative fields
|U(k)| + |u'| (likewise v, w). A' >= A; the two differ where a full wind
value is near zero while its level mean is not, which is exactly where the
split form rounds mean-sized quantities.
"""
import numpy as np
import pytest

from helpers import TOL_SPLIT_ELEM, interior, to_device
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


def _split_run(torch, u, v, w, nx, ny, nz, dx, dy, dz, rho=None, rhon=None, aligned=True):
    from paper_2107_13500_gb300 import pw
    c = pw.make_coeffs(nz, dx, dy, dz, rho, rhon).to_device()
    dev = [to_device(f, nx, torch.float64) for f in (u, v, w)]
    fp, means = zip(*(pw.split_field(t, nx, ny, out=pw.empty_field(nx, ny, nz, torch.float32, aligned=aligned))
                      for t in dev))
    table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    out = pw.advect(*fp, c, nx, ny, mode="split", split_table=table)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    return [t.double().cpu().numpy() for t in out], [m.cpu().numpy() for m in means], fp


def _check(gpu_out, ref, ab, nx, ny):
    stats = {}
    for name, g, o, a in zip(("su", "sv", "sw"), gpu_out, ref, ab):
        gi, oi, ai = interior(g, nx, ny), interior(o, nx, ny), interior(a, nx, ny)
        err = np.abs(gi - oi)
        assert np.all(np.isfinite(gi))
        assert np.all(err <= TOL_SPLIT_ELEM * ai), f"{name}: max err/A {np.max(err / np.maximum(ai, 1e-300)):.3e}"
        mo = np.max(np.abs(oi))
        stats[name] = dict(max_rel=float(np.max(err) / mo) if mo else 0.0,
                           rms_rel=float(np.sqrt(np.mean(err ** 2)) / max(np.sqrt(np.mean(oi ** 2)), 1e-300)))
    return stats


def split_scale(oracle_lib, fields, means, co, nx, ny):
    """A' of the module docstring: absolute product terms on |mean| + |perturbation|."""
    mags = [np.abs(m)[:, None, None] + np.abs(f - m[:, None, None]) for f, m in zip(fields, means)]
    _, ab = oracle_lib.advect(*mags, co, nx, ny, want_abs=True, nthreads=8)
    return ab


def _case(gpu, oracle_lib, u, v, w, nx, ny, nz, dx, dy, dz, rho=None, rhon=None, aligned=True):
    co = oracle_lib.coeffs(nz, dx, dy, dz, rho, rhon)
    ref = oracle_lib.advect(u, v, w, co, nx, ny, nthreads=8)
    g, means, _ = _split_run(gpu, u, v, w, nx, ny, nz, dx, dy, dz, rho, rhon, aligned)
    ab = split_scale(oracle_lib, (u, v, w), means, co, nx, ny)
    return _check(g, ref, ab, nx, ny)


def test_split_small_iid(gpu, oracle_lib):
    cfg = synth.config_small_iid()
    u, v, w = cfg["fields"]()
    print(_case(gpu, oracle_lib, u, v, w, cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"]))


@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("shape", [(37, 13, 5), (100, 17, 11), (31, 7, 3), (1, 1, 2), (5, 3, 1), (66, 9, 6),
                                   (129, 5, 4), (40, 8, 150)])
def test_split_ragged_modes_density(gpu, oracle_lib, shape, aligned):
    """Smooth winds with a 5 m/s mean (where the split matters), stretched
    grid with density, partial tiles and strips, degenerate heights, both
    interior alignments."""
    nx, ny, nz = shape
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    u, v, w = synth.fields_modes(nx, ny, nz, 50.0, 50.0, dz, seed=nx + ny)
    _case(gpu, oracle_lib, u, v, w, nx, ny, nz, 50.0, 50.0, dz, rho, rhon, aligned)


@pytest.mark.parametrize("aligned", [True, False])
def test_split_guard_bands_and_halo_untouched(gpu, aligned):
    """float outputs inside NaN-canary buffers: nothing outside the interior
    is written, for the vector (aligned) and scalar store paths."""
    import torch
    from paper_2107_13500_gb300 import pw
    nx, ny, nz = 70, 6, 5
    u, v, w = synth.fields_modes(nx, ny, nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0), seed=4)
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    dev = [to_device(f, nx, torch.float64) for f in (u, v, w)]
    fp, means = zip(*(pw.split_field(t, nx, ny, out=pw.empty_field(nx, ny, nz, torch.float32, aligned=aligned))
                      for t in dev))
    table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    shape, n = fp[0].shape, fp[0].numel()
    guard = 2048 + (3 if aligned else 0)
    canary = 0x7FC0BEEF
    bufs, outs = [], []
    for _ in range(3):
        b = torch.empty(n + 2 * guard, dtype=torch.float32, device="cuda")
        b.view(torch.int32).fill_(canary)
        bufs.append(b)
        outs.append(b[guard:guard + n].view(shape))
    pw.advect(*fp, c, nx, ny, mode="split", split_table=table, out=tuple(outs))
    torch.cuda.synchronize()
    for b in bufs:
        bits = b.view(torch.int32).cpu().numpy()
        mask = np.ones(bits.shape, dtype=bool)
        mask[guard:guard + n].reshape(shape)[:, 1:ny + 1, 1:nx + 1] = False
        assert np.all(bits[mask] == canary)


def test_split_field_means_and_perturbations(gpu):
    """pw_split_field: level means of the interior and float perturbations
    on every cell, halo included. The means are summed in paired FP32 (each
    double split into a float pair of 48 significant bits, pairs added with
    TwoSum): each of the at most n_add additions on a value's path (its
    thread's columns of a band of at most 16 rows, 128 threads to a band;
    the warp tree; the 4 warps; a lane's share of the bands; the tree over
    the lanes; the join) errs by at most 2^-47 of the magnitudes summed so
    far, so |mean - exact| <= n_add 2^-47 mean|f|."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    for nx, ny, nz in ((70, 33, 6), (512, 512, 4)):
        u, _, _ = synth.fields_modes(nx, ny, nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0), seed=8)
        t = to_device(u, nx, torch.float64)
        fp, mean = pw.split_field(t, nx, ny)
        torch.cuda.synchronize()
        m = mean.cpu().numpy()
        inner = interior(u, nx, ny)
        want = inner.mean(axis=(1, 2))
        bands = -(-ny // 16)
        n_add = -(-nx // 128) * 16 + 5 + 4 + -(-bands // 32) + 5 + 2
        bound = n_add * 2.0 ** -47 * np.abs(inner).mean(axis=(1, 2))
        assert np.all(np.abs(m - want) <= bound), (np.abs(m - want) / bound)
        p = fp.cpu().numpy()[:, :, : nx + 2].astype(np.float64)
        exact = u[:, :, : nx + 2] - m[:, None, None]
        assert np.all(np.abs(p - exact) <= 2.0 ** -24 * np.abs(exact) + 1e-30)


def test_split_field_means_repeat_and_fall_back_to_fp64(gpu):
    """The means are bit-identical from call to call (fixed summation
    order). A level holding values the float pairs cannot carry (1e120, a
    tiny 1e-30 among O(1) values) is summed in FP64 instead: its mean then
    matches the FP64 average to FP64 rounding."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 300, 40, 5
    u = synth.fields_iid(nx, ny, nz, seed=21)[0]
    u[2, 5, 7] = 1e120
    u[3, 9, 11] = 1e-30
    t = to_device(u, nx, torch.float64)
    runs = [pw.split_field(t, nx, ny)[1].clone() for _ in range(3)]
    torch.cuda.synchronize()
    for r in runs[1:]:
        assert torch.equal(r.view(torch.int64), runs[0].view(torch.int64))
    m = runs[0].cpu().numpy()
    inner = interior(u, nx, ny)
    want = inner.mean(axis=(1, 2))
    scale = np.abs(inner).mean(axis=(1, 2))
    assert np.all(np.abs(m[2:4] - want[2:4]) <= 1e-13 * scale[2:4]), (m[2:4], want[2:4])


@pytest.mark.parametrize("nz", [5, 40])
def test_split_field_conversion_is_the_hardware_rounding(gpu, nz):
    """The perturbations equal the GPU's own double->float conversion of
    f - mean[k] bit for bit (round to nearest even). Level 0 has a zero
    interior, so its mean is exactly 0 and its halo cells reach the edge
    cases: float overflow, infinities, NaN, float subnormals and values that
    round to zero or to the smallest normal."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny = 77, 21
    rng = np.random.default_rng(5)
    u = np.zeros((nz, ny + 2, nx + 2))
    u[1:] = rng.uniform(-10, 10, (nz - 1, ny + 2, nx + 2)) * 10.0 ** rng.integers(-3, 4, (nz - 1, ny + 2, nx + 2))
    special = [1e39, -1e39, 3.4028235677973366e38 * (1 + 2 ** -25), np.inf, -np.inf, np.nan, 1e-40, -3e-39,
               1e-46, 2.0 ** -126 * (1 - 2 ** -30), 2.0 ** -150, -2.0 ** -149 * 1.5, 2.0 ** -126, 0.0, -0.0]
    u[0, 0, :len(special)] = special
    u[0, ny + 1, :len(special)] = [-x for x in special]
    t = to_device(u, nx, torch.float64)
    fp, mean = pw.split_field(t, nx, ny)
    torch.cuda.synchronize()
    assert float(mean[0]) == 0.0
    want = (t - mean[:, None, None]).float()[:, :, : nx + 2]
    got = fp[:, :, : nx + 2]
    nan = torch.isnan(want)
    assert torch.equal(torch.isnan(got), nan)
    assert torch.equal(got.view(torch.int32)[~nan], want.view(torch.int32)[~nan])


@pytest.mark.parametrize("which", ["16m_modes", "134m_iid"])
def test_split_full_size(gpu, oracle_lib, which):
    """Full-size workloads in the benchmark's launch configuration; reports
    max and RMS errors relative to the FP64 oracle."""
    cfg = synth.config_16m_modes() if which == "16m_modes" else synth.config_134m_iid()
    u, v, w = cfg["fields"]()
    stats = _case(gpu, oracle_lib, u, v, w, cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"])
    print(which, stats)
