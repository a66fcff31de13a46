"""GPU checks of the FP64 energy-budget diagnostic (pw_energy_budget) and of
the conservation property of every arithmetic path.

On a domain periodic in x and y with w = 0 on the ground and at the lid, the
flux form conserves the mass-weighted energies: sum wu u su, sum wu v sv and
sum ww w sw vanish in exact arithmetic (the oracle's own outputs are pinned
to this on the CPU). A path's rounding error e at a point is bounded by its
per-point tolerance t * S (S its error scale), so its budget residual obeys
    |sum wt q s| <= t * sum wt |q| S,
the bound checked here for each mode. The residual is also held to 1e-13 of
the sum of the absolute summands, sum |wt q s|, for the FP64 and paired
paths, and reported for the FP32 ones. The diagnostic itself is checked
against the oracle's budget of the same GPU outputs: the oracle sums with
compensation (error about one rounding), the GPU in a fixed tree whose
longest path, at these sizes a few hundred additions, keeps it within 1e-13
of the sum of the absolute summands.
"""
import numpy as np
import pytest

from helpers import TOL_F32_ELEM, TOL_F64, TOL_PAIRED, TOL_SPLIT_ELEM, to_device, to_numpy_f64
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


def _periodic_case(nx, ny, nz, seed, modes=True):
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    if modes:
        u, v, w = synth.fields_modes(nx, ny, nz, 50.0, 50.0, dz, seed=seed)
    else:
        u, v, w = synth.fields_iid(nx, ny, nz, seed=seed)
    w[0] = 0.0
    w[nz - 1] = 0.0
    for f in (u, v, w):
        synth.fill_periodic_halo(f, nx, ny)
    return (u, v, w), dz, rho, rhon


def _run_mode(torch, pw, mode, fields, c, nx, ny, nz):
    """GPU source terms of one mode, and the winds the budget pairs them
    with (the FP64 winds for the split path, float winds for f32)."""
    if mode in ("f64", "paired"):
        dev = [to_device(f, nx, torch.float64) for f in fields]
        return dev, pw.advect(*dev, c, nx, ny, mode=mode)
    if mode == "f32":
        dev = [to_device(f, nx, torch.float32) for f in fields]
        return dev, pw.advect(*dev, c, nx, ny, mode="f32")
    dev = [to_device(f, nx, torch.float64) for f in fields]
    fp, means = zip(*(pw.split_field(t, nx, ny) for t in dev))
    table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    return dev, pw.advect(*fp, c, nx, ny, mode="split", split_table=table)


def _mode_scale(oracle_lib, mode, fields, co, nx, ny, means=None):
    u, v, w = fields
    if mode == "f64":
        return oracle_lib.advect(u, v, w, co, nx, ny, want_abs=True, nthreads=8)[1], TOL_F64
    if mode == "paired":
        return oracle_lib.monomial_scale(u, v, w, co, nx, ny, nthreads=8), TOL_PAIRED
    if mode == "f32":
        return oracle_lib.monomial_scale(u, v, w, co, nx, ny, nthreads=8), TOL_F32_ELEM
    mags = [np.abs(m)[:, None, None] + np.abs(f - m[:, None, None]) for f, m in zip(fields, means)]
    return oracle_lib.advect(*mags, co, nx, ny, want_abs=True, nthreads=8)[1], TOL_SPLIT_ELEM


@pytest.mark.parametrize("mode", ["f64", "paired", "f32", "split"])
@pytest.mark.parametrize("shape,modes", [((70, 45, 24), True), ((33, 17, 9), False), ((512, 512, 64), True)])
def test_energy_conservation_of_each_path(gpu, oracle_lib, mode, shape, modes):
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = shape
    fields, dz, rho, rhon = _periodic_case(nx, ny, nz, seed=nx + ny, modes=modes)
    co = oracle_lib.coeffs(nz, 50.0, 50.0, dz, rho, rhon)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz, rho, rhon).to_device()
    wu_h, ww_h = pw.make_energy_weights(nz, dz, rho, rhon)
    wu, ww = (torch.from_numpy(a).cuda() for a in (wu_h, ww_h))
    winds, out = _run_mode(torch, pw, mode, fields, c, nx, ny, nz)
    totals, level = pw.energy_budget(*winds, *out, nx, ny, wu, ww)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    tot = totals.cpu().numpy()
    # the diagnostic against the oracle's budget of the same outputs
    sy = fields[0].shape[2]  # one layout for the oracle: the FP64 winds' row stride
    wn = [to_numpy_f64(t.double(), sy, nx) for t in winds]
    sn = [to_numpy_f64(t.double(), sy, nx) for t in out]
    ref = oracle_lib.energy_budget(*wn, *sn, wu_h, ww_h, nx, ny)
    for n in range(3):
        assert abs(tot[n] - ref[n]) <= 1e-13 * ref[3 + n], (n, tot[n], ref[n])
        assert abs(tot[3 + n] - ref[3 + n]) <= 1e-13 * ref[3 + n]
    # per-level sums add up to the totals
    lv = level.cpu().numpy()
    for n in range(6):
        wt = ww_h if n % 3 == 2 else wu_h
        assert abs(float(np.sum(wt * lv[:, n])) - tot[n]) <= 1e-13 * tot[3 + n % 3]
    # conservation: the residual within the mode's rounding bound
    means = None
    if mode == "split":
        means = [f[:, 1:ny + 1, 1:nx + 1].mean(axis=(1, 2)) for f in fields]
    scale, tol = _mode_scale(oracle_lib, mode, fields, co, nx, ny, means)
    ratios = []
    for n, (q, s, wt) in enumerate(zip(fields, scale, (wu_h, wu_h, ww_h))):
        bound = float(np.sum(wt[:, None, None] * np.abs(q[:, 1:ny + 1, 1:nx + 1]) * s[:, 1:ny + 1, 1:nx + 1]))
        assert abs(tot[n]) <= tol * bound, (mode, n, tot[n], bound)
        ratios.append(abs(tot[n]) / tot[3 + n])
        if mode in ("f64", "paired"):
            assert abs(tot[n]) <= 1e-13 * tot[3 + n], (mode, n, tot[n], tot[3 + n])
    print(f"{mode} {shape}: residual / sum|summands| = {ratios}")


def test_energy_budget_sees_a_broken_tendency(gpu, oracle_lib):
    """The diagnostic is not blind: a source term whose upper vertical flux
    uses tzc1 in place of tzc2 (coefficients swapped on the device) leaves a
    residual many orders above rounding."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 40, 24, 16
    fields, dz, rho, rhon = _periodic_case(nx, ny, nz, seed=5, modes=False)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz, rho, rhon)
    c.tz4 = c.tz4[[1, 0, 2, 3]].copy()
    c.to_device()
    wu_h, ww_h = pw.make_energy_weights(nz, dz, rho, rhon)
    wu, ww = (torch.from_numpy(a).cuda() for a in (wu_h, ww_h))
    winds, out = _run_mode(torch, pw, "f64", fields, c, nx, ny, nz)
    totals, _ = pw.energy_budget(*winds, *out, nx, ny, wu, ww)
    tot = totals.cpu().numpy()
    assert abs(tot[0]) > 1e-6 * tot[3]
