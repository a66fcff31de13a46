"""GPU checks of the adjoint (pw_advect_adjoint), the halo fold and the
autograd/rollout layer: against the oracle's scatter-form adjoint, the
dot-product test <J d, y> = <d, J^T y> (1e-12 in FP64), finite differences
of one evaluation and of a checkpointed 20-step forward-Euler rollout (1e-8
relative), and exact transposition of the periodic halo fill.
"""
import numpy as np
import pytest

from helpers import to_device
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


def _raw(nx, ny, nz, seed, stream, lo=-1.0, hi=1.0):
    """Values on every cell (halo included), padding columns zero."""
    f = synth.empty_field(nx, ny, nz)
    f[:, :, : nx + 2] = synth.uniform(seed, stream, nz * (ny + 2) * (nx + 2), lo, hi).reshape(nz, ny + 2, nx + 2)
    return f


@pytest.mark.parametrize("mode,dtype_name", [("f64", "float64"), ("paired", "float64"), ("f32", "float32")])
@pytest.mark.parametrize("shape", [(37, 13, 6), (64, 8, 3), (5, 3, 2), (33, 9, 1), (70, 20, 40), (1, 1, 3),
                                   (96, 24, 9)])
@pytest.mark.parametrize("aligned", [True, False])
def test_adjoint_matches_oracle(gpu, oracle_lib, mode, dtype_name, shape, aligned):
    """Gather-form GPU adjoint vs the oracle's scatter form, every cell the
    forward reads (halo included). Cotangent halos hold NaN: they must be
    ignored."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = shape
    dt = getattr(torch, dtype_name)
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=51)
    gs = [_raw(nx, ny, nz, 52, s) for s in range(3)]
    if mode == "f32":
        u, v, w = (f.astype(np.float32).astype(np.float64) for f in (u, v, w))
        gs = [g.astype(np.float32).astype(np.float64) for g in gs]
    co = oracle_lib.coeffs(nz, 50.0, 40.0, dz, rho, rhon)
    ref = oracle_lib.advect_adjoint(u, v, w, co, nx, ny, *gs)
    c = pw.make_coeffs(nz, 50.0, 40.0, dz, rho, rhon).to_device()
    du, dv, dw = (to_device(f, nx, dt, aligned=aligned) for f in (u, v, w))
    dg = []
    for g in gs:
        t = to_device(g, nx, dt, aligned=aligned)
        t[:, 0, :] = float("nan")
        t[:, :, 0] = float("nan")
        dg.append(t)
    out = pw.advect_adjoint(du, dv, dw, c, nx, ny, *dg, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    tol = 2e-6 if mode == "f32" else 1e-13
    for name, got, want in zip(("gu", "gv", "gw"), out, ref):
        gn = got.double().cpu().numpy()[:, :, : nx + 2]
        wn = want[:, :, : nx + 2]
        assert np.all(np.isfinite(gn)), name
        scale = max(np.max(np.abs(wn)), 1e-300)
        assert np.max(np.abs(gn - wn)) <= tol * scale, (name, np.max(np.abs(gn - wn)) / scale)


@pytest.mark.parametrize("dy", [50.0, 40.0])
@pytest.mark.parametrize("density", [False, True])
def test_adjoint_f64_shared_product_paths(gpu, oracle_lib, dy, density):
    """The native FP64 adjoint shares products when tcx = tcy (one
    coefficient for an output's x and y parts) and when every level's two
    vertical coefficients are equal (no density: one scaled cotangent per
    cell for both faces). All four combinations against the oracle."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 45, 21, 12
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz) if density else (None, None)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=71)
    gs = [_raw(nx, ny, nz, 72, s) for s in range(3)]
    ref = oracle_lib.advect_adjoint(u, v, w, oracle_lib.coeffs(nz, 50.0, dy, dz, rho, rhon), nx, ny, *gs)
    c = pw.make_coeffs(nz, 50.0, dy, dz, rho, rhon).to_device()
    x = [to_device(a, nx, torch.float64) for a in (u, v, w)]
    g = [to_device(a, nx, torch.float64) for a in gs]
    out = pw.advect_adjoint(*x, c, nx, ny, *g, mode="f64")
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    for name, got, want in zip(("gu", "gv", "gw"), out, ref):
        gn = got.double().cpu().numpy()[:, :, : nx + 2]
        wn = want[:, :, : nx + 2]
        err = np.max(np.abs(gn - wn)) / np.max(np.abs(wn))
        assert err <= 1e-13, (name, err)


@pytest.mark.parametrize("mode", ["f64", "paired"])
def test_adjoint_accumulate(gpu, mode):
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 20, 10, 5
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    f = [to_device(a, nx, torch.float64) for a in synth.fields_iid(nx, ny, nz, seed=3)]
    g = [to_device(_raw(nx, ny, nz, 4, s), nx, torch.float64) for s in range(3)]
    a = pw.advect_adjoint(*f, c, nx, ny, *g, mode=mode)
    b = pw.advect_adjoint(*f, c, nx, ny, *g, mode=mode, out=tuple(x.clone() for x in a), accumulate=True)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(2 * x, y)


@pytest.mark.parametrize("mode", ["f64", "paired", "f32"])
def test_dot_product_adjoint_256(gpu, mode):
    """<J(x) d, y> = <d, J(x)^T y> on the 256 x 256 x 64 workload with the
    small configuration's winds; J(x) d = (F(x + h d) - F(x - h d)) / 2h is
    exact for a quadratic map up to rounding. FP64: 1e-12 relative."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    dt = torch.float32 if mode == "f32" else torch.float64
    nx, ny, nz = 256, 256, 64
    dz = synth.dz_uniform(nz, 20.0)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz).to_device()
    x = [to_device(a, nx, dt) for a in synth.fields_iid(nx, ny, nz, seed=1)]
    d = [to_device(_raw(nx, ny, nz, 61, s), nx, dt) for s in range(3)]
    y = [to_device(_raw(nx, ny, nz, 62, s), nx, dt) for s in range(3)]
    h = 2.0 ** -6
    fwd = "f32" if mode == "f32" else "f64"
    fp = pw.advect(*[a + h * b for a, b in zip(x, d)], c, nx, ny, mode=fwd)
    fm = pw.advect(*[a - h * b for a, b in zip(x, d)], c, nx, ny, mode=fwd)
    inner = (slice(None), slice(1, ny + 1), slice(1, nx + 1))
    lhs = sum(float(((p - m)[inner].double() / (2 * h) * yy[inner].double()).sum()) for p, m, yy in zip(fp, fm, y))
    g = pw.advect_adjoint(*x, c, nx, ny, *y, mode=mode)
    rhs = sum(float((gg[:, :, : nx + 2].double() * dd[:, :, : nx + 2].double()).sum()) for gg, dd in zip(g, d))
    torch.cuda.synchronize()
    rel = abs(lhs - rhs) / max(abs(lhs), abs(rhs))
    assert rel <= (1e-4 if mode == "f32" else 1e-12), rel


@pytest.mark.parametrize("mode", ["f64", "paired", "f32"])
def test_adjoint_256_matches_oracle(gpu, oracle_lib, mode):
    """The benchmarked adjoint workload (256 x 256 x 64, i.i.d. winds, dx = dy
    = 50 m, uniform 20 m levels, U[-1, 1] cotangents) in the bench's field
    layout, every cell against the oracle's scatter form: per field
    max |g - o| / max |o| within 1e-13 (FP64 and paired) or 2e-6 (FP32)."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 256, 256, 64
    dt = torch.float32 if mode == "f32" else torch.float64
    dz = synth.dz_uniform(nz, 20.0)
    u, v, w = synth.fields_iid(nx, ny, nz, seed=1)
    gs = [_raw(nx, ny, nz, 63, s) for s in range(3)]
    if mode == "f32":
        u, v, w = (f.astype(np.float32).astype(np.float64) for f in (u, v, w))
        gs = [g.astype(np.float32).astype(np.float64) for g in gs]
    ref = oracle_lib.advect_adjoint(u, v, w, oracle_lib.coeffs(nz, 50.0, 50.0, dz), nx, ny, *gs)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz).to_device()
    x = [pw.field_from_numpy(a, nx, dt) for a in (u, v, w)]
    g = [pw.field_from_numpy(a, nx, dt) for a in gs]
    out = pw.advect_adjoint(*x, c, nx, ny, *g, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    tol = 2e-6 if mode == "f32" else 1e-13
    for name, got, want in zip(("gu", "gv", "gw"), out, ref):
        gn = got.double().cpu().numpy()[:, :, : nx + 2]
        wn = want[:, :, : nx + 2]
        err = np.max(np.abs(gn - wn)) / np.max(np.abs(wn))
        assert err <= tol, (name, err)


def test_fold_is_transpose_of_fill(gpu):
    """<fill(x), y> = <x, fold(y)> exactly on integer data."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    for nx, ny, nz in ((17, 9, 3), (1, 1, 2), (2, 5, 1)):
        x = to_device(_raw(nx, ny, nz, 71, 0, -8, 8).round(), nx, torch.float64)
        y = to_device(_raw(nx, ny, nz, 72, 0, -8, 8).round(), nx, torch.float64)
        fx = x.clone()
        pw.fill_periodic_halo(fx, nx, ny)
        fy = y.clone()
        pw.fold_periodic_halo(fy, nx, ny)
        torch.cuda.synchronize()
        a = float((fx[:, :, : nx + 2] * y[:, :, : nx + 2]).sum())
        b = float((x[:, :, : nx + 2] * fy[:, :, : nx + 2]).sum())
        assert a == b
        assert float(fy[:, 0, :].abs().sum()) == 0 and float(fy[:, :, 0].abs().sum()) == 0


def test_autograd_backward_is_adjoint(gpu):
    from paper_2107_13500_gb300 import autograd as pa
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 30, 12, 6
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_stretched(nz)).to_device()
    x = [to_device(a, nx, torch.float64).requires_grad_() for a in synth.fields_iid(nx, ny, nz, seed=8)]
    y = [to_device(_raw(nx, ny, nz, 9, s), nx, torch.float64) for s in range(3)]
    inner = (slice(None), slice(1, ny + 1), slice(1, nx + 1))
    out = pa.advect(*x, c, nx, ny, "paired")
    loss = sum((o[inner] * yy[inner]).sum() for o, yy in zip(out, y))
    grads = torch.autograd.grad(loss, x)
    ymask = []
    for yy in y:
        m = torch.zeros_like(yy)
        m[inner] = yy[inner]
        ymask.append(pw.field_like(x[0]).copy_(m))
    want = pw.advect_adjoint(*[t.detach() for t in x], c, nx, ny, *ymask)
    for g, wnt in zip(grads, want):
        assert torch.allclose(g, wnt, rtol=0, atol=1e-13 * float(wnt.abs().max()))


def _fd_noise_free_dot(torch, outs_p, outs_m, y, inner, h):
    """sum y * (F(x + h d) - F(x - h d)) / (2h), differenced element by
    element before the sum so that the sum's own rounding stays at the size
    of the differences, not of F."""
    return sum(float(((op[inner] - om[inner]) * yy[inner]).sum()) for op, om, yy in zip(outs_p, outs_m, y)) / (2 * h)


@pytest.mark.parametrize("mode", ["f64", "paired"])
def test_adjoint_finite_difference_single_step(gpu, mode):
    """One evaluation of the 256 x 256 x 64 workload: the map is quadratic,
    so a central difference with step 1e-6 equals the directional
    derivative up to rounding, and <y, (F(x+hd) - F(x-hd)) / 2h> must
    match <J^T y, d> from the adjoint kernel to 1e-8 relative. The
    difference is taken of the native FP64 forward map for both adjoint
    arithmetics."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 256, 256, 64
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_stretched(nz)).to_device()
    x = [to_device(a, nx, torch.float64) for a in synth.fields_iid(nx, ny, nz, seed=1)]
    y = [to_device(_raw(nx, ny, nz, 91, s), nx, torch.float64) for s in range(3)]
    d = [to_device(_raw(nx, ny, nz, 92, s, -10.0, 10.0), nx, torch.float64) for s in range(3)]
    inner = (slice(None), slice(1, ny + 1), slice(1, nx + 1))
    for t in y:
        keep = torch.zeros_like(t)
        keep[inner] = t[inner]
        t.copy_(keep)
    h = 1e-6
    fp = pw.advect(*[a + h * b for a, b in zip(x, d)], c, nx, ny, mode="f64")
    fm = pw.advect(*[a - h * b for a, b in zip(x, d)], c, nx, ny, mode="f64")
    g = pw.advect_adjoint(*x, c, nx, ny, *y, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    fd = _fd_noise_free_dot(torch, fp, fm, y, inner, h)
    an = sum(float((gg[:, :, : nx + 2] * dd[:, :, : nx + 2]).sum()) for gg, dd in zip(g, d))
    print(f"{mode}: fd {fd!r} adjoint {an!r} rel {abs(fd - an) / abs(an):.3e}")
    assert abs(fd - an) <= 1e-8 * abs(an), (fd, an)


def test_rollout_gradient_checkpointed_and_fd(gpu):
    """20-step forward-Euler rollout (dt = 0.5 s) of the 256 x 256 x 64
    workload's winds, differentiated with checkpoints every 5 steps: the
    gradient equals the uncheckpointed one exactly, and a central finite
    difference with step 1e-6 along a random direction of the winds' size
    matches it to 1e-8 relative. (The rollout is a polynomial of high
    degree, so the difference carries an O(h^2) term besides rounding; at
    this step both stay below 1e-8.)"""
    from paper_2107_13500_gb300 import autograd as pa
    from paper_2107_13500_gb300 import pw
    torch = gpu
    nx, ny, nz = 256, 256, 64
    c = pw.make_coeffs(nz, 50.0, 50.0, synth.dz_uniform(nz, 20.0)).to_device()
    x0 = [to_device(a, nx, torch.float64) for a in synth.fields_iid(nx, ny, nz, seed=1)]
    for t in x0:
        pw.fill_periodic_halo(t, nx, ny)
    y = [to_device(_raw(nx, ny, nz, 81, s), nx, torch.float64) for s in range(3)]
    inner = (slice(None), slice(1, ny + 1), slice(1, nx + 1))

    def rollout(xs, ckpt):
        return pa.rollout(*xs, c, nx, ny, 0.5, 20, mode="f64", checkpoint_every=ckpt)

    def objective(xs, ckpt):
        return sum((o[inner] * yy[inner]).sum() for o, yy in zip(rollout(xs, ckpt), y))

    xs = [t.clone().requires_grad_() for t in x0]
    g_ck = torch.autograd.grad(objective(xs, 5), xs)
    xs2 = [t.clone().requires_grad_() for t in x0]
    g_full = torch.autograd.grad(objective(xs2, 0), xs2)
    for a, b in zip(g_ck, g_full):
        assert torch.equal(a, b)
    d = [to_device(_raw(nx, ny, nz, 82, s, -10.0, 10.0), nx, torch.float64) for s in range(3)]
    for t in d:
        t[:, 0, :] = 0
        t[:, ny + 1, :] = 0
        t[:, :, 0] = 0
        t[:, :, nx + 1] = 0
    h = 1e-6
    with torch.no_grad():
        op = rollout([a + h * b for a, b in zip(x0, d)], 0)
        om = rollout([a - h * b for a, b in zip(x0, d)], 0)
    fd = _fd_noise_free_dot(torch, op, om, y, inner, h)
    an = sum(float((g * dd).sum()) for g, dd in zip(g_ck, d))
    print(f"rollout: fd {fd!r} adjoint {an!r} rel {abs(fd - an) / abs(an):.3e}")
    assert abs(fd - an) <= 1e-8 * abs(an), (fd, an)


@pytest.mark.parametrize("mode", ["f64", "paired", "f32"])
def test_adjoint_euler_identity(gpu, mode):
    """Euler's identity for the quadratic map, J(x) x = 2 F(x), seen through
    the adjoint: <J(x)^T y, x> = 2 <y, F(x)>, summed over every cell the
    forward reads (the outputs' halo is left zero, so F vanishes off the
    computed points). Independent of any finite-difference step."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    dt = torch.float32 if mode == "f32" else torch.float64
    nx, ny, nz = 96, 40, 24
    dz = synth.dz_stretched(nz)
    rho, rhon = synth.density_exponential(dz)
    c = pw.make_coeffs(nz, 50.0, 50.0, dz, rho, rhon).to_device()
    x = [to_device(_raw(nx, ny, nz, 71, s, -10.0, 10.0), nx, dt) for s in range(3)]
    y = [to_device(_raw(nx, ny, nz, 72, s), nx, dt) for s in range(3)]
    f = pw.advect(*x, c, nx, ny, mode="f32" if mode == "f32" else "f64")
    g = pw.advect_adjoint(*x, c, nx, ny, *y, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    cells = (slice(None), slice(None), slice(0, nx + 2))
    lhs = sum(float((gg[cells].double() * xx[cells].double()).sum()) for gg, xx in zip(g, x))
    rhs = 2.0 * sum(float((yy[cells].double() * ff[cells].double()).sum()) for yy, ff in zip(y, f))
    scale = sum(float((gg[cells].double() * xx[cells].double()).abs().sum()) for gg, xx in zip(g, x))
    assert abs(lhs - rhs) <= (1e-5 if mode == "f32" else 1e-12) * scale, (lhs, rhs, scale)
