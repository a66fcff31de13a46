"""Fields of more than 2^31 elements: 2046 x 2046 x 520 cells (2048 x 2048
x 520 = 2,181,038,080 elements with the halo; 17.4 GB per FP64 field), so
that every kernel's addressing has to be 64-bit. Inputs are i.i.d. uniform
winds drawn on the device from a seeded generator. The oracle cannot take
the whole domain, so whole columns are checked: all 520 levels of the
3 x 3 (forward) or 5 x 5 (adjoint) neighbourhood of a column are copied to
the host, the oracle computes that column as a 1 x 1 (3 x 3) domain with
the neighbourhood as its halo, and the GPU's column must match at the
mode's tolerance. The columns include the domain's four corners, whose top
levels lie past 2^31 elements (2^34 bytes for FP64) from the field's start.
"""
import numpy as np
import pytest

from helpers import TOL_SPLIT_ELEM, compare_f32, compare_f64, compare_paired
from paper_2107_13500_gb300 import synth

pytestmark = pytest.mark.gpu

NX, NY, NZ = 2046, 2046, 520
DX = DY = 50.0


@pytest.fixture(scope="module")
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_13500_gb300 import build, pw
    build.build()
    pw.load_library()
    return torch


def _need(torch, fields, elem_bytes):
    """Skip unless `fields` fields of this size fit in free device memory."""
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    want = fields * NZ * (NY + 2) * 2048 * elem_bytes * 1.05
    if free < want:
        pytest.skip(f"needs {want / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")


def _fields(torch, dtype, seed, lo=-10.0, hi=10.0, n=3):
    from paper_2107_13500_gb300 import pw
    gen = torch.Generator(device="cuda").manual_seed(seed)
    out = []
    for _ in range(n):
        f = pw.empty_field(NX, NY, NZ, dtype)
        f.uniform_(lo, hi, generator=gen)
        out.append(f)
    last = (NZ - 1) * out[0].stride(0) + NY * out[0].stride(1) + NX
    assert out[0].numel() > 2 ** 31 and last > 2 ** 31
    return out


def _columns(edge, seed):
    """(i, j) of the checked columns: the corners of the cells at least
    `edge` from the domain's border, and four seeded ones inside."""
    lo, hx, hy = edge, NX + 1 - edge, NY + 1 - edge
    rng = np.random.default_rng(seed)
    cols = [(lo, lo), (hx, hy), (hx, lo), (lo, hy)]
    cols += [(int(rng.integers(lo, hx + 1)), int(rng.integers(lo, hy + 1))) for _ in range(4)]
    return cols


def _block(t, i, j, r):
    """All levels of the (2r+1) x (2r+1) cells around column (i, j), FP64."""
    return np.ascontiguousarray(t[:, j - r:j + r + 1, i - r:i + r + 1].double().cpu().numpy())


def _column_as_block(t, i, j, r):
    """The GPU's column (i, j), placed at the centre of an otherwise zero block."""
    b = np.zeros((NZ, 2 * r + 1, 2 * r + 1))
    b[:, r, r] = t[:, j, i].double().cpu().numpy()
    return b


def _coeffs():
    from paper_2107_13500_gb300 import pw
    dz = synth.dz_uniform(NZ, 20.0)
    return pw.make_coeffs(NZ, DX, DY, dz).to_device(), dz


@pytest.mark.parametrize("mode", ["f64", "f64_batched", "paired", "f32"])
def test_forward_beyond_2_31_elements(gpu, oracle_lib, mode):
    from paper_2107_13500_gb300 import pw
    torch = gpu
    f32 = mode == "f32"
    _need(torch, 6, 4 if f32 else 8)
    x = _fields(torch, torch.float32 if f32 else torch.float64, seed=11)
    c, dz = _coeffs()
    if mode == "f64_batched":
        b = pw.Batch([dict(u=x[0], v=x[1], w=x[2], nx=NX, ny=NY, coeffs=c)], "f64", 0)
        b.run()
        out = b.outputs()[0]
    else:
        out = pw.advect(*x, c, NX, NY, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    co = oracle_lib.coeffs(NZ, DX, DY, dz)
    for i, j in _columns(1, seed=1):
        blk = [_block(t, i, j, 1) for t in x]
        so, ab = oracle_lib.advect(*blk, co, 1, 1, want_abs=True)
        g = [_column_as_block(t, i, j, 1) for t in out]
        if mode in ("f64", "f64_batched"):
            compare_f64(g, so, ab, 1, 1)
        else:
            mb = oracle_lib.monomial_scale(*blk, co, 1, 1)
            if f32:
                compare_f32(g, so, mb, 1, 1)
            else:
                compare_paired(g, so, ab, mb, 1, 1)
    del x, out
    torch.cuda.empty_cache()


def test_split_beyond_2_31_elements(gpu, oracle_lib):
    """pw_split_field and the FP32 split forward: the level means against
    torch's own FP64 mean of the interior, the perturbations of the checked
    columns bit for bit against float(f - mean) formed by torch, and the
    tendencies of those columns against the oracle on the FP64 fields."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    _need(torch, 6, 8)  # three FP64 fields, three float perturbations, three float outputs
    x = _fields(torch, torch.float64, seed=12)
    c, dz = _coeffs()
    fp, means = zip(*(pw.split_field(t, NX, NY) for t in x))
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    # paired sums of at most n_add additions on a value's path (a thread's
    # columns of a band of 16 rows, the warp tree, 4 warps, a lane's bands,
    # the lane tree, the join), each within 2^-47 of the magnitudes summed
    # so far (|f| <= 10)
    n_add = -(-NX // 128) * 16 + 5 + 4 + -(-(-(-NY // 16)) // 32) + 5 + 2
    bound = n_add * 2.0 ** -47 * 10.0
    for t, m in zip(x, means):
        want = t[:, 1:NY + 1, 1:NX + 1].mean(dim=(1, 2))
        assert float((m - want).abs().max()) <= bound
    table = torch.from_numpy(pw.make_split_table(c, *(m.cpu().numpy() for m in means))).cuda()
    out = pw.advect(*fp, c, NX, NY, mode="split", split_table=table)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    co = oracle_lib.coeffs(NZ, DX, DY, dz)
    mh = [m.cpu().numpy() for m in means]
    for i, j in _columns(1, seed=2):
        for t, p, m in zip(x, fp, means):
            want = (t[:, j - 1:j + 2, i - 1:i + 2] - m[:, None, None]).float()
            assert torch.equal(p[:, j - 1:j + 2, i - 1:i + 2].view(torch.int32), want.view(torch.int32))
        blk = [_block(t, i, j, 1) for t in x]
        so = oracle_lib.advect(*blk, co, 1, 1)
        mags = [np.abs(m)[:, None, None] + np.abs(b - m[:, None, None]) for b, m in zip(blk, mh)]
        _, ab = oracle_lib.advect(*mags, co, 1, 1, want_abs=True)
        for name, t, o, a in zip(("su", "sv", "sw"), out, so, ab):
            err = np.abs(t[:, j, i].double().cpu().numpy() - o[:, 1, 1])
            assert np.all(err <= TOL_SPLIT_ELEM * a[:, 1, 1]), (name, i, j)
    del x, fp, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_adjoint_beyond_2_31_elements(gpu, oracle_lib, mode):
    """The adjoint on nine fields past 2^31 elements, columns against the
    oracle's adjoint of their 5 x 5 neighbourhood: a cell's gradient gathers
    the cotangents of the outputs within one cell of it (diagonals
    included), whose own stencils reach two cells from it."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    f32 = mode == "f32"
    dt = torch.float32 if f32 else torch.float64
    _need(torch, 9, 4 if f32 else 8)
    x = _fields(torch, dt, seed=13)
    gs = _fields(torch, dt, seed=14, lo=-1.0, hi=1.0)
    c, dz = _coeffs()
    out = pw.advect_adjoint(*x, c, NX, NY, *gs, mode=mode)
    torch.cuda.synchronize()
    assert pw.device_status() == 0
    co = oracle_lib.coeffs(NZ, DX, DY, dz)
    tol = 2e-6 if f32 else 1e-13
    for i, j in _columns(2, seed=3):
        xb = [_block(t, i, j, 2) for t in x]
        gb = [_block(t, i, j, 2) for t in gs]
        ref = oracle_lib.advect_adjoint(*xb, co, 3, 3, *gb)
        for name, t, r in zip(("gu", "gv", "gw"), out, ref):
            got, want = t[:, j, i].double().cpu().numpy(), r[:, 2, 2]
            assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want)), (name, i, j)
    del x, gs, out
    torch.cuda.empty_cache()


def test_halo_fill_beyond_2_31_elements(gpu):
    """pw_fill_periodic_halo: the halo of the top level equals its periodic
    sources bit for bit."""
    from paper_2107_13500_gb300 import pw
    torch = gpu
    _need(torch, 1, 8)
    (f,) = _fields(torch, torch.float64, seed=15, n=1)
    pw.fill_periodic_halo(f, NX, NY)
    torch.cuda.synchronize()
    top = f[NZ - 1]
    assert torch.equal(top[1:NY + 1, 0], top[1:NY + 1, NX])
    assert torch.equal(top[1:NY + 1, NX + 1], top[1:NY + 1, 1])
    assert torch.equal(top[0, :NX + 2], top[NY, :NX + 2])
    assert torch.equal(top[NY + 1, :NX + 2], top[1, :NX + 2])
    del f
    torch.cuda.empty_cache()
