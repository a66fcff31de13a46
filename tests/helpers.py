"""Shared test helpers: oracle/GPU comparison with one tolerance per arithmetic
mode, guard-band canaries, tensor <-> numpy layout moves.

Error scales (per point, from the oracle): the strict scale A is the sum of
|c||q||a+b| over the face terms c*q*(a+b) of an output, the sum of the
absolute values of the products the formula adds up. The monomial scale M
counts each face term as |c||q|(|a|+|b|); M >= A, and M differs from A only
where the two velocity samples of a face nearly cancel.

Tolerances:
  * native FP64 (PW_F64): |gpu - oracle| <= 1e-13 * A per point and
    max|gpu - oracle| <= 1e-13 * max|oracle| per field.
  * paired FP32 (PW_F64_PAIRED): the same normwise bound; per point
    |gpu - oracle| <= 1e-13 * M. The paired path splits each double into a
    float pair (48 significant bits) before it forms a + b, so that rounding
    is relative to |a| and |b|, not to |a + b|: M, not A, bounds it. The
    worst ratio against A is reported beside it.
  * plain FP32 on full fields (PW_F32), against the oracle on the original
    double fields: |gpu - oracle| <= 32 * 2^-24 * M per point. Rounding the
    inputs c, q, a, b to float (4 roundings), a + b, the two products (3) and
    the five additions of the six face terms (5), each at most 2^-24 of
    quantities bounded by M, plus the float result (1): 13 * 2^-24 * M to
    first order; 32 leaves room for the order of evaluation.
  * FP32 split (PW_F32_SPLIT): |gpu - oracle| <= 64 * 2^-24 * A', A' the
    strict scale evaluated on the magnitude fields |U(k)| + |u'|.
"""
import numpy as np

TOL_F64 = 1e-13
TOL_PAIRED = 1e-13
TOL_F32_ELEM = 32 * 2.0 ** -24
TOL_SPLIT_ELEM = 64 * 2.0 ** -24


def interior(a, nx, ny, k0=0, k1=None):
    return a[k0:k1, 1:ny + 1, 1:nx + 1]


def _ratios(err, scale):
    return err / np.maximum(scale, 1e-300)


def compare_f64(gpu, ora, strict, nx, ny, tol=TOL_F64):
    """Native FP64: both criteria on (su, sv, sw) against the strict scale;
    returns {field: (max err/A, normwise)}."""
    worst = {}
    for name, g, o, a in zip(("su", "sv", "sw"), gpu, ora, strict):
        gi, oi, ai = interior(g, nx, ny), interior(o, nx, ny), interior(a, nx, ny)
        err = np.abs(gi - oi)
        assert np.all(np.isfinite(gi)), f"{name}: non-finite output"
        bad = err > tol * ai
        assert not np.any(bad), (f"{name}: elementwise bound violated at {np.argwhere(bad)[:5]}, "
                                 f"max err/A = {np.max(_ratios(err, ai)):.3e}")
        mo = float(np.max(np.abs(oi)))
        if mo > 0:
            assert float(np.max(err)) <= tol * mo, f"{name}: normwise {np.max(err) / mo:.3e} > {tol}"
        worst[name] = (float(np.max(_ratios(err, ai))), float(np.max(err)) / mo if mo > 0 else 0.0)
    return worst


def compare_paired(gpu, ora, strict, mono, nx, ny, tol=TOL_PAIRED):
    """Paired FP32: per point against the monomial scale, normwise as FP64;
    returns {field: (max err/M, max err/A, normwise)}."""
    worst = {}
    for name, g, o, a, m in zip(("su", "sv", "sw"), gpu, ora, strict, mono):
        gi, oi = interior(g, nx, ny), interior(o, nx, ny)
        ai, mi = interior(a, nx, ny), interior(m, nx, ny)
        err = np.abs(gi - oi)
        assert np.all(np.isfinite(gi)), f"{name}: non-finite output"
        bad = err > tol * mi
        assert not np.any(bad), (f"{name}: elementwise bound violated at {np.argwhere(bad)[:5]}, "
                                 f"max err/M = {np.max(_ratios(err, mi)):.3e}")
        mo = float(np.max(np.abs(oi)))
        if mo > 0:
            assert float(np.max(err)) <= tol * mo, f"{name}: normwise {np.max(err) / mo:.3e} > {tol}"
        worst[name] = (float(np.max(_ratios(err, mi))), float(np.max(_ratios(err, ai))),
                       float(np.max(err)) / mo if mo > 0 else 0.0)
    return worst


def compare_f32(gpu, ora, mono, nx, ny, tol=TOL_F32_ELEM):
    """Plain FP32: per point against the monomial scale; returns
    {field: (max err/M, max relative error, RMS relative error)}."""
    worst = {}
    for name, g, o, m in zip(("su", "sv", "sw"), gpu, ora, mono):
        gi, oi, mi = interior(g, nx, ny).astype(np.float64), interior(o, nx, ny), interior(m, nx, ny)
        err = np.abs(gi - oi)
        assert np.all(np.isfinite(gi)), f"{name}: non-finite output"
        bad = err > tol * mi
        assert not np.any(bad), (f"{name}: elementwise bound violated at {np.argwhere(bad)[:5]}, "
                                 f"max err/M = {np.max(_ratios(err, mi)):.3e}")
        mo = float(np.max(np.abs(oi)))
        rms_o = float(np.sqrt(np.mean(oi ** 2)))
        worst[name] = (float(np.max(_ratios(err, mi))), float(np.max(err)) / mo if mo > 0 else 0.0,
                       float(np.sqrt(np.mean(err ** 2))) / rms_o if rms_o > 0 else 0.0)
    return worst


def check_mode(mode, gpu, ora, strict, mono, nx, ny):
    """The comparison that belongs to an FP64-output mode."""
    if mode == "f64":
        return compare_f64(gpu, ora, strict, nx, ny)
    if mode == "paired":
        return compare_paired(gpu, ora, strict, mono, nx, ny)
    raise ValueError(mode)


def to_numpy_f64(t, sy_np, nx):
    """Copy a GPU field (any padded stride) into a numpy array with row length sy_np."""
    a = t.detach().cpu().numpy()
    out = np.zeros((a.shape[0], a.shape[1], sy_np), dtype=np.float64)
    out[:, :, : nx + 2] = a[:, :, : nx + 2]
    return out


def to_device(a, nx, torch_dtype, device="cuda", aligned=True):
    """Numpy field -> GPU tensor in the library's padded layout for torch_dtype.
    aligned=True puts i = 1 on a 16-byte boundary (vectorised kernels);
    aligned=False leaves i = 0 there (the kernels' general path)."""
    from paper_2107_13500_gb300 import pw
    return pw.field_from_numpy(a, nx, torch_dtype, device, aligned)
