"""Shared test helpers: oracle/GPU comparison with the tolerances derived in
the design notes, guard-band canaries, tensor <-> numpy layout moves."""
import numpy as np

# FP64 paths (native and paired): per point |gpu - oracle| <= TOL_F64 * A,
# A = sum of |product terms| at that point, and per field
# max|gpu - oracle| <= TOL_F64 * max|oracle|.
TOL_F64 = 1e-13
# FP32 split path: every product term carries at most a handful of float
# roundings (2^-24 each) plus the rounding of each perturbation, so
# |gpu - oracle| <= TOL_SPLIT_ELEM * A (64 * 2^-24, about 3.8e-6).
TOL_SPLIT_ELEM = 64 * 2.0 ** -24


def interior(a, nx, ny, k0=0, k1=None):
    return a[k0:k1, 1:ny + 1, 1:nx + 1]


def compare_f64(gpu, ora, absterms, nx, ny, tol=TOL_F64):
    """Assert both FP64 criteria on (su, sv, sw); return the worst ratios."""
    worst = {}
    for name, g, o, a in zip(("su", "sv", "sw"), gpu, ora, absterms):
        gi, oi, ai = interior(g, nx, ny), interior(o, nx, ny), interior(a, nx, ny)
        err = np.abs(gi - oi)
        assert np.all(np.isfinite(gi)), f"{name}: non-finite output"
        bad = err > tol * ai
        assert not np.any(bad), (f"{name}: elementwise bound violated at {np.argwhere(bad)[:5]}, "
                                 f"max err/A = {np.max(err / np.maximum(ai, 1e-300)):.3e}")
        mo = float(np.max(np.abs(oi)))
        if mo > 0:
            assert float(np.max(err)) <= tol * mo, f"{name}: normwise {np.max(err) / mo:.3e} > {tol}"
        worst[name] = (float(np.max(err / np.maximum(ai, 1e-300))), float(np.max(err)) / mo if mo > 0 else 0.0)
    return worst


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
