"""Host-side logic of bench.py that needs no GPU: the kernel-source hash that
keys the stored ncu traffic covers every local header the kernels include."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_source_hash_covers_included_headers():
    names = {m: {os.path.basename(p) for p in bench.kernel_sources(m)} for m in ("paired", "split", "f64")}
    common = {"pw_common.cuh", "pw_ring.cuh", "pw_internal.h"}
    assert names["paired"] >= common | {"pw_paired.cu", "pw_pair.cuh", "pw.h"}
    assert names["split"] >= common | {"pw_split.cu", "pw.h"}
    assert names["f64"] >= common | {"pw_f64.cu", "pw.h"}
    assert bench.kernel_source_hash("paired") != bench.kernel_source_hash("split")


def test_f64_operation_count_matches_the_tile():
    """The FP64 lane-operation count the bench reports for the native kernel
    follows from its 32 x 16 tile: the scaled cells and the six face-sum
    types over 512 points, plus 3 vertical sums and 18 face products per
    point, plus 3 coefficient products on a grid without density (the
    benchmark's) or 6 with one."""
    tx, ty = 32, 16
    scale = ((ty + 1) * (tx + 2) + (ty + 2) * (tx + 1)) / (tx * ty)
    faces = (3 * ty * (tx + 1) + 3 * (ty + 1) * tx) / (tx * ty)
    assert abs(bench.F64_OPS_PER_POINT - (scale + faces + 24)) < 1e-12
    assert abs(bench.F64_OPS_PER_POINT_DENSITY - (scale + faces + 27)) < 1e-12
    assert 32 < bench.F64_OPS_PER_POINT < 33


def test_reference_arm_prints_our_config():
    """Both arms name the same workload in the same config dict."""
    assert bench.CONFIG["workload"] == bench.WORKLOAD
    assert bench.CONFIG["nx"] * bench.CONFIG["ny"] * bench.CONFIG["nz"] == bench.CONFIG["points_per_gpu"]
