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
    assert names["f64"] >= common | {"pw_kernels.cu"}
    assert bench.kernel_source_hash("paired") != bench.kernel_source_hash("split")
