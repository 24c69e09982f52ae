"""The recorded ncu traffic belongs to the kernels in the tree: every row of
profiles/dram_traffic.txt that the bench reads carries the hash of the
current sources of its kernel, so the bench line reports it (a row whose
kernel changed since its capture is reported as null)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rows():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_traffic_rows_match_the_kernel_sources():
    rows = _rows()
    for kernel in bench.KERNEL_SOURCES:
        for key in ("config3@1", "config2@1"):
            match = [r for r in rows if r[0] == kernel and r[1] == key]
            assert len(match) == 1, (kernel, key)
            assert match[0][3] == bench.kernel_source_hash(kernel), (kernel, key)
            assert bench.recorded_traffic(kernel, key, 2) > 0
            assert bench.recorded_traffic(kernel, key, 4) > 0
