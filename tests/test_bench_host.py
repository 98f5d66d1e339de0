"""Host-side helpers of bench.py (no GPU): the kernel-source hash ignores
comments and blank lines, and the stored DRAM traffic of the stage kernels
applies only to the grid it is stated for and to the sources it was taken on."""
from __future__ import annotations

import bench


def test_kernel_hash_ignores_comments_and_blank_lines():
    a = "int x;  // one\n\n// two\nint y;\n"
    b = "int x;\nint y;   \n"
    assert bench._kernel_hash(a) == bench._kernel_hash(b)
    assert bench._kernel_hash(a) != bench._kernel_hash("int x;\nint z;\n")


def test_stored_traffic_only_for_its_grid():
    for prec in bench.BYTES_PER_CELL_STAGE:
        assert bench._ncu_traffic(prec, 2048 * 2048) is None
    v = bench._ncu_traffic("f64", bench.TRAFFIC_CELLS)
    # None once the kernel sources differ from those of the capture; else the
    # FP64 per-launch traffic at 8192^2, near the algorithmic 21 planes x 8 B
    assert v is None or abs(v / (21 * 8 * bench.TRAFFIC_CELLS) - 1.0) < 0.05
