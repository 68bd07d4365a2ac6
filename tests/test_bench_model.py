"""The benchmark's per-kernel byte model (the roofline's algorithmic bytes)
agrees with the counts module's per-step totals, for both operators, every
storage type and both forms of the iteration (CPU only)."""

import pytest

import bench
from oracle import counts

W = {"f64": (8, 8), "f32": (4, 4), "bf16": (2, 4), "f16": (2, 4)}


@pytest.mark.parametrize("storage", sorted(W))
def test_byte_model_matches_counts(storage):
    w, wx = W[storage]
    per_kernel, total = bench.bytes_per_cell(storage)
    assert total == sum(per_kernel.values()) == counts.bytes_per_cell(w, w, wx)
    per_kernel9, total9 = bench.bytes_per_cell9(storage)
    assert total9 == sum(per_kernel9.values()) == counts.bytes_per_cell_9pt(w, w, wx)
    # the two-reduction form moves three fewer vector words per cell (q is
    # formed twice but never stored; the update pass disappears)
    _, merged = bench.bytes_per_cell(storage, variant=1)
    _, merged9 = bench.bytes_per_cell9(storage, variant=1)
    assert total - merged == 3 * w and total9 - merged9 == 3 * w


def test_paper_size_figures():
    _, total = bench.bytes_per_cell("f32")
    assert total == 116
    # 116 B x 548,352,000 cells at the measured 6674.8 GB/s: 9.53 ms per step
    assert abs(total * 548352000 / 6674.8e9 * 1e3 - 9.53) < 0.01
    assert bench.FLOPS_PER_CELL == 44 and bench.FLOPS_PER_CELL_9PT == counts.ops_per_point_9pt()
