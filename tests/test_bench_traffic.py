"""bench.py's DRAM-traffic lookup: the committed ncu figure is reported only while the
kernel's own definition is the one that was captured (CPU only)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """// header
template <typename T>
__global__ void k_one(const T* a, T* b) {
  b[0] = a[0];
}

__global__ void k_two(int* c) {
  c[0] = 1;
}
"""


def test_kernel_source_extracts_one_definition():
    one = bench.kernel_source(SRC, "k_one")
    assert one.startswith("template <typename T>\n__global__ void k_one(")
    assert one.rstrip().endswith("}") and "k_two" not in one
    two = bench.kernel_source(SRC, "k_two")
    assert two.startswith("__global__ void k_two(") and "k_one" not in two
    assert bench.kernel_source(SRC, "k_three") is None


def test_traffic_entries_carry_a_figure_and_a_kernel_hash():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        tr = json.load(f)
    assert tr
    for e in tr.values():
        assert e["dram_bytes_per_launch"] > 0 and len(e["source_sha256_16"]) == 16
    assert bench.ncu_traffic("k_vanka.cu", "k_vanka_sweep", "no such key") is None
    assert bench.ncu_traffic("k_vanka.cu", "no_such_kernel", "vanka_sweep_fp32_finest") is None
