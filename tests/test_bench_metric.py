"""The numerator of bench.py's throughput (space-time dofs per march) and the paper's
throughput its lid-driven lines compare against, pinned to the numbers Sec. 5.2 and
Table 3 print (tests/golden/dof_counts.txt).  CPU only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden", "dof_counts.txt")

# Table 3, n_sm = 1: wall time W in seconds of the march on 13,824 CPU ranks
TABLE3_W = {(4, 2): 149.4, (5, 2): 329.0, (4, 3): 629.4}


def _golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                c, r, _, per_slab, total = line.split()
                rows[(int(c), int(r))] = (None if per_slab == "-" else int(per_slab), int(total))
    return rows


def test_slab_dofs_match_the_papers_counts():
    """slab_dofs(w) x (16 * 2^c slabs) is Table 3's global space-time dof count for every
    printed (c, r), and the per-slab count Sec. 5.2 prints where it prints one."""
    for (c, r), (per_slab, total) in _golden().items():
        n = 2 ** c
        D = bench.slab_dofs(dict(dim=3, n_cells=n, r=r, k=r))
        if per_slab is not None:
            assert D == per_slab
        assert D * 16 * n == total


@pytest.mark.parametrize("name,c,r", [("lid", 4, 2), ("lid5", 5, 2), ("lid_r3", 4, 3)])
def test_lid_workloads_are_table3_rows(name, c, r):
    """Each lid-driven workload is the Table 3 row it is compared with: mesh 2^c, Q_{r+1}/P_r,
    DG(r), 16 * 2^c slabs on [0, 8]; its whole march has Table 3's dof count, and the
    paper's throughput it divides by is that count over Table 3's wall time."""
    w = bench.WORKLOADS[name][0]
    assert (w["dim"], w["n_cells"], w["r"], w["k"], w["T"], w["n_slabs"]) == (3, 2 ** c, r, r, 8.0, 16 * 2 ** c)
    total = _golden()[(c, r)][1]
    assert bench.slab_dofs(w) * w["n_slabs"] == total
    assert bench.PAPER_THETA[name] == pytest.approx(total / TABLE3_W[(c, r)], rel=1e-12)


def test_headline_workload_size():
    """64x64 Q3/P2 DG(2): 3 (2 * 193^2 + 6 * 64^2) = 297,222 dofs per slab (Eq. DefX layout)."""
    w = bench.WORKLOADS["c2"][0]
    assert bench.slab_dofs(w) == 3 * (2 * 193 ** 2 + 6 * 64 ** 2) == 297222
    assert bench.aggregate_value(1, w["n_slabs"], bench.slab_dofs(w), 1000.0) == 16 * 297222


def test_sweep_bytes_of_the_headline_finest_level():
    """The roofline's algorithmic bytes per finest-level FP32 sweep: n_patches B^2 4 + 3 D 4,
    with the patch count and size of the library's own patch tables (4096 cells; B = 114,
    the Q3/P2 DG(2) cell patch of Table 2(b)), and the 9 distinct patch matrices of a
    uniform mesh (interior, 4 edges, 4 corners)."""
    import paper_2502_09159_gb300 as p
    p.build()
    w = bench.WORKLOADS["c2"][0]
    hp = p.host_patch(2, 64, 2, 2, 1.0, 1.0 / 16, p.CELL, 0, with_inverse=False)
    assert (hp["B"], hp["n_patches"], hp["n_classes"]) == (114, 4096, 9)
    level = {"n_patches": hp["n_patches"], "patch_size": hp["B"], "size": bench.slab_dofs(w)}
    assert bench.sweep_alg_bytes(level, "fp32") == 216493128
    assert bench.sweep_alg_bytes(level, "fp64") == 2 * 216493128


def test_parity_key_ignores_only_the_pressure_constants():
    """The bench line's `parity` compares slab 1 with the oracle's after removing the
    pressure mean of each temporal dof: a constant added to the pressure of one temporal
    dof (mode 0 of every cell) leaves the error at zero; any other change is reported."""
    import math
    import numpy as np
    w = bench.WORKLOAD
    d, n, r, k = w["dim"], w["n_cells"], w["r"], w["k"]
    D = bench.slab_dofs(w)
    nv, npm, kt = d * ((r + 1) * n + 1) ** d, math.comb(r + d, d), k + 1
    rng = np.random.default_rng(0)
    ref = rng.standard_normal(D)
    x = ref.copy()
    for a in range(kt):                                  # p += c_a on temporal dof a
        x[kt * nv + a * npm * n ** d:kt * nv + (a + 1) * npm * n ** d:npm] += 3.0 * (a + 1)
    out = bench.parity_against_oracle(ref, x, None)
    assert out["fp32_vcycle"]["rel_err_max"] < 1e-14 and "fp64_vcycle" not in out
    y = x.copy()
    y[kt * nv + 1] += 1e-3                               # a non-constant pressure mode
    y[5] -= 2e-3                                         # a velocity entry
    e = bench.parity_against_oracle(ref, x, y)["fp64_vcycle"]
    assert abs(e["rel_err_max"] - 2e-3 / np.abs(ref).max()) < 1e-9
    assert e["rel_err_velocity_l2"] > 0 and e["rel_err_pressure_l2"] > 0


def test_clock_samples_summary():
    """The `clocks` key from nvidia-smi rows: median SM clock under load, the maximum, and
    every throttle reason that was active in any sample (unreadable values skipped)."""
    rows = ["0, 2070, 2070, 655.20, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
            "0, 1980, 2070, 1391.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
            "0, 2070, 2070, 1380.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
            "0, [N/A], 2070, [N/A], [N/A], Not Active, Not Active, Not Active, Not Active\n",
            "garbage line\n"]
    s = bench.summarise_clocks(rows)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    s = bench.summarise_clocks(rows[:1] + ["0, 1500, 2070, 700, 0x8, Active, Active, Not Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and s["sm_mhz"] == 1785.0
    assert bench.summarise_clocks([]) is None and bench.summarise_clocks(["a, b"]) is None
