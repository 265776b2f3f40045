"""Vertex-star Vanka (the remark after Eq. vanka) against the oracle, through the C ABI.

Patches: all velocity dofs in the closure of the (up to 2^d) cells around a vertex and all
pressure modes of those cells, for every vertex including the boundary ones, all temporal
dofs of the slab; B = (k+1) (d (2 (r+1) + 1)^d + 2^d C(r+d, d)) for an interior vertex.

  * 2D Q3/P2disc DG(2): B = 366, the vertex-star configuration of the 64x64 workload
    (same patch matrices up to h), on a 4x4 mesh with vertex stars on every smoothed level;
  * 3D Q2/P1disc DG(1) on 2x2x2 cells: B = 814, the centre star covers the whole mesh
    (singular in the pressure constants, inverted bordered);
  * 3D Q2/P1disc DG(0) on 4x4x4 cells: B = 407, 125 stars.

Tolerances: sweep and smoothing step FP64 1e-12 / FP32 1e-5, V-cycle FP64 1e-11 / FP32 1e-4.
The reading of the vertex-star sets is the oracle's (pinned by closed-form counts in
tests/test_oracle_pins.py); it is not pinned against the paper's Table 2(d).
"""
import numpy as np
import pytest

from oracle.stokes import MGConfig, Multigrid
from workloads import random_vector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402

stmg.build()

NU, TAU = 0.9, 0.2
CASES = [(2, 4, 2, 2, 366), (3, 2, 1, 1, 814), (3, 4, 1, 0, 407)]
IDS = ["2d-n4-q3p2-dg2-B366", "3d-n2-q2p1-dg1-B814", "3d-n4-q2p1-dg0-B407"]


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dev(v, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dtype)


def free_vec(slab, seed):
    v = random_vector(slab.size, seed)
    v[slab.dirichlet] = 0.0
    return v


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_vertex_star_sweep_and_vcycle(case):
    dim, n, r, k, B = case
    levels = stmg.host_default_hierarchy(n, r, k)
    og = Multigrid(dim, levels, NU, TAU, MGConfig(smoother="vsp"))
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                         smoothers=[stmg.VSP] * len(levels))
    assert g.levels[0]["patch_size"] == B
    assert g.levels[0]["n_patches"] == (n + 1) ** dim
    assert max(len(p) for p in og.smoothers[0].patches) == B
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        assert g.levels[l]["smoother"] == stmg.VSP
        res = free_vec(s, 500 + l)
        ref = W.omega * W.correction(res)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(g.vanka_sweep(dev(res), x, l), ref) < 1e-12
        x32 = torch.zeros(s.size, dtype=torch.float32, device="cuda")
        assert rel(g.vanka_sweep(dev(res, torch.float32), x32, l).double(), ref) < 1e-5
        b, x0 = free_vec(s, 510 + l), free_vec(s, 520 + l)
        assert rel(g.smooth(dev(b), dev(x0), l, steps=1), W.step(b, x0)) < 1e-12
    b = free_vec(og.slabs[0], 530)
    ref = og.vcycle(b)
    for _ in range(2):                                  # graph capture, then replay
        assert rel(g.vcycle(dev(b), "fp64"), ref) < 1e-11
        assert rel(g.vcycle(dev(b), "fp32"), ref) < 1e-4
    g.device_status()
    g.close()
