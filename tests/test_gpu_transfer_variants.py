"""The two forms of the grid transfers (App. A: P and P^T of Eq. DeftTps / DefoTsl) on the
GPU against the FP64 oracle, each form forced through cfg.transfer_variant:
  1  per coarse cell (shared-memory sum factorisation, atomics on shared fine nodes),
  2  gather form, one thread per output value (2D levels; 3D levels keep form 1).
Tolerances as in the parity tests: FP64 1e-12, FP32 2e-6, FP64 V-cycle 1e-11.  Needs a GPU."""
import numpy as np
import pytest

from oracle.stokes import MGConfig, Multigrid
from workloads import random_vector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402

NU, TAU = 0.9, 0.2

# (dim, n, r, k, levels, n_sub): every 2D shape of the gather form -- Q3->Q2, Q4->Q2 and
# Q5->Q3 on one mesh, Q2 n -> n/2 (also from a ragged 6 -> 3), Q2 -> Q2 with DG(2) -> DG(1)
# in time, a macro step of two subintervals -- and one 3D hierarchy (form 1 kept)
CASES = [
    (2, 4, 2, 2, None, 1),
    (2, 4, 3, 0, None, 1),
    (2, 2, 4, 3, None, 1),
    (2, 6, 1, 1, [(6, 1, 1), (3, 1, 1)], 1),
    (2, 4, 1, 2, [(4, 1, 2), (4, 1, 1), (2, 1, 1), (1, 1, 1)], 1),
    (2, 4, 2, 1, None, 2),
    (3, 2, 2, 1, None, 1),
]
IDS = ["2d-q3q2-dg2", "2d-q4q2-dg0", "2d-q5q3-dg3", "2d-h-ragged", "2d-time-only", "2d-macro2", "3d-fallback"]


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dev(v, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dtype)


def free_vec(slab, seed):
    v = random_vector(slab.size, seed)
    v[slab.dirichlet] = 0.0
    return v


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def oracle_case(request):
    dim, n, r, k, levels, nsub = request.param
    levels = levels or stmg.host_default_hierarchy(n, r, k)
    og = Multigrid(dim, levels, NU, TAU, MGConfig(), nsub=nsub)
    return request.param, levels, og


@pytest.mark.parametrize("variant", [1, 2])
def test_transfer_forms_match_oracle(oracle_case, variant):
    (dim, n, r, k, _, nsub), levels, og = oracle_case
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * nsub * 5, n_slabs=5, levels=levels,
                         n_sub=nsub, use_graphs=False, transfer_variant=variant)
    try:
        for l in range(len(og.slabs) - 1):
            tcpb = g.levels[l]["transfer_cells_per_block"]
            if variant == 2 and dim == 2:
                assert tcpb == (0, 0)                 # the gather form is in use
            else:
                assert min(tcpb) >= 1
            P = og.P[l]
            fine, coarse = og.slabs[l], og.slabs[l + 1]
            r_f = random_vector(fine.size, 17 + l)
            assert rel(g.restrict(dev(r_f), l), P.T @ r_f) < 1e-12
            assert rel(g.restrict(dev(r_f, torch.float32), l).double(), P.T @ r_f) < 2e-6
            # the gather form writes every coarse value: stale output must not leak through
            stale = torch.full((coarse.size,), 7.0, dtype=torch.float64, device="cuda")
            assert rel(g.restrict(dev(r_f), l, out=stale), P.T @ r_f) < 1e-12
            y_c = random_vector(coarse.size, 19 + l)
            x_f = free_vec(fine, 23 + l)
            assert rel(g.prolongate_add(dev(y_c), dev(x_f), l), x_f + P @ y_c) < 1e-12
            x32 = dev(x_f, torch.float32)
            assert rel(g.prolongate_add(dev(y_c, torch.float32), x32, l).double(), x_f + P @ y_c) < 2e-6
        b = free_vec(og.slabs[0], 31)
        ref = og.vcycle(b)
        assert rel(g.vcycle(dev(b), "fp64"), ref) < 1e-11
        assert rel(g.vcycle(dev(b), "fp32"), ref) < 1e-4
    finally:
        g.close()


def test_forms_agree_on_the_bench_hierarchy():
    """64x64 Q3/P2, DG(2), levels 64 (Q3, Q2), 32, 16, 8: the two forms give the same
    FP64 V-cycle up to rounding, and FGMRES with the FP32 V-cycle converges in the same
    number of iterations (to within one: the rounding of the two forms differs)."""
    kw = dict(dim=2, n_cells=64, r=2, k=2, nu=1.0, T=1.0, n_slabs=16, coarse_n=8, k_min=2,
              precond_precision="fp32")
    g1 = stmg.SpaceTimeMG(**kw, transfer_variant=1)
    g2 = stmg.SpaceTimeMG(**kw, transfer_variant=2)
    try:
        assert all(lv["transfer_cells_per_block"] == (0, 0) for lv in g2.levels[:-1])
        b = dev(random_vector(g1.size(0), 5))
        v1, v2 = g1.vcycle(b, "fp64"), g2.vcycle(b, "fp64")
        assert rel(v2, v1.cpu().numpy()) < 1e-12
        # a consistent right-hand side (S has the pressure constants in its kernel)
        x = random_vector(g1.size(0), 6)
        rhs = g1.apply(dev(x))
        _, i1 = g1.solve_slab(rhs)
        _, i2 = g2.solve_slab(rhs)
        assert i1["status"] == 0 and i2["status"] == 0
        assert i1["rel_residual"] <= 1.001e-8 and i2["rel_residual"] <= 1.001e-8
        assert abs(i1["iterations"] - i2["iterations"]) <= 1
    finally:
        g1.close()
        g2.close()
