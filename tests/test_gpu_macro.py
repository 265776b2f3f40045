"""Macro time steps (Remark rem:GLSP): systems of n_sub DG(k) subintervals on the GPU
against the FP64 oracle, through the C ABI.  Needs a GPU."""
import numpy as np
import pytest

from oracle.stokes import MGConfig, Multigrid, errors, march
from workloads import manufactured_2d, polynomial_2d, random_vector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402

NU, TAU = 0.9, 0.2
# (dim, n, r, k, n_sub): n_sub (k+1) up to 8 temporal dofs per system
CASES = [(2, 4, 2, 1, 2), (2, 4, 1, 0, 3), (2, 2, 1, 3, 2), (3, 2, 1, 1, 2)]
IDS = ["2d-r2k1-x2", "2d-r1k0-x3", "2d-r1k3-x2", "3d-r1k1-x2"]


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
def case(request):
    dim, n, r, k, nsub = request.param
    levels = stmg.host_default_hierarchy(n, r, k)
    og = Multigrid(dim, levels, NU, TAU, MGConfig(), nsub=nsub)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * nsub * 5, n_slabs=5, n_sub=nsub,
                         use_graphs=False)
    yield og, g
    g.close()


def test_apply_sweep_transfers_match_oracle(case):
    og, g = case
    for l, s in enumerate(og.slabs):
        assert g.size(l) == s.size
        x = random_vector(s.size, 3 + l)
        assert rel(g.apply(dev(x), l), s.S @ x) < 1e-12
        assert rel(g.apply_transpose(dev(x), l), s.S.T @ x) < 1e-12
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        res = free_vec(s, 7 + l)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(g.vanka_sweep(dev(res), x, l), W.omega * W.correction(res)) < 1e-12
        P = og.P[l]
        r_f = random_vector(s.size, 17 + l)
        assert rel(g.restrict(dev(r_f), l), P.T @ r_f) < 1e-12
        y_c = random_vector(og.slabs[l + 1].size, 19 + l)
        x_f = free_vec(s, 23 + l)
        assert rel(g.prolongate_add(dev(y_c), dev(x_f), l), x_f + P @ y_c) < 1e-12


def test_vcycle_matches_oracle(case):
    og, g = case
    b = free_vec(og.slabs[0], 31)
    ref = og.vcycle(b)
    assert rel(g.vcycle(dev(b), "fp64"), ref) < 1e-11
    assert rel(g.vcycle(dev(b), "fp32"), ref) < 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_macro_march_matches_oracle_and_time_marching(prec):
    """Config-1 field on 8x8, Q2/P1, DG(1): 2 systems of 2 subintervals against the
    oracle's macro march, and against 4 steps of time marching on the GPU."""
    pb = manufactured_2d(nu=1.0, time="sin_pi")
    sols_o, _, slab, _ = march(pb, 8, 1, 1, 2, solver="direct", nsub=2)
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=2, n_sub=2, precond_precision=prec,
                         rel_tol=1e-12)
    g1 = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=4, rel_tol=1e-12)
    x, x1 = None, None
    marched = []
    for s in range(4):
        x1, info = g1.solve_slab(g1.slab_rhs(g1.forcing(pb.forcing, s), x1))
        assert info["status"] == 0
        marched.append(x1.cpu().numpy())
    for s in range(2):
        x, info = g.solve_slab(g.slab_rhs(g.forcing(pb.forcing, s), x))
        assert info["status"] == 0 and info["rel_residual"] <= 1e-12
        got = slab.remove_pressure_mean(x.cpu().numpy())
        assert rel(got, slab.remove_pressure_mean(sols_o[s])) < 1e-9
        for j in range(2):                               # subinterval j of system s = step 2 s + j
            for b_ in range(2):
                a = 2 * j + b_
                assert rel(slab.vel(got, a), marched[2 * s + j][b_ * g1.levels[0]["n_vel"]:
                                                              (b_ + 1) * g1.levels[0]["n_vel"]]) < 1e-9
    g.close()
    g1.close()


def test_macro_exact_reproduction():
    """v = t curl(x^2(1-x)^2 y^2(1-y)^2), p = t(x-1/2)(y-1/2) on 2x2 cells, Q4/P3, DG(1),
    two systems of two subintervals: reproduced to the solver tolerance."""
    pb = polynomial_2d(m=1, nu=0.7)
    g = stmg.SpaceTimeMG(dim=2, n_cells=2, r=3, k=1, nu=0.7, T=1.0, n_slabs=2, n_sub=2, rel_tol=1e-12)
    _, _, slab, _ = march(pb, 2, 3, 1, 2, solver="direct", nsub=2, slabs_to_run=1)
    x = None
    sols = []
    for s in range(2):
        x, info = g.solve_slab(g.slab_rhs(g.forcing(pb.forcing, s), x))
        assert info["status"] == 0
        sols.append(x.cpu().numpy())
    e = errors(pb, slab, sols)
    assert e["v_L2L2"] < 1e-9 and e["v_L2H1"] < 1e-8 and e["p_L2L2"] < 1e-8
    g.close()


# h-coarsening in time inside a macro step (App. A, Eq. DeftPrRe / DefTlspr): levels of
# fewer, longer subintervals; (n, r, k, n_sub) fine -> coarse
H_TIME_CASES = [
    (2, 4, 1, 1, 4, [(4, 1, 1, 4), (4, 1, 1, 2), (4, 1, 1, 1), (2, 1, 1, 1), (1, 1, 1, 1)]),
    (2, 4, 2, 1, 2, [(4, 2, 1, 2), (4, 1, 1, 1), (2, 1, 1, 1), (1, 1, 1, 1)]),       # h in time with p in space
    (2, 2, 1, 3, 2, [(2, 1, 3, 2), (2, 1, 3, 1), (2, 1, 1, 1), (1, 1, 1, 1)]),       # DG(3), then p in time
    (2, 4, 1, 0, 4, [(4, 1, 0, 4), (2, 1, 0, 2), (1, 1, 0, 1)]),                      # h in space and time together
    (3, 2, 1, 1, 2, [(2, 1, 1, 2), (2, 1, 1, 1), (1, 1, 1, 1)]),
]
H_TIME_IDS = ["2d-q2-dg1-x4-421", "2d-q3-dg1-x2-p", "2d-q2-dg3-x2", "2d-dg0-x4-hst", "3d-q2-dg1-x2"]


@pytest.mark.parametrize("hc", H_TIME_CASES, ids=H_TIME_IDS)
def test_h_in_time_levels_match_oracle(hc):
    """Operator, sweep and both transfers on every level pair, and the V-cycle, against the
    oracle's hierarchy with the same temporal meshes (FP64 1e-12 / 1e-11, FP32 2e-6 / 1e-4)."""
    dim, n, r, k, nsub, levels = hc
    og = Multigrid(dim, levels, NU, TAU, MGConfig(), nsub=nsub)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * nsub * 5, n_slabs=5, n_sub=nsub,
                         levels=levels, use_graphs=False)
    assert [l["n_sub"] for l in g.levels] == [l[3] for l in levels]
    for l, s in enumerate(og.slabs):
        assert g.size(l) == s.size
        x = random_vector(s.size, 53 + l)
        assert rel(g.apply(dev(x), l), s.S @ x) < 1e-12
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        res = free_vec(s, 57 + l)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(g.vanka_sweep(dev(res), x, l), W.omega * W.correction(res)) < 1e-12
        P = og.P[l]
        r_f = random_vector(s.size, 61 + l)
        assert rel(g.restrict(dev(r_f), l), P.T @ r_f) < 1e-12
        assert rel(g.restrict(dev(r_f, torch.float32), l).double(), P.T @ r_f) < 2e-6
        y_c = random_vector(og.slabs[l + 1].size, 67 + l)
        x_f = free_vec(s, 71 + l)
        assert rel(g.prolongate_add(dev(y_c), dev(x_f), l), x_f + P @ y_c) < 1e-12
    b = free_vec(og.slabs[0], 73)
    ref = og.vcycle(b)
    assert rel(g.vcycle(dev(b), "fp64"), ref) < 1e-11
    assert rel(g.vcycle(dev(b), "fp32"), ref) < 1e-4
    g.device_status()
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_h_in_time_default_hierarchy_solves_macro_march(prec):
    """time_h = 1: the default hierarchy first halves the subintervals (4 -> 2 -> 1) on the
    finest mesh; two macro systems of four subintervals, Q2/P1, DG(1) on 8x8 cells, solved
    to 1e-12, equal the oracle's direct macro march."""
    pb = manufactured_2d(nu=1.0, time="sin_pi")
    sols_o, _, slab, _ = march(pb, 8, 1, 1, 2, solver="direct", nsub=4)
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=2, n_sub=4, time_h=True,
                         precond_precision=prec, rel_tol=1e-12)
    assert [(l["n"], l["n_sub"]) for l in g.levels[:3]] == [(8, 4), (8, 2), (8, 1)]
    x = None
    for s in range(2):
        x, info = g.solve_slab(g.slab_rhs(g.forcing(pb.forcing, s), x))
        assert info["status"] == 0 and info["rel_residual"] <= 1e-12
        got = slab.remove_pressure_mean(x.cpu().numpy())
        assert rel(got, slab.remove_pressure_mean(sols_o[s])) < 1e-9
    g.close()
