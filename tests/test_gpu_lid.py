"""Non-homogeneous Dirichlet data on the GPU (stmg_dirichlet_lift, boundary values in the
slab coupling) against the oracle, exact reproduction, and a small lid-driven cavity run
(Sec. 5.2) marched on both sides.  Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.stokes import Slab, errors, march
from workloads import lid_driven_3d, polynomial_boundary, random_vector

pytestmark = pytest.mark.gpu

import paper_2502_09159_gb300 as stmg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dim,n,r,k,precs", [(2, 3, 2, 1, ("fp64", "fp32")), (2, 4, 1, 2, ("fp32",)),
                                             (3, 2, 2, 1, ("fp32",))])
def test_lift_matches_oracle(dim, n, r, k, precs):
    """Also on handles set up for the FP32 V-cycle only (their finest FP64 operator is the
    one FGMRES uses)."""
    slab = Slab(dim, n, r, k, 0.8, 0.125)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=0.8, T=1.0, n_slabs=8, levels=[(n, r, k)],
                         use_graphs=False, autotune=False, precisions=precs, precond_precision=precs[-1])
    gv, b = random_vector(slab.size, 1), random_vector(slab.size, 2)
    assert rel(g.dirichlet_lift(dev(gv), dev(b)), slab.lift(gv, b)) < 1e-12
    # homogeneous data: interior rows unchanged, boundary rows zero
    gz = np.where(slab.dirichlet, 0.0, gv)
    assert rel(g.dirichlet_lift(dev(gz), dev(b)), np.where(slab.dirichlet, 0.0, b)) < 1e-15
    g.close()


def test_boundary_vector_matches_oracle():
    pb = polynomial_boundary(3)
    slab = Slab(3, 2, 2, 1, 1.0, 0.25)
    g = stmg.SpaceTimeMG(dim=3, n_cells=2, r=2, k=1, T=1.0, n_slabs=4, use_graphs=False, autotune=False)
    ref = slab.boundary_vector(pb.boundary, 2 * 0.25)
    assert rel(g.boundary_vector(pb.boundary, 2), ref) < 1e-14
    g.close()


@pytest.mark.parametrize("dim,n,r,k,prec", [(2, 4, 2, 1, "fp64"), (2, 8, 1, 1, "fp32"), (3, 2, 1, 1, "fp64")])
def test_exact_reproduction_with_boundary_data(dim, n, r, k, prec):
    """v = t (y^2, x^2[, ...]), p = t (x - 1/2): the GPU march with lifted boundary data
    reproduces the field to the solver tolerance."""
    N = 3
    pb = polynomial_boundary(dim, nu=0.6)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=0.6, T=1.0, n_slabs=N, precond_precision=prec,
                         rel_tol=1e-12)
    slab = Slab(dim, n, r, k, 0.6, 1.0 / N)
    x = None
    sols = []
    for s in range(N):
        b = g.dirichlet_lift(g.boundary_vector(pb.boundary, s), g.slab_rhs(g.forcing(pb.forcing, s), x))
        x, info = g.solve_slab(b)
        assert info["status"] == 0
        sols.append(x.cpu().numpy())
    e = errors(pb, slab, sols)
    assert e["v_L2L2"] < 1e-9 and e["v_L2H1"] < 1e-8 and e["p_L2L2"] < 1e-8
    g.close()


def test_lid_driven_cavity_small_matches_oracle():
    """Lid-driven cavity on 2^3 cells, Q2/P1, DG(1), the first 4 of 16 slabs on [0, 8]."""
    pb = lid_driven_3d()
    n, r, k, N, run = 2, 1, 1, 16, 4
    sols_o, _, slab, _ = march(pb, n, r, k, N, solver="direct", slabs_to_run=run)
    g = stmg.SpaceTimeMG(dim=3, n_cells=n, r=r, k=k, nu=1.0, T=8.0, n_slabs=N, rel_tol=1e-12)
    F = g.zeros(0)
    x = None
    for s in range(run):
        b = g.dirichlet_lift(g.boundary_vector(pb.boundary, s), g.slab_rhs(F, x))
        x, info = g.solve_slab(b)
        assert info["status"] == 0
        got = slab.remove_pressure_mean(x.cpu().numpy())
        assert rel(got, slab.remove_pressure_mean(sols_o[s])) < 1e-9
    g.close()


def test_march_host_boundary_data_matches_oracle():
    """The same cavity through stmg_march_host (host boundary data in, host solutions out,
    copies overlapped with the solves) against the oracle's direct march."""
    pb = lid_driven_3d()
    n, r, k, N, run = 2, 1, 1, 16, 4
    sols_o, _, slab, _ = march(pb, n, r, k, N, solver="direct", slabs_to_run=run)
    g = stmg.SpaceTimeMG(dim=3, n_cells=n, r=r, k=k, nu=1.0, T=8.0, n_slabs=N, rel_tol=1e-12)
    G = np.stack([g.boundary_vector(pb.boundary, s).cpu().numpy() for s in range(run)])
    X = np.full_like(G, np.nan)
    infos = g.march_host(G, X, boundary_data=True)
    assert [i["status"] for i in infos] == [0] * run
    for s in range(run):
        assert rel(slab.remove_pressure_mean(X[s]), slab.remove_pressure_mean(sols_o[s])) < 1e-9
    g.close()
