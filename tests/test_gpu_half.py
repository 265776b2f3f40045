"""FP32 V-cycle with half-precision patch inverses (FP16 rows scaled to [-1, 1], FP32 row
scales): the sweep and the V-cycle against the FP64 oracle at FP16 tolerances, and FGMRES
still reaching its FP64 tolerance.  Needs a GPU."""
import numpy as np
import pytest

from oracle.stokes import MGConfig, Multigrid, Slab
from workloads import manufactured_2d, random_vector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402

NU, TAU = 0.9, 0.2
CASES = [(2, 4, 2, 2), (2, 3, 1, 1), (3, 2, 2, 1)]


def rel(a, b):
    a = a.detach().cpu().numpy().astype(np.float64) if hasattr(a, "detach") else np.asarray(a)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def free_vec(slab, seed):
    v = random_vector(slab.size, seed)
    v[slab.dirichlet] = 0.0
    return v


@pytest.mark.parametrize("case", CASES, ids=["2d-r2k2", "2d-n3-r1k1", "3d-r2k1"])
def test_half_inverse_sweep_and_vcycle(case):
    dim, n, r, k = case
    levels = stmg.host_default_hierarchy(n, r, k) if n & (n - 1) == 0 else [(n, r, k), (n, 1, 1)]
    og = Multigrid(dim, levels, NU, TAU, MGConfig())
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                         precisions=("fp32",), precond_precision="fp32", half_inverses=True, use_graphs=False)
    g32 = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                           precisions=("fp32",), precond_precision="fp32", use_graphs=False)
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        res = free_vec(s, 7 + l)
        ref = W.omega * W.correction(res)
        x = torch.zeros(s.size, dtype=torch.float32, device="cuda")
        assert rel(g.vanka_sweep(torch.from_numpy(res).to("cuda", torch.float32), x, l), ref) < 3e-3
        # about half the bytes of the FP32 inverses
        assert g.levels[l]["inverse_bytes"][1] < 0.6 * g32.levels[l]["inverse_bytes"][1]
    b = free_vec(og.slabs[0], 31)
    ref = og.vcycle(b)
    assert rel(g.vcycle(torch.from_numpy(b).to("cuda"), "fp32"), ref) < 1e-2
    g.close()
    g32.close()


def test_half_inverses_reach_the_fp64_tolerance():
    """Config-1 field on 8x8, Q2/P1, DG(1): FGMRES with the half-inverse V-cycle reaches
    1e-10 in at most two more iterations than with FP32 inverses, and the solutions agree."""
    pb = manufactured_2d(nu=1.0, time="sin_pi")
    kw = dict(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=4, precond_precision="fp32", rel_tol=1e-10)
    gh = stmg.SpaceTimeMG(half_inverses=True, **kw)
    gf = stmg.SpaceTimeMG(**kw)
    slab = Slab(2, 8, 1, 1, 1.0, 0.25)
    xh = xf = None
    for s in range(4):
        bh = gh.slab_rhs(gh.forcing(pb.forcing, s), xh)
        xh, ih = gh.solve_slab(bh)
        xf, i_f = gf.solve_slab(gf.slab_rhs(gf.forcing(pb.forcing, s), xf))
        assert ih["status"] == 0 and ih["rel_residual"] <= 1e-10
        assert ih["iterations"] <= i_f["iterations"] + 2
        a = slab.remove_pressure_mean(xh.cpu().numpy())
        c = slab.remove_pressure_mean(xf.cpu().numpy())
        assert rel(a, c) < 1e-8
    gh.close()
    gf.close()
