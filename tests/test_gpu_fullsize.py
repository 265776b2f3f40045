"""Oracle parity at the full size of the 2D headline configuration, on the hierarchy,
launch shapes and code paths that bench.py times.

Workload: 64x64 cells, Q3/P2disc (r = 2), DG(2), 16 slabs (tau = 1/16), nu = 1; the
hierarchy of Alg. 2/3 with h_0 = 1/8 and DG(2) on every level:
(64, 2, 2) -> (64, 1, 2) -> (32, 1, 2) -> (16, 1, 2) -> (8, 1, 2), the last solved
directly (D = 2310: the tiled FP64 coarse product).  The handles are tuned as in the bench
(autotune on, V-cycles captured in CUDA graphs), so the tuned patches-per-block shape of
the 4096-patch finest sweep, its evict-first inverse stream (217 MB of FP32 inverses, more
than L2 holds) and the tuned transfer forms are the ones compared.

The oracle assembles this exact system (scipy.sparse, FP64) and its cell-Vanka inverses
(numpy, per patch) in about 15-20 s.  Tolerances are those of tests/test_gpu_parity.py:
FP64 1e-12 (apply, residual, sweep, transfers, coarse solve), 1e-11 (V-cycle); FP32 2e-6
(apply, transfers), 1e-5 (sweep), 1e-4 (V-cycle); a slab solved to 1e-12 agrees with the
oracle's FGMRES + V-cycle solution at 1e-12 to 1e-9 (pressure mean removed).
"""
import numpy as np
import pytest

from oracle.stokes import MGConfig, Multigrid, default_hierarchy, fgmres
from workloads import fourier_forcing_2d, random_vector

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402

stmg.build()

N, R, K, NU, T, SLABS, COARSE_N = 64, 2, 2, 1.0, 1.0, 16, 8
TAU = T / SLABS


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dev(v, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dtype)


def free_vec(slab, seed):
    v = random_vector(slab.size, seed)
    v[slab.dirichlet] = 0.0
    return v


@pytest.fixture(scope="module")
def oracle():
    levels = default_hierarchy(N, R, K, COARSE_N, K)
    return Multigrid(2, levels, NU, TAU, MGConfig())


@pytest.fixture(scope="module")
def gpu():
    """The bench's handle: FP32 V-cycle in FP64 FGMRES, both precisions set up, tuned."""
    g = stmg.SpaceTimeMG(dim=2, n_cells=N, r=R, k=K, nu=NU, T=T, n_slabs=SLABS, precond_precision="fp32",
                         coarse_n=COARSE_N, k_min=K, precisions=("fp64", "fp32"))
    yield g
    g.close()


def test_hierarchy_is_the_benched_one(oracle, gpu):
    assert [(l["n"], l["r"], l["k"]) for l in gpu.levels] == [tuple(l[:3]) for l in oracle.levels]
    assert [l["size"] for l in gpu.levels] == [s.size for s in oracle.slabs]
    assert gpu.levels[0]["size"] == 297222 and gpu.levels[-1]["size"] == 2310
    fin = gpu.levels[0]
    assert fin["n_patches"] == 4096 and fin["patch_size"] == 114
    assert fin["inverse_bytes"][1] > 129e6 and fin["streaming"] == 1    # evict-first stream on the finest level


def test_apply_and_residual_every_level(oracle, gpu):
    for l, s in enumerate(oracle.slabs):
        x = random_vector(s.size, 300 + l)
        b = random_vector(s.size, 340 + l)
        ref = s.S @ x
        assert rel(gpu.apply(dev(x), l), ref) < 1e-12
        assert rel(gpu.residual(dev(b), dev(x), l), b - ref) < 1e-12
        assert rel(gpu.apply(dev(x, torch.float32), l).double(), ref) < 2e-6
        assert rel(gpu.residual(dev(b, torch.float32), dev(x, torch.float32), l).double(), b - ref) < 2e-6


def test_sweep_every_level_tuned_shape(oracle, gpu):
    for l, (s, W) in enumerate(zip(oracle.slabs[:-1], oracle.smoothers)):
        res = free_vec(s, 370 + l)
        ref = W.omega * W.correction(res)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(gpu.vanka_sweep(dev(res), x, l), ref) < 1e-12
        x32 = torch.zeros(s.size, dtype=torch.float32, device="cuda")
        assert rel(gpu.vanka_sweep(dev(res, torch.float32), x32, l).double(), ref) < 1e-5
        b, x0 = free_vec(s, 380 + l), free_vec(s, 390 + l)
        assert rel(gpu.smooth(dev(b), dev(x0), l, steps=1), W.step(b, x0)) < 1e-12
    gpu.device_status()


def test_transfers_every_level_pair(oracle, gpu):
    for l in range(len(oracle.slabs) - 1):
        P = oracle.P[l]
        fine, coarse = oracle.slabs[l], oracle.slabs[l + 1]
        r_f = random_vector(fine.size, 400 + l)
        assert rel(gpu.restrict(dev(r_f), l), P.T @ r_f) < 1e-12
        assert rel(gpu.restrict(dev(r_f, torch.float32), l).double(), P.T @ r_f) < 2e-6
        y_c = random_vector(coarse.size, 410 + l)
        x_f = free_vec(fine, 420 + l)
        assert rel(gpu.prolongate_add(dev(y_c), dev(x_f), l), x_f + P @ y_c) < 1e-12
        out = gpu.prolongate_add(dev(y_c, torch.float32), dev(x_f, torch.float32), l).double()
        assert rel(out, x_f + P @ y_c) < 2e-6


def test_coarse_solve_tiled(oracle, gpu):
    cs = oracle.slabs[-1]
    assert cs.size == 2310                              # > 1024: the tiled FP64 product
    bc = free_vec(cs, 430)
    ref = oracle.coarse_inv @ bc
    assert rel(gpu.coarse_solve(dev(bc)), ref) < 1e-12
    assert rel(gpu.coarse_solve(dev(bc, torch.float32)).double(), ref) < 2e-6


def test_vcycle_graph(oracle, gpu):
    b = free_vec(oracle.slabs[0], 440)
    ref = oracle.vcycle(b)
    for _ in range(2):                                  # capture, then replay
        assert rel(gpu.vcycle(dev(b), "fp64"), ref) < 1e-11
        assert rel(gpu.vcycle(dev(b), "fp32"), ref) < 1e-4


def test_slab_solve_against_the_oracle(oracle, gpu):
    """Slab 1 of the bench march (forcing of seeds 1, 2): the GPU solve to 1e-12 with the
    FP64 V-cycle equals the oracle's FGMRES + V-cycle solution to 1e-12 within 1e-9; the
    bench's solve (FP32 V-cycle, 1e-8) is within 1e-7 of it."""
    pb = fourier_forcing_2d(nu=NU)
    s0 = oracle.slabs[0]
    F = s0.rhs_forcing(pb.forcing, 0.0)
    xo, info_o = fgmres(lambda z: s0.S @ z, oracle.vcycle, F, tol=1e-12)
    assert info_o.converged
    ref = s0.remove_pressure_mean(xo)
    Fg = gpu.forcing(pb.forcing, 0)
    assert rel(Fg, F) < 1e-12
    g64 = stmg.SpaceTimeMG(dim=2, n_cells=N, r=R, k=K, nu=NU, T=T, n_slabs=SLABS, precond_precision="fp64",
                           coarse_n=COARSE_N, k_min=K, precisions=("fp64",), rel_tol=1e-12)
    x, info = g64.solve_slab(dev(F))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    assert rel(s0.remove_pressure_mean(x.cpu().numpy()), ref) < 1e-9
    g64.close()
    x32, info32 = gpu.solve_slab(gpu.slab_rhs(Fg))
    assert info32["status"] == 0 and info32["rel_residual"] <= 1e-8
    err = rel(s0.remove_pressure_mean(x32.cpu().numpy()), ref)
    assert err < 1e-7, err
