"""GPU parity: every hot-path call of libstmg (through the C ABI) against the FP64 oracle
on the same seeded inputs.

Tolerances (relative, max-norm over max-norm of the reference):
  FP64 apply / residual / sweep / smoothing step / transfers / coarse solve: 1e-12
  FP64 V-cycle: 1e-11;  solves to 1e-12 agree to 1e-9 (pressure mean removed)
  FP32: apply / transfers 2e-6, sweep 1e-5, V-cycle 1e-4 (single-precision rounding
  of O(B) and O(levels) operations).
"""
import numpy as np
import pytest

from oracle.stokes import MGConfig, Multigrid, Slab, fgmres, march, slab_prolongation
from workloads import fourier_forcing_2d, manufactured_2d, random_vector, taylor_green_3d

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402

stmg.build()

NU, TAU = 0.9, 0.2


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dev(v, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dtype)


# (dim, n, r, k, explicit levels or None)
CASES = [
    (2, 4, 1, 1, None),
    (2, 3, 2, 2, [(3, 2, 2), (3, 1, 1)]),          # ragged: 9 cells
    (2, 4, 3, 0, None),                             # DG(0)
    (2, 2, 4, 3, None),                             # largest degrees
    (2, 5, 1, 1, [(5, 1, 1)]),                      # single level, odd n
    (3, 2, 1, 1, None),
    (3, 2, 2, 1, None),
    (3, 2, 3, 2, None),                             # 3D Q4/P3, DG(2)
    (3, 2, 4, 1, None),                             # 3D Q5/P4: largest spatial degree
]
IDS = ["2d-n4-r1k1", "2d-n3-r2k2", "2d-n4-r3k0", "2d-n2-r4k3", "2d-n5-single", "3d-n2-r1k1", "3d-n2-r2k1",
       "3d-n2-r3k2", "3d-n2-r4k1"]

_cache = {}


def setup_case(case, smoother="cell"):
    key = (case[:4], smoother)
    if key in _cache:
        return _cache[key]
    dim, n, r, k, levels = case
    levels = levels or stmg.host_default_hierarchy(n, r, k)
    og = Multigrid(dim, levels, NU, TAU, MGConfig(smoother=smoother))
    sm = [stmg.VSP if smoother == "vsp" else stmg.CELL] * len(levels)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                         smoothers=sm, use_graphs=False)
    _cache[key] = (og, g)
    return og, g


def free_vec(slab, seed):
    v = random_vector(slab.size, seed)
    v[slab.dirichlet] = 0.0
    return v


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_and_residual(case):
    og, g = setup_case(case)
    for l, s in enumerate(og.slabs):
        x = random_vector(s.size, 3 + l)
        b = random_vector(s.size, 40 + l)
        ref = s.S @ x
        assert rel(g.apply(dev(x), l), ref) < 1e-12
        assert rel(g.residual(dev(b), dev(x), l), b - ref) < 1e-12
        assert rel(g.apply(dev(x, torch.float32), l).double(), ref) < 2e-6
        assert rel(g.apply_transpose(dev(x), l), s.S.T @ x) < 1e-12
        assert rel(g.apply_transpose(dev(x, torch.float32), l).double(), s.S.T @ x) < 2e-6


def reg_supported(r, k, prec):
    """The register-resident 2D operator covers FP32 up to Q5 (r <= 3), FP64 up to Q3 (r <= 2)
    and k + 1 <= 4; other shapes fall back to the node-centred form when it is forced."""
    return k + 1 <= 4 and r <= (3 if prec == "fp32" else 2)


def pair_supported(r, k):
    """The pair-split register form covers Q3 (r = 2) with k + 1 <= 4, in both precisions;
    where it is forced on other levels they take the register-resident form."""
    return r == 2 and k + 1 <= 4


def forced_variant(variant, r, k, prec):
    if variant == 4 and pair_supported(r, k):
        return 4
    if variant in (3, 4):
        return 3 if reg_supported(r, k, prec) else 2
    return variant


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("case", [c for c in CASES if c[0] == 2], ids=[i for c, i in zip(CASES, IDS) if c[0] == 2])
def test_apply_variants_2d(case, variant):
    """Every operator kernel forced on every 2D level: the per-cell form (atomics on shared
    nodes), the node-centred form (tiles of 4x4 cells, ragged tiles on 3x3 / 5x5 meshes,
    every output written once) and the register-resident form (one thread per cell and
    temporal dof) and its pair-split form (two lanes per item, Q3 levels; ragged warps on the
    3x3 mesh): apply, residual, S^T and the lift against the oracle."""
    og, _ = setup_case(case)
    dim, n, r, k, levels = case
    levels = levels or stmg.host_default_hierarchy(n, r, k)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                         use_graphs=False, autotune=False, apply_variant=variant)
    for l, s in enumerate(og.slabs):
        lr, lk = levels[l][1], levels[l][2]
        want = tuple(forced_variant(variant, lr, lk, p) for p in ("fp64", "fp32"))
        assert g.levels[l]["apply_variant"] == want
        x = random_vector(s.size, 63 + l)
        b = random_vector(s.size, 67 + l)
        ref = s.S @ x
        y = torch.full((s.size,), float("nan"), dtype=torch.float64, device="cuda")   # every entry is written
        assert rel(g.apply(dev(x), l, out=y), ref) < 1e-12
        assert rel(g.residual(dev(b), dev(x), l), b - ref) < 1e-12
        assert rel(g.apply_transpose(dev(x), l), s.S.T @ x) < 1e-12
        assert rel(g.apply(dev(x, torch.float32), l).double(), ref) < 2e-6
        assert rel(g.residual(dev(b, torch.float32), dev(x, torch.float32), l).double(), b - ref) < 2e-6
    s0 = og.slabs[0]
    gv, bv = random_vector(s0.size, 71), random_vector(s0.size, 73)
    assert rel(g.dirichlet_lift(dev(gv), dev(bv)), s0.lift(gv, bv)) < 1e-12
    g.close()


@pytest.mark.parametrize("variant", [1, 3])
@pytest.mark.parametrize("case", CASES[:7], ids=IDS[:7])
def test_sweep_variants_against_oracle(case, variant):
    """The block sweep and the pipelined block sweep forced on every level (B <= 512 for the
    pipelined one; these cases have B <= 404) against the oracle's correction."""
    og, _ = setup_case(case)
    dim, n, r, k, levels = case
    levels = levels or stmg.host_default_hierarchy(n, r, k)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                         use_graphs=False, autotune=False, sweep_variant=variant)
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        assert g.levels[l]["sweep_variant"] == (variant, variant)
        res = free_vec(s, 77 + l)
        ref = W.omega * W.correction(res)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(g.vanka_sweep(dev(res), x, l), ref) < 1e-12
        x32 = torch.zeros(s.size, dtype=torch.float32, device="cuda")
        assert rel(g.vanka_sweep(dev(res, torch.float32), x32, l).double(), ref) < 1e-5
    g.device_status()
    g.close()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_vanka_sweep_and_smoothing_step(case):
    og, g = setup_case(case)
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        res = free_vec(s, 7 + l)
        ref = W.omega * W.correction(res)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(g.vanka_sweep(dev(res), x, l), ref) < 1e-12
        x32 = torch.zeros(s.size, dtype=torch.float32, device="cuda")
        assert rel(g.vanka_sweep(dev(res, torch.float32), x32, l).double(), ref) < 1e-5
        b, x0 = free_vec(s, 11 + l), free_vec(s, 13 + l)
        assert rel(g.smooth(dev(b), dev(x0), l, steps=1), W.step(b, x0)) < 1e-12
    g.device_status()


@pytest.mark.parametrize("case", [c for c in CASES if c[4] != [(5, 1, 1)]],
                         ids=[i for c, i in zip(CASES, IDS) if c[4] != [(5, 1, 1)]])
def test_transfers(case):
    og, g = setup_case(case)
    for l in range(len(og.slabs) - 1):
        P = og.P[l]
        fine, coarse = og.slabs[l], og.slabs[l + 1]
        r_f = random_vector(fine.size, 17 + l)
        assert rel(g.restrict(dev(r_f), l), P.T @ r_f) < 1e-12
        y_c = random_vector(coarse.size, 19 + l)
        x_f = free_vec(fine, 23 + l)
        assert rel(g.prolongate_add(dev(y_c), dev(x_f), l), x_f + P @ y_c) < 1e-12
        assert rel(g.restrict(dev(r_f, torch.float32), l).double(), P.T @ r_f) < 2e-6


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_coarse_solve_and_vcycle(case):
    og, g = setup_case(case)
    cs = og.slabs[-1]
    bc = free_vec(cs, 29)
    assert rel(g.coarse_solve(dev(bc)), og.coarse_inv @ bc) < 1e-12
    s0 = og.slabs[0]
    b = free_vec(s0, 31)
    ref = og.vcycle(b)
    assert rel(g.vcycle(dev(b), "fp64"), ref) < 1e-11
    assert rel(g.vcycle(dev(b), "fp32"), ref) < 1e-4


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sweep_variants_agree_full_size(dtype):
    """The bench workload's levels (64x64, Q3/P2, DG(2)): the persistent TMA-pipelined
    sweep and the tuner's choice equal the one-block-per-patch-group sweep."""
    gs = [stmg.SpaceTimeMG(dim=2, n_cells=64, r=2, k=2, n_slabs=16, sweep_variant=v, use_graphs=False,
                           precisions=("fp64",) if dtype == torch.float64 else ("fp32",),
                           precond_precision="fp64" if dtype == torch.float64 else "fp32") for v in (2, 1, 0, 3)]
    w = 1 if dtype == torch.float32 else 0
    assert gs[0].levels[0]["sweep_variant"][w] == 2 and gs[3].levels[0]["sweep_variant"][w] == 3
    for l in range(len(gs[0].levels) - 1):
        res = torch.from_numpy(random_vector(gs[0].size(l), 50 + l)).to("cuda", dtype)
        out = []
        for g in gs:
            x = torch.zeros_like(res)
            for _ in range(2):
                g.vanka_sweep(res, x, l)
            out.append(x)
        tol = 1e-13 if dtype == torch.float64 else 2e-6
        for o in (out[0], out[2], out[3]):              # TMA, tuned and pipelined against the block sweep
            assert ((o - out[1]).abs().max() / out[1].abs().max()).item() < tol
    for g in gs:
        g.device_status()
        g.close()


@pytest.mark.parametrize("coarse_n", [4, 8])
def test_vcycle_with_coarser_mesh_stop(coarse_n):
    """Alg. 2 with h_0 = 1/coarse_n: the coarsest level is an 8x8 (D = 1540, tiled FP64
    coarse product) or 4x4 mesh solved directly."""
    dim, n, r, k = 2, 16, 1, 1
    levels = stmg.host_default_hierarchy(n, r, k, coarse_n)
    og = Multigrid(dim, levels, NU, TAU, MGConfig())
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, coarse_n=coarse_n)
    assert [(l["n"], l["r"], l["k"]) for l in g.levels] == [tuple(x) for x in levels]
    cs = og.slabs[-1]
    bc = free_vec(cs, 51)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-6)):
        assert rel(g.coarse_solve(dev(bc, dt)).double(), og.coarse_inv @ bc) < tol
    b = free_vec(og.slabs[0], 53)
    ref = og.vcycle(b)
    assert rel(g.vcycle(dev(b), "fp64"), ref) < 1e-11
    assert rel(g.vcycle(dev(b), "fp32"), ref) < 1e-4


PERSIST_CASES = [
    (2, 4, 1, 1, None),                                     # levels 1.. : (2,1,1) smoothed, (1,1,1) coarse
    (2, 4, 3, 0, None),                                     # DG(0) below a p-step in space
    (2, 2, 4, 3, None),                                     # the Q2 levels under r = 4, k = 3
    (2, 16, 2, 2, [(16, 2, 2), (16, 1, 2), (8, 1, 2), (4, 1, 1), (2, 1, 1)]),   # p-in-time inside the kernel
]


@pytest.mark.parametrize("smoother", ["cell", "vsp"])
@pytest.mark.parametrize("case", PERSIST_CASES, ids=["2d-n4-r1k1", "2d-n4-r3k0", "2d-n2-r4k3", "2d-n16-r2k2-pt"])
def test_persistent_levels_vcycle(case, smoother):
    """The levels below the finest run in one persistent kernel (forced): V-cycles in both
    precisions against the oracle, graph and eager, and equal to one kernel per operation."""
    dim, n, r, k, levels = case
    levels = levels or stmg.host_default_hierarchy(n, r, k)
    og = Multigrid(dim, levels, NU, TAU, MGConfig(smoother=smoother))
    sm = [stmg.VSP if smoother == "vsp" else stmg.CELL] * len(levels)
    b = free_vec(og.slabs[0], 81)
    ref = og.vcycle(b)
    outs = {}
    for persistent in (2, 0):
        for graphs in (True, False):
            g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                                 smoothers=sm, use_graphs=graphs, persistent=persistent)
            flags = [l["persistent"] for l in g.levels]
            if persistent == 2:
                assert flags[0] == (0, 0) and flags[-1] == (1, 1), flags   # the finest level keeps its kernels
            else:
                assert all(f == (0, 0) for f in flags)
            for _ in range(2):                                  # capture, then replay
                x64, x32 = g.vcycle(dev(b), "fp64"), g.vcycle(dev(b), "fp32")
                assert rel(x64, ref) < 1e-11
                assert rel(x32, ref) < 1e-4
            outs[(persistent, graphs)] = (x64.cpu().numpy(), x32.cpu().numpy())
            g.device_status()
            g.close()
    for key in outs:
        assert rel(outs[key][0], outs[(0, False)][0]) < 1e-12


def test_persistent_levels_solve():
    """FGMRES with the persistent V-cycle (FP32) solves to 1e-10 and agrees with the solve
    that runs one kernel per operation."""
    pb = fourier_forcing_2d(nu=1.0)
    xs = []
    for persistent in (2, 0):
        g = stmg.SpaceTimeMG(dim=2, n_cells=16, r=2, k=2, nu=1.0, T=1.0, n_slabs=16, precond_precision="fp32",
                             coarse_n=4, k_min=2, rel_tol=1e-10, persistent=persistent)
        b = g.slab_rhs(g.forcing(pb.forcing, 0))
        x, info = g.solve_slab(b)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10
        xs.append((x.cpu().numpy(), info["iterations"]))
        g.close()
    assert abs(xs[0][1] - xs[1][1]) <= 1
    s0 = Slab(2, 16, 2, 2, 1.0, 1.0 / 16)
    assert rel(s0.remove_pressure_mean(xs[0][0]), s0.remove_pressure_mean(xs[1][0])) < 1e-8


@pytest.mark.parametrize("case", [c for c in CASES if c[0] == 2], ids=[i for c, i in zip(CASES, IDS) if c[0] == 2])
def test_fused_prolongation_residual(case):
    """The FP32 V-cycle with the transfers folded into the residuals (the default on
    register-resident 2D levels: the descent's residual restricted in the same launch, the
    coarser correction prolongated inside the first postsmoothing residual; Q3 <- Q2 and
    Q2 <- Q2 on one mesh, Q2 <- Q2 from half the cells, ragged 3x3 and 5x5 meshes among
    them) against the oracle's V-cycle (FP32 tolerance) and against the same V-cycle with
    separate kernels (FP32 roundings apart), twice in a row (the second V-cycle starts from
    the buffers the first left: the restriction must overwrite the coarse right-hand side
    and zero the coarse iterate again)."""
    og, _ = setup_case(case)
    dim, n, r, k, levels = case
    levels = levels or stmg.host_default_hierarchy(n, r, k)
    b = free_vec(og.slabs[0], 91)
    ref = og.vcycle(b)
    outs = {}
    for fuse in (True, False):
        g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, levels=levels,
                             use_graphs=False, autotune=False, apply_variant=3, precisions=("fp32",),
                             precond_precision="fp32", fuse_transfers=fuse)
        for rep in range(2):
            x = g.vcycle(dev(b), "fp32")
            assert rel(x, ref) < 1e-4
        outs[fuse] = x.cpu().numpy()
        g.device_status()
        g.close()
    assert rel(outs[True], outs[False]) < 2e-5


def test_vcycle_graph_equals_eager():
    case = CASES[0]
    dim, n, r, k, _ = case
    og, ge = setup_case(case)
    gg = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=NU, T=TAU * 5, n_slabs=5, use_graphs=True)
    b = dev(free_vec(og.slabs[0], 37))
    for prec in ("fp64", "fp32"):
        x1 = ge.vcycle(b, prec)
        for _ in range(3):                               # capture, then replays
            x2 = gg.vcycle(b, prec)
            assert rel(x2, x1.cpu().numpy()) < (1e-13 if prec == "fp64" else 1e-6)
    assert gg.kernel_launches > 0


@pytest.mark.parametrize("smoother", ["vsp"])
def test_vertex_star_smoother(smoother):
    case = (2, 4, 1, 1, None)
    og, g = setup_case(case, smoother)
    for l, (s, W) in enumerate(zip(og.slabs[:-1], og.smoothers)):
        res = free_vec(s, 41 + l)
        x = torch.zeros(s.size, dtype=torch.float64, device="cuda")
        assert rel(g.vanka_sweep(dev(res), x, l), W.omega * W.correction(res)) < 1e-12
    b = free_vec(og.slabs[0], 43)
    assert rel(g.vcycle(dev(b), "fp64"), og.vcycle(b)) < 1e-11


def test_solve_slab_matches_direct_solve():
    dim, n, r, k = 2, 8, 2, 1
    pb = manufactured_2d(nu=1.0)
    slab = Slab(dim, n, r, k, 1.0, 0.25)
    F = slab.rhs_forcing(pb.forcing, 0.0)
    xd = slab.direct_solve(F)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=1.0, T=1.0, n_slabs=4, rel_tol=1e-12)
    x, info = g.solve_slab(dev(F))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    xs = slab.remove_pressure_mean(x.cpu().numpy())
    assert rel(xs, slab.remove_pressure_mean(xd)) < 1e-9
    for a in range(slab.kt):
        assert np.abs(slab.B @ slab.vel(x.cpu().numpy(), a)).max() < 1e-10


def test_arnoldi_forms_agree():
    """The Arnoldi step in its two forms (w held in registers across the passes for up to 16
    basis vectors, else the split-pass form) on a solve of 25 iterations (the oracle's
    count with omega = 0.3 to 1e-12), so that the register form's 16 instances and the
    split form beyond them are all taken: the same iterations and solutions, and the
    oracle's solution to 1e-9."""
    pb = fourier_forcing_2d(nu=1.0)
    levels = stmg.host_default_hierarchy(8, 1, 1)
    og = Multigrid(2, levels, 1.0, 0.25, MGConfig(omega=0.3))
    s0 = og.slabs[0]
    F = s0.rhs_forcing(pb.forcing, 0.0)
    xo, info_o = fgmres(lambda z: s0.S @ z, og.vcycle, F, tol=1e-12)
    assert info_o.converged and info_o.iterations > 16
    out = []
    for form in (0, 1):
        g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=4, levels=levels, omega=0.3,
                             rel_tol=1e-12, precisions=("fp64",), arnoldi_form=form)
        x, info = g.solve_slab(dev(F))
        assert info["status"] == 0 and info["rel_residual"] <= 1e-12
        out.append((s0.remove_pressure_mean(x.cpu().numpy()), info["iterations"]))
        g.device_status()
        g.close()
    assert out[0][1] == out[1][1] and abs(out[0][1] - info_o.iterations) <= 1
    assert rel(out[0][0], out[1][0]) < 1e-12
    assert rel(out[0][0], s0.remove_pressure_mean(xo)) < 1e-9


def test_forcing_and_slab_rhs():
    dim, n, r, k = 2, 4, 2, 2
    pb = fourier_forcing_2d(nu=1.0)
    slab = Slab(dim, n, r, k, 1.0, 1.0 / 16)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=1.0, T=1.0, n_slabs=16)
    F = g.forcing(pb.forcing, slab=3)
    Fo = slab.rhs_forcing(pb.forcing, 3 / 16)
    assert rel(F, Fo) < 1e-12
    x_prev = free_vec(slab, 47)                         # a previous solution: zero on the boundary
    b = g.slab_rhs(F, dev(x_prev))
    ref = Fo + slab.coupling(slab.vel(x_prev, slab.kt - 1))
    assert rel(b, ref) < 1e-12
    x_any = random_vector(slab.size, 47)                # boundary values enter the jump term too
    ref_any = Fo + slab.coupling(slab.vel(x_any, slab.kt - 1))
    assert rel(g.slab_rhs(F, dev(x_any)), ref_any) < 1e-12
    assert torch.equal(g.slab_rhs(F), F)                # no previous slab: b is F itself


def test_forcing_3d():
    pb = taylor_green_3d(nu=1e-2)
    slab = Slab(3, 2, 2, 1, 1e-2, 1.0 / 8)
    g = stmg.SpaceTimeMG(dim=3, n_cells=2, r=2, k=1, nu=1e-2, T=1.0, n_slabs=8)
    assert rel(g.forcing(pb.forcing, slab=2), slab.rhs_forcing(pb.forcing, 2 / 8)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_time_marching_config1(prec):
    """Config 1 (8x8, Q2/P1/DG(1), 4 slabs, nu = 1, manufactured field x sin(pi t)):
    GPU time marching against the oracle's, and the manufactured-solution error."""
    pb = manufactured_2d(nu=1.0, time="sin_pi")
    sols_o, infos_o, slab, _ = march(pb, 8, 1, 1, 4, tol=1e-12)
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=4, precond_precision=prec,
                         rel_tol=1e-12)
    x = None
    for s in range(4):
        F = g.forcing(pb.forcing, s)
        b = g.slab_rhs(F, x)
        x, info = g.solve_slab(b)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-12
        d = slab.remove_pressure_mean(x.cpu().numpy())
        assert rel(d, slab.remove_pressure_mean(sols_o[s])) < 1e-9
        assert info["iterations"] <= infos_o[s].iterations + (1 if prec == "fp64" else 4)


def test_fp32_preconditioner_reaches_fp64_tolerance():
    dim, n, r, k = 2, 16, 2, 2
    pb = fourier_forcing_2d(nu=1.0)
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, nu=1.0, T=1.0, n_slabs=16, precond_precision="fp32")
    F = g.forcing(pb.forcing, 0)
    x, info = g.solve_slab(g.slab_rhs(F))
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8
    r_ = g.residual(g.slab_rhs(F), x)
    b = g.slab_rhs(F)
    assert (torch.linalg.norm(r_) / torch.linalg.norm(b)).item() <= 1.001e-8


def test_host_buffers_solve():
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1)
    pb = manufactured_2d()
    b = g.slab_rhs(g.forcing(pb.forcing, 0))
    xd, info_d = g.solve_slab(b)
    bh = b.cpu().numpy().copy()
    xh = np.zeros_like(bh)
    info = g.solve_slab_host(bh, xh)
    assert info["status"] == 0 and info["iterations"] == info_d["iterations"]
    assert rel(xh, xd.cpu().numpy()) < 1e-12


def test_march_host_matches_oracle_march():
    """Config 1 marched through stmg_march_host (host forcing in, host solutions out, copies
    overlapped with the solves) against the oracle's march, slab by slab."""
    pb = manufactured_2d(nu=1.0, time="sin_pi")
    sols_o, _, slab, _ = march(pb, 8, 1, 1, 4, tol=1e-12)
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, nu=1.0, T=1.0, n_slabs=4, precond_precision="fp32",
                         rel_tol=1e-12)
    Fh = np.stack([g.forcing(pb.forcing, s).cpu().numpy() for s in range(4)])
    Fp = torch.from_numpy(Fh).pin_memory()
    Xp = torch.full_like(Fp, float("nan")).pin_memory()
    infos = g.march_host(Fp.numpy(), Xp.numpy())
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-12 for i in infos)
    for s in range(4):
        assert rel(slab.remove_pressure_mean(Xp[s].numpy()), slab.remove_pressure_mean(sols_o[s])) < 1e-9
    with pytest.raises(ValueError):
        g.march_host(Fh[:, :5].copy(), Fh[:, :5].copy())


def test_error_statuses():
    with pytest.raises(stmg.StmgError):
        stmg.SpaceTimeMG(dim=2, n_cells=4, r=5, k=1)                 # not built: r > 4
    with pytest.raises(stmg.StmgError):
        stmg.SpaceTimeMG(dim=2, n_cells=6, r=1, k=1)                 # default rule needs 2^c
    with pytest.raises(stmg.StmgError):
        stmg.SpaceTimeMG(dim=2, n_cells=4, r=1, k=1, levels=[(4, 1, 1), (1, 1, 1)])   # 4 -> 1 invalid
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1, gmres_max_iter=1)
    b = g.slab_rhs(g.forcing(manufactured_2d().forcing, 0))
    _, info = g.solve_slab(b)
    assert info["status"] == stmg._lib.ERR_NOT_CONVERGED
    bn = b.clone()
    bn[5] = float("nan")
    with pytest.raises(stmg.StmgError):
        g.solve_slab(bn)
    with pytest.raises(ValueError):
        g.apply(torch.zeros(3, dtype=torch.float64, device="cuda"))


def test_bounded_wait_timeout_is_reported_and_recoverable():
    """Failure handling without a GPU fault: the Arnoldi step's grid barrier is armed so
    that it cannot complete; its bounded waits expire, the solve reports STMG_ERR_TIMEOUT,
    and the next solve on the same handle converges."""
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=1, k=1)
    b = g.slab_rhs(g.forcing(manufactured_2d().forcing, 0))
    _, ref = g.solve_slab(b)
    g.inject_wait_fault()
    with pytest.raises(stmg.StmgError) as e:
        g.solve_slab(b)
    assert e.value.status == stmg._lib.ERR_TIMEOUT
    _, again = g.solve_slab(b)
    assert again["status"] == 0 and again["iterations"] == ref["iterations"]
    g.device_status()
    g.close()


def test_out_of_memory_is_reported():
    """3D 64^3 Q3/P2 DG(2) with FP64 patch inverses needs about 770 GB: stmg_create must
    fail with STMG_ERR_OOM (and leave the device usable)."""
    with pytest.raises(stmg.StmgError) as e:
        stmg.SpaceTimeMG(dim=3, n_cells=64, r=2, k=2, precisions=("fp64",), precond_precision="fp64",
                         autotune=False, use_graphs=False)
    assert e.value.status == stmg._lib.ERR_OOM
    g = stmg.SpaceTimeMG(dim=2, n_cells=4, r=1, k=1)
    assert g.apply(torch.ones(g.size(0), dtype=torch.float64, device="cuda")).abs().sum().item() > 0
    g.close()


def test_profiling_counters():
    g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=2, k=1, precond_precision="fp32")
    g.set_profiling(2)
    b = g.slab_rhs(g.forcing(manufactured_2d().forcing, 0))
    _, info = g.solve_slab(b)
    p = g.profile(reset=True)
    assert p["fine_sweep"]["launches"] == 2 * info["iterations"]
    assert p["fine_sweep"]["ms"] > 0 and p["operator"]["launches"] >= info["iterations"]


def test_overlapped_iterations_match_serial():
    """FGMRES runs its next iteration on the device while the host checks the previous one
    (unless the residual history predicts convergence); with profiling on it does not.
    Both orders give the same iteration counts and solutions that meet the tolerance, over
    a march of three slabs with the FP32 V-cycle: the solve that overlaps ends with nothing
    of a discarded iteration left in its solution."""
    pb = manufactured_2d()
    outs = []
    for prof in (0, 2):
        g = stmg.SpaceTimeMG(dim=2, n_cells=8, r=2, k=1, nu=1.0, T=0.75, n_slabs=3, precond_precision="fp32",
                             rel_tol=1e-10)
        g.set_profiling(prof)
        x_prev, xs = None, []
        for s in range(3):
            b = g.slab_rhs(g.forcing(pb.forcing, s), x_prev)
            x, info = g.solve_slab(b)
            assert info["status"] == 0 and info["rel_residual"] <= 1e-10
            r = g.residual(b, x, 0)
            assert r.norm().item() <= 1e-10 * b.norm().item() * 1.01
            xs.append((x.cpu().numpy(), info["iterations"]))
            x_prev = x
        outs.append(xs)
        g.device_status()
        g.close()
    # the FP32 V-cycle's scatter-adds round in whatever order the atomics land, so the two
    # runs' iterates differ by rounding; both meet the residual tolerance, and they agree
    # to that tolerance times the condition of the slab system
    for (xa, ia), (xb, ib) in zip(*outs):
        assert ia == ib
        assert rel(xa, xb) < 1e-6


def test_tune_cache_round_trip(tmp_path, monkeypatch):
    """STMG_TUNE_CACHE: the first handle tunes and writes its launch shapes, a second handle
    of the same configuration reads them (no timing) and runs the same V-cycle."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("STMG_TUNE_CACHE", str(cache))
    kw = dict(dim=2, n_cells=16, r=2, k=2, nu=1.0, T=1.0, n_slabs=16, coarse_n=4, k_min=2)
    g1 = stmg.SpaceTimeMG(**kw)
    assert cache.exists() and cache.read_text().count("\n") == 1
    g2 = stmg.SpaceTimeMG(**kw)
    assert g1.levels == g2.levels
    b = torch.from_numpy(random_vector(g1.size(0), 5)).to("cuda")
    for prec in ("fp64", "fp32"):
        x1, x2 = g1.vcycle(b, prec), g2.vcycle(b, prec)
        assert rel(x2, x1.cpu().numpy()) < (1e-13 if prec == "fp64" else 1e-6)
    g3 = stmg.SpaceTimeMG(**{**kw, "k": 1, "k_min": 1})         # another configuration: a second line
    assert cache.read_text().count("\n") == 2
    for g in (g1, g2, g3):
        g.close()
