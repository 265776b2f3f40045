"""CPU checks of libstmg's host side: the library loads, exports every symbol that
include/*.h declares, and its setup numerics agree with the FP64 oracle."""
import os
import re

import numpy as np
import pytest

from oracle.fe import SpaceFE, TimeFE
from oracle.stokes import MGConfig, Multigrid, Slab, cell_patches, default_hierarchy, vertex_star_patches

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2502_09159_gb300 as p
    p.build()
    return p


def test_library_exports_every_declared_symbol(pkg):
    import ctypes
    from paper_2502_09159_gb300 import _lib
    lib = _lib.load()
    text = ""
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            with open(os.path.join(ROOT, "include", h)) as f:
                text += f.read()
    names = set(re.findall(r"\b(stmg_[a-z0-9_]+)\s*\(", text))
    assert len(names) >= 50
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(_lib._SIGS) == names          # the binding covers exactly the header
    assert lib.stmg_status_string(0) == b"ok"
    assert lib.stmg_status_string(7).startswith(b"not implemented")


def test_create_without_gpu_fails_cleanly(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        pkg.SpaceTimeMG(dim=2, n_cells=2)


@pytest.mark.parametrize("n,r,k", [(8, 1, 1), (64, 2, 2), (32, 2, 1), (16, 3, 3), (4, 4, 2), (2, 1, 0),
                                   (1, 1, 1), (128, 2, 1), (4, 1, 3)])
def test_hierarchy_matches_oracle(pkg, n, r, k):
    assert pkg.host_default_hierarchy(n, r, k) == default_hierarchy(n, r, k)
    for cn in (1, 2, 8):
        for km in (1, 2, 4):
            if cn <= n:
                assert pkg.host_default_hierarchy(n, r, k, cn, km) == default_hierarchy(n, r, k, cn, km)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_tables_1d_match_oracle_element_matrices(pkg, r):
    t = pkg.host_tables_1d(r)
    s = SpaceFE(2, 1, r)                     # h = 1: element matrices are the 1D tables
    assert np.allclose(t["xi"], s.xi, atol=1e-15)
    assert np.abs(np.kron(t["M1"], t["M1"]) - s.Me).max() < 1e-14
    assert np.abs(np.kron(t["M1"], t["K1"]) + np.kron(t["K1"], t["M1"]) - s.Ae).max() < 1e-12
    loc = s.local_nodes()
    for comp in range(2):
        ref = np.array([[(t["G1"] if comp == 0 else t["N1"])[e[0], p[0]] *
                         (t["G1"] if comp == 1 else t["N1"])[e[1], p[1]] for p in loc] for e in s.modes])
        assert np.abs(ref - s.Be[comp]).max() < 1e-13


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_time_tables_match_oracle(pkg, k):
    tau = 0.37
    t = pkg.host_time_tables(k, tau)
    o = TimeFE(k, tau)
    assert np.abs(t["nodes"] - o.nodes).max() < 1e-14
    assert np.abs(t["weights"] - o.weights).max() < 1e-14
    assert np.abs(t["K"] - o.K).max() < 1e-13
    assert np.abs(t["M"] - np.diag(o.M)).max() < 1e-15
    assert np.abs(t["phi_left"] - o.phi_left).max() < 1e-13


def _oracle_dofs(slab, pat):
    d = np.array(pat, dtype=np.int64)
    return np.where(slab.dirichlet[d], -1, d)


@pytest.mark.parametrize("dim,n,r,k", [(2, 3, 1, 1), (2, 3, 2, 2), (2, 4, 1, 0), (2, 2, 3, 1), (3, 2, 1, 1)])
def test_cell_patch_inverses_match_oracle(pkg, dim, n, r, k):
    nu, tau = 0.8, 0.25
    levels = [(n, r, k), (1, 1, min(k, 1))] if n > 1 else [(n, r, k)]
    mg = Multigrid(dim, levels, nu, tau, MGConfig())
    slab, W = mg.slabs[0], mg.smoothers[0]
    pats = cell_patches(slab)
    check = sorted(set([0, len(pats) // 2, len(pats) - 1, 1 % len(pats)]))
    for p in check:
        hp = pkg.host_patch(dim, n, r, k, nu, tau, pkg.CELL, p)
        assert np.array_equal(hp["dofs"], _oracle_dofs(slab, pats[p]))
        A = W.inv[p]
        assert np.abs(hp["inverse"] - A).max() <= 1e-10 * np.abs(A).max()
    v = pkg.host_valence(dim, n, r, k, pkg.CELL)
    free = ~slab.dirichlet
    assert np.allclose(1.0 / v[free], W.weight[free])


@pytest.mark.parametrize("n", [3, 2])
def test_vsp_patch_inverses_match_oracle(pkg, n):
    """n = 2 includes the centre star covering the whole mesh (bordered inverse)."""
    dim, r, k, nu, tau = 2, 1, 1, 1.0, 0.5
    mg = Multigrid(dim, [(n, r, k), (1, 1, 1)], nu, tau, MGConfig(smoother="vsp"))
    slab, W = mg.slabs[0], mg.smoothers[0]
    pats = vertex_star_patches(slab)
    for p in sorted(set([0, 1, 4, 5 % len(pats), len(pats) - 1])):
        hp = pkg.host_patch(dim, n, r, k, nu, tau, pkg.VSP, p)
        b = len(pats[p])
        assert np.array_equal(hp["dofs"][:b], _oracle_dofs(slab, pats[p]))
        assert np.all(hp["dofs"][b:] == -2)
        A = W.inv[p]
        assert np.abs(hp["inverse"][:b, :b] - A).max() <= 1e-10 * np.abs(A).max()
        assert np.all(hp["inverse"][b:, :] == 0) and np.all(hp["inverse"][:, b:] == 0)


@pytest.mark.parametrize("dim,n,r,k", [(2, 1, 1, 1), (3, 1, 1, 1), (2, 2, 1, 0)])
def test_coarse_inverse_matches_oracle(pkg, dim, n, r, k):
    nu, tau = 1.3, 0.2
    mg = Multigrid(dim, [(n, r, k)], nu, tau, MGConfig())
    G = pkg.host_coarse_inverse(dim, n, r, k, nu, tau)
    assert np.abs(G - mg.coarse_inv).max() <= 1e-10 * np.abs(mg.coarse_inv).max()


@pytest.mark.parametrize("n", [1, 7, 255, 256, 300, 383, 640])
@pytest.mark.parametrize("threads", [1, 3, 0])
def test_host_invert_matches_numpy(pkg, n, threads):
    """The setup's Gauss-Jordan (blocked in panels of 32 columns from n = 256 on, rows
    split over threads) against numpy's LU-based inverse: sizes on both sides of the
    blocked form, ragged last panels, uneven row ranges per thread."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + np.sqrt(n) * np.eye(n)
    X = pkg.host_invert(A, threads)
    ref = np.linalg.inv(A)
    assert np.abs(X - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("n", [5, 300])
def test_host_invert_pivots(pkg, n):
    """A matrix whose diagonal is zero and whose largest entries sit off it (a scaled
    cyclic shift plus a small perturbation) can only be inverted with row interchanges."""
    rng = np.random.default_rng(1)
    A = 10.0 * np.roll(np.eye(n), 1, axis=1) + 0.01 * rng.standard_normal((n, n))
    np.fill_diagonal(A, 0.0)
    X = pkg.host_invert(A, 0)
    assert np.abs(X @ A - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("n", [6, 290])
def test_host_invert_reports_singular(pkg, n):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((n, n))
    A[:, -1] = A[:, 0] + 2.0 * A[:, 1]               # rank n - 1
    with pytest.raises(pkg.StmgError):
        pkg.host_invert(A, 0)


@pytest.mark.parametrize("n", [4, 8])
def test_coarse_inverse_blocked_path_matches_oracle(pkg, n):
    """Coarse levels large enough for the blocked, threaded form: D = 630 and D = 2310 (the
    coarsest level of the 64x64 Q3/P2 DG(2) hierarchy with an 8x8 coarsest mesh), each
    with 3 bordering rows."""
    dim, r, k, nu, tau = 2, 1, 2, 1.0, 1.0 / 16
    mg = Multigrid(dim, [(n, r, k)], nu, tau, MGConfig())
    G = pkg.host_coarse_inverse(dim, n, r, k, nu, tau)
    assert G.shape[0] >= 256
    assert np.abs(G - mg.coarse_inv).max() <= 1e-10 * np.abs(mg.coarse_inv).max()
