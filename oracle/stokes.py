"""Oracle: slab systems, transfers, hierarchy, Vanka smoothers, V-cycle, FGMRES.

Test infrastructure only (see oracle/__init__.py).  FP64, assembled sparse
matrices, plain loops; each function names the passage of the paper it follows.

Readings of the paper taken here (the paper is silent, ambiguous or garbled):
* nu multiplies the vector Laplacian in the slab matrix (the weak form, Problem DVP,
  has it; Eq. InAlg omits it).
* Sign convention S = [[K (x) M_h + M_tau (x) nu A_h, -M_tau (x) B_h^T],
                       [-M_tau (x) B_h, 0]]:
  the momentum rows carry -<p, div w> as in the weak form; the continuity rows are
  negated so that the spatial part is symmetric.  This leaves the solution, every
  additive-Vanka correction and every GMRES iterate unchanged (the row scaling is an
  orthogonal diagonal that cancels).
* Homogeneous Dirichlet velocity dofs: their rows and columns of every level matrix
  are replaced by the identity; right-hand sides and corrections vanish there.
* Cell-Vanka patch matrices are the global submatrix R_T S R_T^T on all dofs of the
  space-time cell, Dirichlet dofs included (as identity rows); the additive sum is
  weighted by 1/valence per dof (Eq. vanka0, vanka and the remark that follows them).
* The coarsest level is solved directly with a bordered system fixing the mean of
  the pressure of every temporal dof (the subspace (M_p 1)^perp of Eq. DefRsSs).
* Transfers are the canonical embeddings of App. A, restriction = transpose.
* Hierarchy: the rule decoded from Table 2(b) (see `default_hierarchy`).
* GMRES stops when ||b - S x||_2 <= tol ||b||_2, without restarts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe import SpaceFE, TimeFE, gauss_legendre, lagrange_values, legendre_unit, slab_size


# ---------------------------------------------------------------------------
# Slab operator and right-hand side (Problem LocAlg, Eq. InAlg, DefDtauh)
# ---------------------------------------------------------------------------
class SlabGeometry:
    """Spaces, layout and Dirichlet mask of one slab system, without assembled matrices
    (enough for right-hand sides, error norms and row-wise evaluation at any size)."""

    def __init__(self, dim, n, r, k, nu, tau, nsub=1):
        self.space = SpaceFE(dim, n, r)
        self.time = TimeFE(k, tau, nsub)
        self.dim, self.n, self.r, self.k, self.nu, self.tau, self.nsub = dim, n, r, k, nu, tau, nsub
        sp_ = self.space
        self.nv, self.npr = sp_.n_vel, sp_.n_pres
        self.kt = self.time.kt
        self.size = self.kt * (self.nv + self.npr)
        assert self.size == slab_size(dim, n, r, k, nsub)
        dir_v = sp_.vel_dirichlet()
        self.dirichlet = np.concatenate([np.tile(dir_v, self.kt), np.zeros(self.kt * self.npr, bool)])

    # layout helpers ---------------------------------------------------------
    def vel(self, X, a):
        return X[a * self.nv:(a + 1) * self.nv]

    def pres(self, X, a):
        o = self.kt * self.nv
        return X[o + a * self.npr:o + (a + 1) * self.npr]

    def remove_pressure_mean(self, X):
        """Copy of X with the mean of each temporal pressure removed (means are mode-0
        coefficients weighted equally on the uniform mesh)."""
        Y = X.copy()
        o = self.kt * self.nv
        mode0 = np.arange(self.space.n_cells) * self.space.n_pm
        for a in range(self.kt):
            idx = o + a * self.npr + mode0
            Y[idx] -= Y[idx].mean()
        return Y

    def boundary_vector(self, fn, t0):
        """Slab vector with fn(x, t_n^a) (a tuple of dim velocity arrays) on the boundary
        velocity dofs of every temporal dof, zero elsewhere."""
        sp_ = self.space
        g = np.zeros(self.size)
        bnodes = np.nonzero(sp_.dirichlet)[0]
        X = tuple(sp_.node_coords[bnodes, d] for d in range(self.dim))
        for a in range(self.kt):
            ta = t0 + self.tau / 2 * (self.time.nodes[a] + 1.0)
            vals = fn(X, ta)
            for comp in range(self.dim):
                g[a * self.nv + comp * sp_.n_nodes + bnodes] = np.broadcast_to(vals[comp], bnodes.shape)
        return g

    def rhs_forcing(self, f, t0):
        """F_n of Eq. DefFn: (F_n^a)_i = Q_n(<f, phi_a chi_i>) = tau/2 w_a <f(t_n^a), chi_i>,
        spatial integral with (r+4)^d Gauss points; zero on Dirichlet dofs."""
        t = self.time
        F = np.zeros(self.size)
        for a in range(self.kt):
            ta = t0 + self.tau / 2 * (t.nodes[a] + 1.0)
            load = self.space.assemble_load(lambda X: f(X, ta))
            F[a * self.nv:(a + 1) * self.nv] = self.tau / 2 * t.weights[a] * load
        F[self.dirichlet] = 0.0
        return F


def slab_rows(geo: SlabGeometry, x, rows):
    """Rows `rows` of S x (Eq. InAlg / DefDtauh with the identity on Dirichlet rows and
    columns), evaluated one by one from the element matrices of the cells that touch each
    row's dof: for any mesh size, without assembling S."""
    sp_, t = geo.space, geo.time
    kt, dim, nv, npr = geo.kt, geo.dim, geo.nv, geo.npr
    poff = kt * nv
    G, R1, n = sp_.G, sp_.r + 1, sp_.n
    vdir = sp_.dirichlet
    out = np.zeros(len(rows))

    def xv(a, comp, nodes):                       # velocity entries, Dirichlet columns removed
        v = x[a * nv + comp * sp_.n_nodes + nodes]
        return np.where(vdir[nodes], 0.0, v)

    for q, i in enumerate(rows):
        if i < poff:                              # velocity row (a, comp, node)
            a, rest = divmod(i, nv)
            comp, node = divmod(rest, sp_.n_nodes)
            if vdir[node]:
                out[q] = x[i]
                continue
            g = np.array([(node // G ** d) % G for d in range(dim)])
            cands = [sorted({min(gd // R1, n - 1), max(gd - 1, 0) // R1}) for gd in g]
            s = 0.0
            for cell in np.array(np.meshgrid(*cands, indexing="ij")).reshape(dim, -1).T:
                c = int((cell * n ** np.arange(dim)).sum())
                loc = g - cell * R1
                if np.any(loc < 0) or np.any(loc > R1):
                    continue
                p = int((loc * sp_.np1 ** np.arange(dim)).sum())
                nodes = sp_.cell_nodes[c]
                for b in range(kt):
                    ub = xv(b, comp, nodes)
                    s += t.K[a, b] * (sp_.Me[p] @ ub)
                s += t.M[a, a] * geo.nu * (sp_.Ae[p] @ xv(a, comp, nodes))
                pc = x[poff + a * npr + c * sp_.n_pm + np.arange(sp_.n_pm)]
                s -= t.M[a, a] * (sp_.Be[comp][:, p] @ pc)
            out[q] = s
        else:                                     # pressure row (a, cell, mode)
            a, rest = divmod(i - poff, npr)
            c, m = divmod(rest, sp_.n_pm)
            nodes = sp_.cell_nodes[c]
            out[q] = -t.M[a, a] * sum(sp_.Be[comp][m] @ xv(a, comp, nodes) for comp in range(dim))
    return out


class Slab(SlabGeometry):
    """Space-time slab system of one level: spaces, matrices and the Dirichlet mask."""

    def __init__(self, dim, n, r, k, nu, tau, nsub=1):
        super().__init__(dim, n, r, k, nu, tau, nsub)
        sp_ = self.space
        self.Mv = sp_.mass()
        self.Av = sp_.laplace()
        self.B = sp_.divergence()
        self.S_raw = self._assemble_raw()
        free = sp.diags((~self.dirichlet).astype(float))
        fix = sp.diags(self.dirichlet.astype(float))
        self.S = (free @ self.S_raw @ free + fix).tocsr()

    def _assemble_raw(self):
        """S of Eq. InAlg before any boundary condition is imposed."""
        t = self.time
        Mt = sp.csr_matrix(t.M)
        vel = sp.kron(sp.csr_matrix(t.K), self.Mv) + sp.kron(Mt, self.nu * self.Av)
        vp = -sp.kron(Mt, self.B.T)
        pv = -sp.kron(Mt, self.B)
        pp = sp.csr_matrix((self.kt * self.npr, self.kt * self.npr))
        return sp.bmat([[vel, vp], [pv, pp]], format="csr")

    def lift(self, g, b):
        """Right-hand side with non-homogeneous Dirichlet values g (entries on the boundary
        dofs): interior rows b - S_raw[:, D] g_D, boundary rows g.  The solution of S x = lift
        then satisfies x_D = g_D and the interior rows of S_raw x = b."""
        gd = np.where(self.dirichlet, g, 0.0)
        y = b - self.S_raw @ gd
        y[self.dirichlet] = g[self.dirichlet]
        return y

    def coupling(self, v_prev):
        """(C_tau (x) M_h) V_{n-1} of Eq. InAlg: velocity row a gets phi_a(t_{n-1}^+) M_h v_{n-1}."""
        out = np.zeros(self.size)
        mv = self.Mv @ v_prev
        for a in range(self.kt):
            out[a * self.nv:(a + 1) * self.nv] = self.time.phi_left[a] * mv
        out[self.dirichlet] = 0.0
        return out

    def pressure_nullspace(self):
        """Columns spanning {(0, e_a (x) 1)}: the constant pressure of each temporal dof,
        expressed in the Legendre basis (mode 0 of every cell)."""
        N = np.zeros((self.size, self.kt))
        o = self.kt * self.nv
        mode0 = np.arange(self.space.n_cells) * self.space.n_pm
        for a in range(self.kt):
            N[o + a * self.npr + mode0, a] = 1.0
        return N

    def direct_solve(self, b):
        """Bordered sparse LU solve of S x = b with zero-mean pressure per temporal dof."""
        N = sp.csr_matrix(self.pressure_nullspace())
        Z = sp.csr_matrix((self.kt, self.kt))
        Bd = sp.bmat([[self.S, N], [N.T, Z]], format="csc")
        sol = spla.spsolve(Bd, np.concatenate([b, np.zeros(self.kt)]))
        return sol[:self.size]


# ---------------------------------------------------------------------------
# Transfers (App. A: Eq. DefPrRe, DeftTps, DeftTrs, DefPrRer, DefPrRek, DefoTsl)
# ---------------------------------------------------------------------------
def prolong_space(coarse: SpaceFE, fine: SpaceFE):
    """Canonical prolongation between nested spatial spaces (h: n -> 2n, p: r' -> r, or both):
    the coarse function re-expressed in the fine basis (Eq. DefTps).

    Velocity: P[I, J] = phi_J^coarse(x_I) at the fine nodes.  Pressure: per fine cell,
    the L2 projection of each coarse Legendre mode onto the fine cell's modes (exact:
    the restriction of a P_r' polynomial to a sub-cell is in P_r).  Returns (Pv, Pp),
    Pv scalar (per velocity component)."""
    assert fine.dim == coarse.dim
    d = fine.dim
    # velocity
    xf = fine.node_coords                                     # [Nf, d]
    cc = np.minimum(np.floor(xf / coarse.h + 1e-12).astype(int), coarse.n - 1)
    xi = xf / coarse.h - cc                                   # local coordinates in [0,1]
    loc = coarse.local_nodes()
    vals = np.ones((len(xf), len(loc)))
    for dd in range(d):
        L = lagrange_values(coarse.xi, xi[:, dd])             # [np1c, Nf]
        vals *= L[loc[:, dd]].T
    stride = coarse.G ** np.arange(d)
    J = ((cc[:, None, :] * (coarse.r + 1) + loc[None, :, :]) * stride).sum(-1)
    I = np.repeat(np.arange(len(xf))[:, None], len(loc), axis=1)
    keep = np.abs(vals) > 0.0
    Pv = sp.csr_matrix((vals[keep], (I[keep], J[keep])), shape=(fine.n_nodes, coarse.n_nodes))
    # pressure: project with a Gauss rule exact for degree 2r
    nq = fine.r + 2
    x1, w1 = gauss_legendre(nq)
    x1, w1 = (x1 + 1) / 2, w1 / 2
    qidx = np.array([list(reversed(t)) for t in np.ndindex(*([nq] * d))])
    wq = np.prod(w1[qidx], axis=1)
    rows, cols, data = [], [], []
    for fc, cidx in enumerate(fine.cell_index):
        X = (cidx[None, :] + x1[qidx]) * fine.h                # physical points [Q, d]
        par = np.minimum(np.floor((cidx + 0.5) * fine.h / coarse.h).astype(int), coarse.n - 1)
        pc = int((par * coarse.n ** np.arange(d)).sum())
        Xc = X / coarse.h - par                                # coarse-local coords
        psi_f = np.ones((fine.n_pm, len(qidx)))
        for m, e in enumerate(fine.modes):
            for dd in range(d):
                psi_f[m] *= legendre_unit(e[dd], x1[qidx[:, dd]])
        psi_c = np.ones((coarse.n_pm, len(qidx)))
        for m, e in enumerate(coarse.modes):
            for dd in range(d):
                psi_c[m] *= legendre_unit(e[dd], Xc[:, dd])
        E = (psi_f * wq) @ psi_c.T                             # [mf, mc]
        for mf in range(fine.n_pm):
            for mc in range(coarse.n_pm):
                if abs(E[mf, mc]) > 1e-14:
                    rows.append(fc * fine.n_pm + mf)
                    cols.append(pc * coarse.n_pm + mc)
                    data.append(E[mf, mc])
    Pp = sp.csr_matrix((data, (rows, cols)), shape=(fine.n_pres, coarse.n_pres))
    return Pv, Pp


def prolong_time(tc: TimeFE, tf: TimeFE):
    """Prolongation in time: P[a, b] = phi_b^coarse(t_a^fine), the coarse DG function
    evaluated at the fine temporal nodes (the canonical embedding of Eq. DeftPrRe for a
    coarser temporal mesh, of Eq. DefPrRek for a lower degree, or both).

    The system's time span is split into tf.nsub fine and tc.nsub coarse subintervals,
    tf.nsub = m tc.nsub (m = 1: p in time only; m = 2: h in time, each coarse subinterval
    the union of two fine ones).  Fine node a lies in fine subinterval j_f at the local
    Radau coordinate s in (-1, 1]; it belongs to coarse subinterval j_c = j_f // m, at the
    local coordinate xi = (2 (j_f - m j_c) + s + 1) / m - 1.  A fine node at the right end
    of a coarse subinterval (s = 1, last fine subinterval of it) takes the value of that
    coarse subinterval's polynomial: DG functions are evaluated from the left there."""
    m = tf.nsub // tc.nsub
    assert tf.nsub == m * tc.nsub and abs(tc.tau - m * tf.tau) <= 1e-14 * tc.tau
    kf1, kc1 = tf.k + 1, tc.k + 1
    P = np.zeros((tf.kt, tc.kt))
    for jf in range(tf.nsub):
        jc = jf // m
        xi = (2.0 * (jf - m * jc) + tf.nodes1 + 1.0) / m - 1.0
        P[jf * kf1:(jf + 1) * kf1, jc * kc1:(jc + 1) * kc1] = lagrange_values(tc.nodes1, xi).T
    return P


def slab_prolongation(coarse: Slab, fine: Slab):
    """Space-time prolongation of a slab vector (Eq. DeftTps, DefoTsl): P_t (x) P_space per
    variable, rows of fine Dirichlet dofs and columns of coarse Dirichlet dofs removed."""
    Pv, Pp = prolong_space(coarse.space, fine.space)
    fd = fine.space.dirichlet
    cd = coarse.space.dirichlet
    Pv = sp.diags((~fd).astype(float)) @ Pv @ sp.diags((~cd).astype(float))
    Pvv = sp.block_diag([Pv] * fine.dim)
    Pt = sp.csr_matrix(prolong_time(coarse.time, fine.time))
    return sp.block_diag([sp.kron(Pt, Pvv), sp.kron(Pt, Pp)], format="csr")


# ---------------------------------------------------------------------------
# Hierarchy (Alg. 2 ConstructHierarchy, Alg. 3 CombineHierarchies)
# ---------------------------------------------------------------------------
def default_hierarchy(n, r, k, coarse_n=1, k_min=1):
    """Level list fine -> coarse as (n, r, k), the rule decoded from Table 2(b).

    Space (Alg. 2 on (h, r)): (n, r), (n, r//2), ..., (n, 1), then (n/2, 1), ..., (1, 1).
    Time (Alg. 2 on (tau, k), no geometric coarsening in time when marching): k, k//2,
    ..., 1, then 1 once more (the geometric loop re-adds the last pair).  Alg. 3 aligns
    both lists at the coarse end and pads the shorter one at the fine end with its
    finest entry (P4).  k = 0 gives k = 0 on every level.  coarse_n is the coarsest mesh
    (Alg. 2's h_0 = 1 / coarse_n) and k_min the lowest temporal degree; the paper's runs
    use coarse_n = k_min = 1."""
    space = []
    rr = r
    while rr >= 1:
        space.append((n, rr))
        rr //= 2
    nn = n // 2
    while nn >= max(coarse_n, 1):
        space.append((nn, 1))
        nn //= 2
    if k == 0:
        time = [0]
    else:
        # polynomial loop down to k_min (Alg. 2's r_0 in time; 1 in the paper's runs), then
        # the last degree once more
        time = [k]
        while time[-1] // 2 >= max(k_min, 1):
            time.append(time[-1] // 2)
        time.append(time[-1])
    L = max(len(space), len(time))
    space = [space[0]] * (L - len(space)) + space
    time = [time[0]] * (L - len(time)) + time
    return [(s[0], s[1], t) for s, t in zip(space, time)]


def vanka_patch_entries(levels, dim):
    """N_sm^el of Table 2(b)/(d) for cell patches: sum over levels of n^d B^2 with
    B = (k+1)(d (r+2)^d + C(r+d, d)) (the coarsest level included, as the table counts it)."""
    tot = 0
    for (n, r, k) in levels:
        B = (k + 1) * (dim * (r + 2) ** dim + math.comb(r + dim, dim))
        tot += n ** dim * B * B
    return tot


# ---------------------------------------------------------------------------
# Vanka smoother (Eq. vanka0, vanka; remark on cell and vertex-star patches)
# ---------------------------------------------------------------------------
def cell_patches(slab: Slab):
    """Dof index sets of the space-time cells: all k+1 temporal copies of the cell's
    velocity dofs (all components) and pressure modes."""
    s = slab.space
    pats = []
    for c in range(s.n_cells):
        idx = []
        for a in range(slab.kt):
            for comp in range(slab.dim):
                idx.extend(a * slab.nv + comp * s.n_nodes + s.cell_nodes[c])
        for a in range(slab.kt):
            idx.extend(slab.kt * slab.nv + a * slab.npr + c * s.n_pm + np.arange(s.n_pm))
        pats.append(np.array(idx))
    return pats


def vertex_star_patches(slab: Slab):
    """Vertex-star patches: for every mesh vertex (boundary vertices included), all velocity
    dofs in the closure of the cells around it and all their pressure modes; whole slab in
    time (remark after Eq. vanka).  The sets are pinned to this reading by closed-form
    counts; the reading is parity unpinned: Table 2(d) does not decode."""
    s = slab.space
    d = slab.dim
    pats = []
    for v in np.ndindex(*([s.n + 1] * d)):
        v = np.array(list(reversed(v)))
        cells = []
        for off in np.ndindex(*([2] * d)):
            c = v - 1 + np.array(list(reversed(off)))
            if np.all(c >= 0) and np.all(c < s.n):
                cells.append(int((c * s.n ** np.arange(d)).sum()))
        nodes = np.unique(np.concatenate([s.cell_nodes[c] for c in cells]))
        idx = []
        for a in range(slab.kt):
            for comp in range(d):
                idx.extend(a * slab.nv + comp * s.n_nodes + nodes)
        for a in range(slab.kt):
            for c in sorted(cells):
                idx.extend(slab.kt * slab.nv + a * slab.npr + c * s.n_pm + np.arange(s.n_pm))
        pats.append(np.array(idx))
    return pats


class Vanka:
    """Additive Vanka smoother: x <- x + omega D_w sum_T R_T^T [R_T S R_T^T]^{-1} R_T (b - S x)."""

    def __init__(self, slab: Slab, patches, omega):
        self.slab, self.patches, self.omega = slab, patches, omega
        S = slab.S
        self.inv = [self._local_inverse(S[p][:, p].toarray(), p) for p in patches]
        cnt = np.zeros(slab.size)
        for p in patches:
            cnt[p] += 1
        self.weight = 1.0 / cnt

    def _local_inverse(self, A, p):
        """[R_T S R_T^T]^{-1}.  A patch that contains every cell of the mesh (the centre
        vertex star of a 2x2 mesh) has only boundary velocity dofs around it, so its
        matrix is singular in the pressure constant of each temporal dof; it is inverted
        with the same bordering as the coarsest level (zero-mean pressure correction)."""
        s = self.slab
        N = s.pressure_nullspace()[p]
        if np.count_nonzero(N) < s.kt * s.space.n_cells:
            return np.linalg.inv(A)
        kt = s.kt
        Bd = np.block([[A, N], [N.T, np.zeros((kt, kt))]])
        return np.linalg.inv(Bd)[:len(p), :len(p)]

    def correction(self, res):
        """D_w sum_T R_T^T A_T R_T res (Eq. vanka0 with valence weights)."""
        out = np.zeros_like(res)
        for p, A in zip(self.patches, self.inv):
            out[p] += A @ res[p]
        return self.weight * out

    def step(self, b, x):
        """One smoothing iteration (Eq. vanka)."""
        return x + self.omega * self.correction(b - self.slab.S @ x)


# ---------------------------------------------------------------------------
# V-cycle (Alg. 1 with the subroutines of App. B)
# ---------------------------------------------------------------------------
@dataclass
class MGConfig:
    omega: float = 0.7
    nu1: int = 1
    nu2: int = 1
    smoother: str = "cell"          # "cell" or "vsp"


class Multigrid:
    """hp space-time multigrid on a level list (fine -> coarse) from `default_hierarchy`.

    Level operators are rediscretised on every level; between consecutive levels the
    transfer is whatever (n, r, k) change they have (h or p in space, p in time)."""

    def __init__(self, dim, levels, nu, tau, cfg: MGConfig = MGConfig(), nsub=1):
        """levels: (n, r, k) or (n, r, k, nsub_l) fine -> coarse; tau and nsub are the
        finest level's subinterval length and count (a level of nsub_l subintervals covers
        the same system time span with subintervals of length tau nsub / nsub_l: h-coarsening
        in time when nsub_l < nsub)."""
        self.cfg = cfg
        self.levels = [tuple(l) if len(l) == 4 else (l[0], l[1], l[2], nsub) for l in levels]
        span = tau * nsub
        self.slabs = [Slab(dim, n, r, k, nu, span / ns, ns) for (n, r, k, ns) in self.levels]
        self.P = [slab_prolongation(self.slabs[i + 1], self.slabs[i]) for i in range(len(levels) - 1)]
        self.smoothers = []
        for s in self.slabs[:-1]:
            pats = cell_patches(s) if cfg.smoother == "cell" else vertex_star_patches(s)
            self.smoothers.append(Vanka(s, pats, cfg.omega))
        # coarsest level: dense bordered inverse
        cs = self.slabs[-1]
        N = cs.pressure_nullspace()
        A = np.block([[cs.S.toarray(), N], [N.T, np.zeros((cs.kt, cs.kt))]])
        self.coarse_inv = np.linalg.inv(A)[:cs.size, :cs.size]

    def vcycle(self, b, lvl=0):
        """x = V(b) with zero initial guess on level `lvl` (0 = finest)."""
        if lvl == len(self.slabs) - 1:
            return self.coarse_inv @ b
        s, W = self.slabs[lvl], self.smoothers[lvl]
        x = np.zeros_like(b)
        for _ in range(self.cfg.nu1):
            x = W.step(b, x)
        r = b - s.S @ x
        y = self.vcycle(self.P[lvl].T @ r, lvl + 1)
        x = x + self.P[lvl] @ y
        for _ in range(self.cfg.nu2):
            x = W.step(b, x)
        return x


# ---------------------------------------------------------------------------
# Flexible GMRES (right preconditioning, modified Gram-Schmidt, no restart)
# ---------------------------------------------------------------------------
@dataclass
class SolveInfo:
    iterations: int
    rel_residual: float
    converged: bool
    history: List[float] = field(default_factory=list)


def fgmres(apply, precond, b, x0=None, tol=1e-8, maxit=200):
    """Solve A x = b; stop when ||b - A x||_2 <= tol ||b||_2 (Remark on the choice of
    GMRES: the slab system is non-symmetric)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), SolveInfo(0, 0.0, True, [0.0])
    r = b - apply(x)
    beta = np.linalg.norm(r)
    hist = [beta / bnorm]
    if beta <= tol * bnorm:
        return x, SolveInfo(0, beta / bnorm, True, hist)
    V = [r / beta]
    Z = []
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    j = 0
    for j in range(maxit):
        z = precond(V[j])
        Z.append(z)
        w = apply(z)
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V.append(w / H[j + 1, j])
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = math.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]) / bnorm)
        if abs(g[j + 1]) <= tol * bnorm or H[j + 1, j] == 0.0 and den == 0.0:
            break
    m = j + 1
    y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
    x = x + sum(y[i] * Z[i] for i in range(m))
    rel = np.linalg.norm(b - apply(x)) / bnorm
    return x, SolveInfo(m, rel, rel <= tol * (1 + 1e-6), hist)


# ---------------------------------------------------------------------------
# Time marching (Eq. AlgSysTMS) and error norms
# ---------------------------------------------------------------------------
def march(problem, n, r, k, n_slabs, cfg: MGConfig = MGConfig(), tol=1e-8, levels=None,
          solver="mg", slabs_to_run=None, nsub=1):
    """Solve system by system: D X_n = B_n + (C_tau (x) M_h) V_{n-1}, V_0 = 0, each system a
    macro step of `nsub` subintervals (Remark rem:GLSP; nsub = 1 is Eq. AlgSysTMS), n_slabs
    systems on (0, T]; with problem.boundary set, its values are imposed on the boundary
    dofs (Slab.lift).

    solver = "mg": FGMRES preconditioned by one V-cycle; "direct": bordered sparse LU.
    Returns (list of system solutions, list of SolveInfo, the finest Slab, Multigrid)."""
    tau = problem.T / (n_slabs * nsub)
    levels = levels or default_hierarchy(n, r, k)
    mg = Multigrid(problem.dim, levels, problem.nu, tau, cfg, nsub) if solver == "mg" else None
    slab = mg.slabs[0] if mg else Slab(problem.dim, n, r, k, problem.nu, tau, nsub)
    v_prev = np.zeros(slab.nv)
    sols, infos = [], []
    bnd = getattr(problem, "boundary", None)
    for s in range(slabs_to_run or n_slabs):
        t0 = s * nsub * tau
        b = slab.rhs_forcing(problem.forcing, t0) + slab.coupling(v_prev)
        if bnd is not None:
            b = slab.lift(slab.boundary_vector(bnd, t0), b)
        if solver == "mg":
            x, info = fgmres(lambda z: slab.S @ z, mg.vcycle, b, tol=tol)
        else:
            x = slab.direct_solve(b)
            info = SolveInfo(0, np.linalg.norm(b - slab.S @ x) / np.linalg.norm(b), True)
        sols.append(x)
        infos.append(info)
        v_prev = slab.vel(x, slab.kt - 1).copy()
    return sols, infos, slab, mg


def errors(problem, slab: Slab, sols, nq_v=None, nq_p=None, nq_t=None):
    """Space-time errors against the closed-form solution (Table 1 quantities):
    L2(L2) and L2(H1-seminorm) of the velocity, L2(L2) of div v_h, and L2(L2) of the
    pressure with the spatial mean removed at every time point.  Gauss rules with r+4
    points per direction in space and k+3 per slab in time by default; nq_v (velocity,
    gradient, divergence) and nq_p (pressure) override the spatial rule, nq_t the
    temporal one.  (Table 1 of the paper is reproduced with nq_v = r+2, nq_p = r+1.)"""
    sp_, tf = slab.space, slab.time
    tau = slab.tau

    def rule(nq):
        xq, wq1 = gauss_legendre(nq)
        xq, wq1 = (xq + 1) / 2, wq1 / 2
        qidx = np.array([list(reversed(t)) for t in np.ndindex(*([len(xq)] * slab.dim))])
        return xq, np.prod(wq1[qidx], axis=1) * sp_.h ** slab.dim

    xv, wv = rule(nq_v or slab.r + 4)
    xp, wp = rule(nq_p or slab.r + 4)
    tq, tw = gauss_legendre(nq_t or slab.k + 3)
    phi_t = lagrange_values(tf.nodes1, tq)                    # [b, q] on one subinterval
    k1 = slab.k + 1
    e_v = e_h1 = e_div = e_p = 0.0
    for s, X in enumerate(sols):
        for jsub in range(tf.nsub):
            t0 = (s * tf.nsub + jsub) * tau
            for qi in range(len(tq)):
                t = t0 + tau / 2 * (tq[qi] + 1)
                V = sum(phi_t[b_, qi] * slab.vel(X, jsub * k1 + b_) for b_ in range(k1))
                P = sum(phi_t[b_, qi] * slab.pres(X, jsub * k1 + b_) for b_ in range(k1))
                wt = tau / 2 * tw[qi]
                x, v, gv, _ = sp_.eval_cells(V, P, xv, grad=True)
                ve = problem.velocity(tuple(x), t)
                ge = problem.velocity_grad(tuple(x), t)
                e_v += wt * sum(((v[c] - ve[c]) ** 2 * wv).sum() for c in range(slab.dim))
                e_h1 += wt * sum(((gv[c][j] - ge[c][j]) ** 2 * wv).sum()
                                 for c in range(slab.dim) for j in range(slab.dim))
                div = sum(gv[c][c] for c in range(slab.dim))
                e_div += wt * ((div ** 2) * wv).sum()
                x, _, _, p = sp_.eval_cells(V, P, xp)
                pe = problem.pressure(tuple(x), t)
                pm = (p * wp).sum() / wp.sum() / sp_.n_cells
                pem = (pe * wp).sum() / wp.sum() / sp_.n_cells
                e_p += wt * ((((p - pm) - (pe - pem)) ** 2) * wp).sum()
    return {"v_L2L2": math.sqrt(e_v), "v_L2H1": math.sqrt(e_h1), "div_L2L2": math.sqrt(e_div),
            "p_L2L2": math.sqrt(e_p)}
