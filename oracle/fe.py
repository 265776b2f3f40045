"""Oracle finite-element building blocks (FP64, numpy / scipy.sparse).

Test infrastructure only (see oracle/__init__.py).  Written from Sec. 2-3 of the
paper: Q_{r+1} / P_r^disc in space on a uniform mesh of [0,1]^d (Eq. Def:VKQK,
Def:VhQh), DG(k) in time with the Lagrange basis at the right Gauss-Radau points
(Eq. GF, BasYk), and the matrices of Eq. DefKMC and Eq. DefMAB.

Conventions (the layout every part of the project uses):
* Velocity: tensor Lagrange basis of degree r+1 at the r+2 Gauss-Lobatto nodes of
  [0,1] in each direction; global node grid G = (r+1) n + 1 points per direction,
  lexicographic, x fastest.  A velocity vector is component-major:
  [v_x(all nodes), v_y(all nodes) (, v_z)].
* Pressure: per cell the orthonormal Legendre products L_i(xi) L_j(eta) (L_l(zeta))
  of total degree <= r, L_i(xi) = sqrt(2i+1) P_i(2 xi - 1); cells lexicographic,
  modes ordered by (total degree, z degree, y degree).
* Slab vector (Eq. DefX): [V^1 .. V^{k+1}, P^1 .. P^{k+1}].
"""
from __future__ import annotations

from math import comb

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as npleg


# ---------------------------------------------------------------------------
# Quadrature rules on [-1, 1]
# ---------------------------------------------------------------------------
def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1,1] (numpy's leggauss)."""
    x, w = npleg.leggauss(n)
    return np.asarray(x, float), np.asarray(w, float)


def gauss_lobatto(n):
    """n-point Gauss-Lobatto rule on [-1,1]: the end points and the roots of P'_{n-1};
    weights from exact integration of the Lagrange basis."""
    if n < 2:
        raise ValueError("Gauss-Lobatto needs at least 2 points")
    c = np.zeros(n)
    c[n - 1] = 1.0
    inner = np.sort(npleg.legroots(npleg.legder(c)).real) if n > 2 else np.zeros(0)
    x = np.concatenate(([-1.0], inner, [1.0]))
    return x, _interpolatory_weights(x)


def radau_right(k):
    """Right-sided (k+1)-point Gauss-Radau rule on [-1,1] (Sec. 3.1, Eq. GF).

    The nodes are the roots of P_k - P_{k+1}; the last one is +1.  The weights make
    the rule interpolatory (exact for P_k, and by Radau's theorem for P_{2k})."""
    c = np.zeros(k + 2)
    c[k] = 1.0
    c[k + 1] = -1.0
    x = np.sort(npleg.legroots(c).real)
    x[-1] = 1.0
    return x, _interpolatory_weights(x)


def _interpolatory_weights(x):
    gx, gw = gauss_legendre(len(x) + 1)
    return lagrange_values(x, gx) @ gw


# ---------------------------------------------------------------------------
# 1D bases
# ---------------------------------------------------------------------------
def lagrange_values(nodes, t):
    """Values ell_j(t_q) of the Lagrange basis at `nodes`; shape (len(nodes), len(t))."""
    nodes = np.asarray(nodes, float)
    t = np.atleast_1d(np.asarray(t, float))
    out = np.ones((len(nodes), len(t)))
    for j in range(len(nodes)):
        for m in range(len(nodes)):
            if m != j:
                out[j] *= (t - nodes[m]) / (nodes[j] - nodes[m])
    return out


def lagrange_derivs(nodes, t):
    """Derivatives ell_j'(t_q) of the Lagrange basis; shape (len(nodes), len(t))."""
    nodes = np.asarray(nodes, float)
    t = np.atleast_1d(np.asarray(t, float))
    n = len(nodes)
    out = np.zeros((n, len(t)))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(t), 1.0 / (nodes[j] - nodes[m]))
            for l in range(n):
                if l != j and l != m:
                    term = term * (t - nodes[l]) / (nodes[j] - nodes[l])
            out[j] += term
    return out


def legendre_unit(i, xi):
    """Orthonormal Legendre polynomial on [0,1]: sqrt(2i+1) P_i(2 xi - 1)."""
    c = np.zeros(i + 1)
    c[i] = 1.0
    return np.sqrt(2 * i + 1) * npleg.legval(2 * np.asarray(xi, float) - 1, c)


def pressure_modes(dim, r):
    """Exponent tuples (x, y[, z]) of P_r in the project's mode order:
    by total degree, then z degree, then y degree (all ascending)."""
    modes = []
    if dim == 2:
        for s in range(r + 1):
            for j in range(s + 1):
                modes.append((s - j, j))
    else:
        for s in range(r + 1):
            for l in range(s + 1):
                for j in range(s - l + 1):
                    modes.append((s - l - j, j, l))
    assert len(modes) == comb(r + dim, dim)
    return modes


# ---------------------------------------------------------------------------
# Temporal DG(k) element (Eq. GF, BasYk, DefKMC)
# ---------------------------------------------------------------------------
class TimeFE:
    """DG(k) on a system of `nsub` consecutive subintervals of length tau (a macro time
    step, Remark rem:GLSP; nsub = 1 is time marching, Eq. AlgSysTMS), Lagrange basis at the
    right Radau points of every subinterval.

    One subinterval (Eq. DefKMC):
      K1[a,b] = int phi_b' phi_a dt + phi_b(t_{n-1}^+) phi_a(t_{n-1}^+)
      M1[a,b] = int phi_b phi_a dt
      C1[a,b] = delta_{b,k+1} phi_a(t_{n-1}^+)
    K1 does not depend on tau (the 2/tau of the derivative cancels the tau/2 of the
    measure); M1 scales with tau.  Integrals use a Gauss rule exact for the integrand.
    The system of nsub subintervals (Eq. GloSys restricted to a macro step) has the
    temporal matrices K = block-lower-bidiagonal(diagonal K1, subdiagonal -C1) and
    M = blockdiag(M1); its temporal dofs are numbered subinterval by subinterval, and
    its nodes are given as reference coordinates s + 2 j on [-1, 2 nsub - 1] (subinterval
    j maps to [2j - 1, 2j + 1]).  Only the first subinterval couples to the previous
    system: phi_left = (phi_a(t^+), 0, ..., 0).
    """

    def __init__(self, k, tau, nsub=1):
        self.k, self.tau, self.nsub = k, tau, nsub
        s, w = radau_right(k)
        self.nodes1, self.weights1 = s, w
        gx, gw = gauss_legendre(k + 2)
        phi = lagrange_values(s, gx)                    # [a, q]
        dphi = lagrange_derivs(s, gx)                   # d/dt_hat
        phi_m1 = lagrange_values(s, [-1.0])[:, 0]
        # reference interval [-1,1]: dt = tau/2 dt_hat, d/dt = 2/tau d/dt_hat
        K1 = (phi * gw) @ dphi.T + np.outer(phi_m1, phi_m1)
        M1 = (tau / 2) * (phi * gw) @ phi.T
        C1 = np.zeros((k + 1, k + 1))
        C1[:, k] = phi_m1
        k1 = k + 1
        self.kt = nsub * k1
        self.K = np.zeros((self.kt, self.kt))
        self.M = np.zeros((self.kt, self.kt))
        for j in range(nsub):
            self.K[j * k1:(j + 1) * k1, j * k1:(j + 1) * k1] = K1
            self.M[j * k1:(j + 1) * k1, j * k1:(j + 1) * k1] = M1
            if j > 0:
                self.K[j * k1:(j + 1) * k1, (j - 1) * k1:j * k1] = -C1
        self.nodes = np.concatenate([s + 2.0 * j for j in range(nsub)])
        self.weights = np.tile(w, nsub)
        self.phi_left = np.concatenate([phi_m1, np.zeros((nsub - 1) * k1)])   # phi_a(t_{n-1}^+)
        self.C = np.zeros((self.kt, self.kt))
        self.C[:k1, self.kt - 1] = phi_m1
        self.K1, self.M1, self.C1 = K1, M1, C1

    def basis_at(self, that):
        """phi_a at reference times that in [-1, 2 nsub - 1]; shape (kt, len(that)).  A
        point on the border of two subintervals counts to the later one."""
        that = np.atleast_1d(np.asarray(that, dtype=float))
        out = np.zeros((self.kt, len(that)))
        k1 = self.k + 1
        j = np.clip(np.floor((that + 1.0) / 2.0).astype(int), 0, self.nsub - 1)
        for jj in range(self.nsub):
            m = j == jj
            if m.any():
                out[jj * k1:(jj + 1) * k1, m] = lagrange_values(self.nodes1, that[m] - 2.0 * jj)
        return out


# ---------------------------------------------------------------------------
# Spatial Q_{r+1}/P_r^disc on the uniform mesh of [0,1]^dim (Eq. Def:VKQK, DefMAB)
# ---------------------------------------------------------------------------
class SpaceFE:
    def __init__(self, dim, n, r):
        if dim not in (2, 3) or r < 1 or n < 1:
            raise ValueError("need dim in {2,3}, r >= 1, n >= 1")
        self.dim, self.n, self.r = dim, n, r
        self.h = 1.0 / n
        self.np1 = r + 2                                  # velocity nodes per direction per cell
        self.G = (r + 1) * n + 1                          # global nodes per direction
        self.n_nodes = self.G ** dim                      # scalar velocity nodes
        self.n_vel = dim * self.n_nodes                   # M^v
        self.modes = pressure_modes(dim, r)
        self.n_pm = len(self.modes)
        self.n_cells = n ** dim
        self.n_pres = self.n_cells * self.n_pm            # M^p
        self.xi = (gauss_lobatto(self.np1)[0] + 1.0) / 2.0   # GLL nodes on [0,1]
        self._element_matrices()
        self._maps()

    # -- local numbering ---------------------------------------------------
    def local_nodes(self):
        """Multi-indices of the (r+2)^dim cell nodes, x fastest."""
        return np.array([list(reversed(t)) for t in np.ndindex(*([self.np1] * self.dim))])

    def cells(self):
        """Multi-indices of the cells, x fastest."""
        return np.array([list(reversed(t)) for t in np.ndindex(*([self.n] * self.dim))])

    def _maps(self):
        cells = self.cells()                              # [C, dim]
        loc = self.local_nodes()                          # [P, dim]
        glob = cells[:, None, :] * (self.r + 1) + loc[None, :, :]
        stride = self.G ** np.arange(self.dim)
        self.cell_nodes = (glob * stride).sum(-1)         # [C, P] global scalar node ids
        self.cell_index = cells
        nodes = np.array([list(reversed(t)) for t in np.ndindex(*([self.G] * self.dim))])
        self.node_index = nodes                           # [N, dim]
        self.dirichlet = np.any((nodes == 0) | (nodes == self.G - 1), axis=1)
        cell_of = np.minimum(nodes // (self.r + 1), self.n - 1)
        local_of = nodes - cell_of * (self.r + 1)
        self.node_coords = (cell_of + self.xi[local_of]) * self.h

    # -- element matrices by d-dimensional Gauss quadrature -----------------
    def _ref_values(self, pts1d):
        """phi[p, q], dphi[j][p, q] (reference derivative), psi[m, q] at the tensor points."""
        d = self.dim
        L = lagrange_values(self.xi, pts1d)               # [np1, nq]
        dL = lagrange_derivs(self.xi, pts1d)
        leg = np.array([legendre_unit(i, pts1d) for i in range(self.r + 1)])
        qidx = np.array([list(reversed(t)) for t in np.ndindex(*([len(pts1d)] * d))])  # [Q, d]
        loc = self.local_nodes()
        phi = np.ones((len(loc), len(qidx)))
        for dd in range(d):
            phi *= L[loc[:, dd]][:, qidx[:, dd]]
        dphi = []
        for j in range(d):
            v = np.ones((len(loc), len(qidx)))
            for dd in range(d):
                tab = dL if dd == j else L
                v *= tab[loc[:, dd]][:, qidx[:, dd]]
            dphi.append(v)
        psi = np.ones((self.n_pm, len(qidx)))
        for m, e in enumerate(self.modes):
            for dd in range(d):
                psi[m] *= leg[e[dd]][qidx[:, dd]]
        return phi, dphi, psi, qidx

    def _element_matrices(self):
        d, h = self.dim, self.h
        nq = self.r + 3
        x, w = gauss_legendre(nq)
        x, w = (x + 1) / 2, w / 2
        phi, dphi, psi, qidx = self._ref_values(x)
        wq = np.prod(w[qidx], axis=1) * h ** d            # physical weights
        self.Me = (phi * wq) @ phi.T
        self.Ae = sum((dphi[j] / h * wq) @ (dphi[j] / h).T for j in range(d))
        # Be[c][m, p] = int d_c phi_p psi_m
        self.Be = [(psi * wq) @ (dphi[c] / h).T for c in range(d)]

    # -- global matrices ------------------------------------------------------
    def _assemble_scalar(self, Ae):
        cn = self.cell_nodes
        rows = np.repeat(cn, cn.shape[1], axis=1).ravel()
        cols = np.tile(cn, (1, cn.shape[1])).ravel()
        data = np.tile(Ae.ravel(), self.n_cells)
        return sp.csr_matrix((data, (rows, cols)), shape=(self.n_nodes, self.n_nodes))

    def mass_scalar(self):
        return self._assemble_scalar(self.Me)

    def laplace_scalar(self):
        return self._assemble_scalar(self.Ae)

    def mass(self):
        """Vector velocity mass M_h (Eq. DefMAB), no boundary treatment."""
        return sp.block_diag([self.mass_scalar()] * self.dim, format="csr")

    def laplace(self):
        """Vector Laplacian A_h (Eq. DefMAB), no boundary treatment."""
        return sp.block_diag([self.laplace_scalar()] * self.dim, format="csr")

    def divergence(self):
        """B_h with (B)_{l,j} = int div(chi_j) chi_l^p (Eq. DefMAB); shape (M^p, M^v)."""
        rows, cols, data = [], [], []
        prow = np.arange(self.n_cells)[:, None] * self.n_pm + np.arange(self.n_pm)[None, :]
        for c in range(self.dim):
            r_ = np.repeat(prow, self.cell_nodes.shape[1], axis=1).ravel()
            c_ = np.tile(self.cell_nodes + c * self.n_nodes, (1, self.n_pm)).ravel()
            rows.append(r_)
            cols.append(c_)
            data.append(np.tile(self.Be[c].ravel(), self.n_cells))
        return sp.csr_matrix((np.concatenate(data), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_pres, self.n_vel))

    def pressure_mass(self):
        """M_h^p: diagonal h^d I for the orthonormal Legendre basis (computed, not assumed)."""
        nq = self.r + 2
        x, w = gauss_legendre(nq)
        x, w = (x + 1) / 2, w / 2
        _, _, psi, qidx = self._ref_values(x)
        wq = np.prod(w[qidx], axis=1) * self.h ** self.dim
        Mpe = (psi * wq) @ psi.T
        return sp.block_diag([sp.csr_matrix(Mpe)] * self.n_cells, format="csr")

    def vel_dirichlet(self):
        """Boolean mask over the M^v velocity dofs: True on the boundary."""
        return np.tile(self.dirichlet, self.dim)

    # -- evaluation -------------------------------------------------------------
    def eval_cells(self, V, P, pts1d, grad=False):
        """Evaluate a velocity vector V (M^v) and pressure vector P (M^p) at the tensor
        points pts1d (in [0,1]) of every cell.  Returns (x [dim][C,Q], v [dim][C,Q],
        gradv [dim][dim][C,Q] or None, p [C,Q])."""
        phi, dphi, psi, qidx = self._ref_values(pts1d)
        cells = self.cell_index
        x = [(cells[:, dd][:, None] + pts1d[qidx[:, dd]][None, :]) * self.h for dd in range(self.dim)]
        v, gv = [], []
        for c in range(self.dim):
            U = V[c * self.n_nodes:(c + 1) * self.n_nodes][self.cell_nodes]    # [C, P]
            v.append(U @ phi)
            if grad:
                gv.append([U @ (dphi[j] / self.h) for j in range(self.dim)])
        Pc = P.reshape(self.n_cells, self.n_pm)
        p = Pc @ psi
        return x, v, (gv if grad else None), p

    def assemble_load(self, f_at, nq=None):
        """Load vector (int f . chi_i) over all velocity dofs for f_at(x) -> tuple of dim
        arrays; Gauss rule with nq = r+4 points per direction (no boundary treatment)."""
        nq = nq or (self.r + 4)
        x1, w1 = gauss_legendre(nq)
        x1, w1 = (x1 + 1) / 2, w1 / 2
        phi, _, _, qidx = self._ref_values(x1)
        wq = np.prod(w1[qidx], axis=1) * self.h ** self.dim
        cells = self.cell_index
        X = tuple((cells[:, dd][:, None] + x1[qidx[:, dd]][None, :]) * self.h for dd in range(self.dim))
        fv = f_at(X)
        out = np.zeros(self.n_vel)
        for c in range(self.dim):
            contrib = (np.asarray(fv[c]) * wq) @ phi.T              # [C, P]
            np.add.at(out, c * self.n_nodes + self.cell_nodes.ravel(), contrib.ravel())
        return out


def slab_size(dim, n, r, k, nsub=1):
    """Dofs per system D = nsub (k+1)(d ((r+1)n+1)^d + C(r+d,d) n^d); boundary dofs counted."""
    return nsub * (k + 1) * (dim * ((r + 1) * n + 1) ** dim + comb(r + dim, dim) * n ** dim)
