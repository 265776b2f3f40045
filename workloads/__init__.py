"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds problem data only: closed-form manufactured solutions of the
instationary Stokes system (Eq. SE), the forcing f = d_t v - nu Lap v + grad p that
goes with them, seeded random Fourier forcings, and seeded random vectors.  It
contains none of the discretisation's arithmetic (no basis, quadrature, matrix,
smoother or solver), so both the CPU oracle and the GPU path can import it.

Every callable takes coordinate arrays of any (broadcastable) shape and a scalar
time and returns arrays of the same shape: velocities as a tuple of d arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Tuple

import numpy as np

PI = math.pi


# ---------------------------------------------------------------------------
# 1D building blocks of the separable fields
# ---------------------------------------------------------------------------
def _s(x):   # sin^2(pi x)
    return np.sin(PI * x) ** 2


def _s1(x):  # d/dx sin^2(pi x)
    return PI * np.sin(2 * PI * x)


def _s2(x):
    return 2 * PI ** 2 * np.cos(2 * PI * x)


def _s3(x):
    return -4 * PI ** 3 * np.sin(2 * PI * x)


def _q(x):   # sin(pi x) cos(pi x)
    return 0.5 * np.sin(2 * PI * x)


def _q1(x):
    return PI * np.cos(2 * PI * x)


def _q2(x):
    return -2 * PI ** 2 * np.sin(2 * PI * x)


@dataclass
class Problem:
    """A Stokes problem on [0,1]^dim x (0,T]: forcing and (optional) exact solution."""
    dim: int
    nu: float
    T: float
    forcing: Callable            # f(x, t) -> tuple of dim arrays; x is a tuple of dim arrays
    velocity: Callable | None    # v(x, t) -> tuple of dim arrays (None: no closed form)
    pressure: Callable | None    # p(x, t) -> array
    velocity_grad: Callable | None = None  # grad v(x,t) -> [dim][dim] arrays, [i][j] = d_j v_i
    name: str = ""
    boundary: Callable | None = None       # Dirichlet velocity data g(x, t) on the boundary (None: 0)


def _time_factor(kind: str):
    if kind == "sin_pi":
        return (lambda t: math.sin(PI * t)), (lambda t: PI * math.cos(PI * t))
    if kind == "sin":
        return (lambda t: math.sin(t)), (lambda t: math.cos(t))
    raise ValueError(kind)


def manufactured_2d(nu: float = 1.0, time: str = "sin_pi", T: float = 1.0) -> Problem:
    """The 2D convergence-test field of Sec. 5.1 (Eq. conv-test).

    v = g(t) (sin^2(pi x) sin(pi y) cos(pi y), -sin(pi x) cos(pi x) sin^2(pi y)),
    p = g(t) sin(pi x) cos(pi x) sin(pi y) cos(pi y).
    The second velocity component carries a minus sign: with the printed plus sign
    the field is not divergence free; with the minus sign it is the curl of
    sin^2(pi x) sin^2(pi y) / (2 pi) and vanishes on the boundary.
    g(t) = sin(pi t) ("sin_pi") or sin(t) ("sin", the paper's Table 1 runs).
    """
    g, dg = _time_factor(time)

    def velocity(x, t):
        X, Y = x
        return (g(t) * _s(X) * _q(Y), -g(t) * _q(X) * _s(Y))

    def velocity_grad(x, t):
        X, Y = x
        G = g(t)
        return [[G * _s1(X) * _q(Y), G * _s(X) * _q1(Y)],
                [-G * _q1(X) * _s(Y), -G * _q(X) * _s1(Y)]]

    def pressure(x, t):
        X, Y = x
        return g(t) * _q(X) * _q(Y)

    def forcing(x, t):
        X, Y = x
        G, dG = g(t), dg(t)
        f1 = dG * _s(X) * _q(Y) - nu * G * (_s2(X) * _q(Y) + _s(X) * _q2(Y)) + G * _q1(X) * _q(Y)
        f2 = -dG * _q(X) * _s(Y) + nu * G * (_q2(X) * _s(Y) + _q(X) * _s2(Y)) + G * _q(X) * _q1(Y)
        return (f1, f2)

    return Problem(2, nu, T, forcing, velocity, pressure, velocity_grad, f"manufactured_2d[{time}]")


def taylor_green_3d(nu: float = 1e-2, T: float = 1.0) -> Problem:
    """3D divergence-free field v = sin(pi t) curl(psi (1,1,1)),
    psi = sin^2(pi x) sin^2(pi y) sin^2(pi z); p = sin(pi t)(x y z - 1/8)."""
    g, dg = _time_factor("sin_pi")
    fs = (_s, _s1, _s2, _s3)

    def dpsi(order, X, Y, Z):
        # order = (ox, oy, oz): derivative orders of the separable psi
        return fs[order[0]](X) * fs[order[1]](Y) * fs[order[2]](Z)

    # v_i = sum_j c_ij d_j psi with curl(psi e), e=(1,1,1):
    # v = (d_y psi - d_z psi, d_z psi - d_x psi, d_x psi - d_y psi)
    C = [(0, 1, -1), (-1, 0, 1), (1, -1, 0)]
    unit = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]

    def _add(a, b):
        return tuple(i + j for i, j in zip(a, b))

    def velocity(x, t):
        X, Y, Z = x
        return tuple(g(t) * sum(C[i][j] * dpsi(unit[j], X, Y, Z) for j in range(3)) for i in range(3))

    def velocity_grad(x, t):
        X, Y, Z = x
        return [[g(t) * sum(C[i][j] * dpsi(_add(unit[j], unit[m]), X, Y, Z) for j in range(3))
                 for m in range(3)] for i in range(3)]

    def pressure(x, t):
        X, Y, Z = x
        return g(t) * (X * Y * Z - 0.125)

    def forcing(x, t):
        X, Y, Z = x
        G, dG = g(t), dg(t)
        grad_p = (Y * Z, X * Z, X * Y)
        out = []
        for i in range(3):
            v_i = sum(C[i][j] * dpsi(unit[j], X, Y, Z) for j in range(3))
            lap_v_i = sum(C[i][j] * dpsi(_add(unit[j], _add(unit[m], unit[m])), X, Y, Z)
                          for j in range(3) for m in range(3))
            out.append(dG * v_i - nu * G * lap_v_i + G * grad_p[i])
        return tuple(out)

    return Problem(3, nu, T, forcing, velocity, pressure, velocity_grad, "taylor_green_3d")


def fourier_forcing_2d(nu: float = 1.0, T: float = 1.0, modes: int = 8, seed_psi: int = 1,
                       seed_phi: int = 2, drift: float = 0.0) -> Problem:
    """f = curl(psi) + grad(phi), psi, phi = sum_m c_m sin(pi a_m x) sin(pi b_m y) sin(pi t + theta_m(t)),
    c_m ~ N(0,1), a_m, b_m ~ U{1..4}, theta_m ~ U[0, 2 pi) drawn with numpy's PCG64 from the
    given seeds; theta_m(t) = theta_m + drift * t.  No closed-form solution."""
    def draw(seed):
        rng = np.random.default_rng(seed)
        c = rng.standard_normal(modes)
        a = rng.integers(1, 5, size=modes)
        b = rng.integers(1, 5, size=modes)
        th = rng.uniform(0.0, 2 * PI, size=modes)
        return c, a, b, th

    P, F = draw(seed_psi), draw(seed_phi)

    def grad_field(par, X, Y, t):
        c, a, b, th = par
        gx = np.zeros(np.broadcast(X, Y).shape)
        gy = np.zeros_like(gx)
        for m in range(modes):
            w = c[m] * math.sin(PI * t + th[m] + drift * t)
            gx = gx + w * PI * a[m] * np.cos(PI * a[m] * X) * np.sin(PI * b[m] * Y)
            gy = gy + w * PI * b[m] * np.sin(PI * a[m] * X) * np.cos(PI * b[m] * Y)
        return gx, gy

    def forcing(x, t):
        X, Y = x
        px, py = grad_field(P, X, Y, t)
        qx, qy = grad_field(F, X, Y, t)
        return (py + qx, -px + qy)

    return Problem(2, nu, T, forcing, None, None, None, f"fourier_2d[{seed_psi},{seed_phi},{drift}]")


def polynomial_2d(m: int = 1, nu: float = 1.0, T: float = 1.0) -> Problem:
    """Polynomial field for exact-reproduction checks:
    v = t^m curl(psi), psi = x^2 (1-x)^2 y^2 (1-y)^2 (a Q4 velocity, zero on the boundary),
    p = t^m (x - 1/2)(y - 1/2) (zero mean)."""
    def w(z):
        return z ** 2 * (1 - z) ** 2

    def w1(z):
        return 2 * z * (1 - z) ** 2 - 2 * z ** 2 * (1 - z)

    def w2(z):
        return 2 * (1 - z) ** 2 - 8 * z * (1 - z) + 2 * z ** 2

    def w3(z):
        return -12 * (1 - z) + 12 * z

    def g(t):
        return t ** m

    def dg(t):
        return m * t ** (m - 1) if m > 0 else 0.0

    def velocity(x, t):
        X, Y = x
        return (g(t) * w(X) * w1(Y), -g(t) * w1(X) * w(Y))

    def velocity_grad(x, t):
        X, Y = x
        G = g(t)
        return [[G * w1(X) * w1(Y), G * w(X) * w2(Y)], [-G * w2(X) * w(Y), -G * w1(X) * w1(Y)]]

    def pressure(x, t):
        X, Y = x
        return g(t) * (X - 0.5) * (Y - 0.5)

    def forcing(x, t):
        X, Y = x
        G, dG = g(t), dg(t)
        f1 = dG * w(X) * w1(Y) - nu * G * (w2(X) * w1(Y) + w(X) * w3(Y)) + G * (Y - 0.5)
        f2 = -dG * w1(X) * w(Y) + nu * G * (w3(X) * w(Y) + w1(X) * w2(Y)) + G * (X - 0.5)
        return (f1, f2)

    return Problem(2, nu, T, forcing, velocity, pressure, velocity_grad, f"polynomial_2d[m={m}]")


def polynomial_boundary(dim: int = 2, nu: float = 1.0, T: float = 1.0) -> Problem:
    """Divergence-free quadratic velocity that does not vanish on the boundary, for checks
    of non-homogeneous Dirichlet data: v = t (y^2, x^2) in 2D, v = t (y^2, z^2, x^2) in 3D
    (each component independent of its own coordinate), p = t (x - 1/2).  v lies in Q_2 and
    p in P_1, both linear in t: reproduced exactly by Q_{r+1}/P_r, DG(k) for r, k >= 1."""
    def velocity(x, t):
        if dim == 2:
            X, Y = x
            return (t * Y ** 2, t * X ** 2)
        X, Y, Z = x
        return (t * Y ** 2, t * Z ** 2, t * X ** 2)

    def velocity_grad(x, t):
        zero = np.zeros(np.broadcast(*x).shape)
        if dim == 2:
            X, Y = x
            return [[zero, 2 * t * Y + zero], [2 * t * X + zero, zero]]
        X, Y, Z = x
        return [[zero, 2 * t * Y + zero, zero], [zero, zero, 2 * t * Z + zero], [2 * t * X + zero, zero, zero]]

    def pressure(x, t):
        return t * (x[0] - 0.5)

    def forcing(x, t):
        # d_t v - nu Lap v + grad p: Lap of each quadratic component is 2 t
        v = velocity(x, 1.0)
        out = [vi - 2.0 * nu * t for vi in v]
        out[0] = out[0] + t
        return tuple(out)

    return Problem(dim, nu, T, forcing, velocity, pressure, velocity_grad, f"polynomial_boundary_{dim}d",
                   boundary=velocity)


def lid_driven_3d(nu: float = 1.0, T: float = 8.0) -> Problem:
    """Lid-driven cavity of Sec. 5.2: no forcing, no-slip walls, and on the lid z = 1 the
    velocity sin(pi t / 4) in the x direction (the paper gives the profile as a scalar; the
    x component is this reading), imposed on every node of the closed lid face."""
    def zero(x, t):
        z = np.zeros(np.broadcast(*x).shape)
        return (z, z.copy(), z.copy())

    def boundary(x, t):
        X, Y, Z = x
        lid = np.isclose(Z, 1.0).astype(float)
        return (math.sin(PI * t / 4.0) * lid, 0.0 * lid, 0.0 * lid)

    return Problem(3, nu, T, zero, None, None, None, "lid_driven_3d", boundary=boundary)


def random_vector(n: int, seed: int = 3, dtype=np.float64) -> np.ndarray:
    """Seeded U[-1, 1] vector of length n (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n).astype(dtype)


def problem_by_name(name: str, **kw) -> Problem:
    return {"manufactured_2d": manufactured_2d, "taylor_green_3d": taylor_green_3d,
            "fourier_2d": fourier_forcing_2d, "polynomial_2d": polynomial_2d,
            "polynomial_boundary": polynomial_boundary, "lid_driven_3d": lid_driven_3d}[name](**kw)
