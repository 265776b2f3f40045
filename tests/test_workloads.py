"""The closed-form inputs both sides share (workloads/), checked by finite differences
(CPU only): each exact solution is divergence free, its gradient is the derivative of its
velocity, its forcing is d_t v - nu Lap v + grad p (Eq. SE), and it vanishes on the
boundary where the problem has homogeneous data.  The seeded Fourier forcing is a curl
plus a gradient and is reproducible by seed."""
import numpy as np
import pytest

from workloads import (fourier_forcing_2d, lid_driven_3d, manufactured_2d, polynomial_2d, polynomial_boundary,
                       random_vector, taylor_green_3d)

H1 = 1e-5          # central first differences: error ~ h^2 * |v'''|
H2 = 2e-3          # fourth-order second differences: error ~ h^4 * |v^(6)|


def _points(dim, n=40, seed=0):
    rng = np.random.default_rng(seed)
    return tuple(rng.uniform(0.05, 0.95, n) for _ in range(dim))


def _shift(x, d, h):
    return tuple(xi + (h if i == d else 0.0) for i, xi in enumerate(x))


def _d1(fn, x, d, h=H1):
    return (fn(_shift(x, d, h)) - fn(_shift(x, d, -h))) / (2 * h)


def _d2(fn, x, d, h=H2):
    f = [fn(_shift(x, d, s * h)) for s in (-2, -1, 0, 1, 2)]
    return (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h)


CASES = [
    ("manufactured_2d sin_pi", lambda: manufactured_2d(nu=0.7), True),
    ("manufactured_2d sin", lambda: manufactured_2d(nu=1.0, time="sin"), True),
    ("taylor_green_3d", lambda: taylor_green_3d(nu=0.3), True),
    ("polynomial_2d m=1", lambda: polynomial_2d(m=1, nu=0.5), True),
    ("polynomial_2d m=2", lambda: polynomial_2d(m=2, nu=1.5), True),
    ("polynomial_boundary 2d", lambda: polynomial_boundary(2, nu=0.8), False),
    ("polynomial_boundary 3d", lambda: polynomial_boundary(3, nu=1.2), False),
]


@pytest.mark.parametrize("name,make,homogeneous", CASES, ids=[c[0] for c in CASES])
def test_exact_solutions_satisfy_the_stokes_equations(name, make, homogeneous):
    pb = make()
    dim = pb.dim
    x = _points(dim)
    for t in (0.3, 0.71):
        v = pb.velocity(x, t)
        G = pb.velocity_grad(x, t)
        scale = max(np.abs(np.asarray(vi)).max() for vi in v) + 1.0
        # the gradient is the velocity's derivative, and its trace vanishes
        for i in range(dim):
            for j in range(dim):
                fd = _d1(lambda y: pb.velocity(y, t)[i], x, j)
                assert np.abs(np.asarray(G[i][j]) - fd).max() < 1e-7 * scale, (i, j)
        div = sum(np.asarray(G[i][i]) for i in range(dim))
        assert np.abs(div).max() < 1e-12 * scale
        # f = d_t v - nu Lap v + grad p
        f = pb.forcing(x, t)
        for i in range(dim):
            dt = (pb.velocity(x, t + H1)[i] - pb.velocity(x, t - H1)[i]) / (2 * H1)
            lap = sum(_d2(lambda y: pb.velocity(y, t)[i], x, d) for d in range(dim))
            gp = _d1(lambda y: pb.pressure(y, t), x, i)
            want = dt - pb.nu * lap + gp
            assert np.abs(np.asarray(f[i]) - want).max() < 1e-6 * (np.abs(want).max() + 1.0), i
    if homogeneous:
        # zero velocity on every face of [0,1]^d
        rng = np.random.default_rng(1)
        for d in range(dim):
            for side in (0.0, 1.0):
                xb = tuple(np.full(20, side) if e == d else rng.uniform(0, 1, 20) for e in range(dim))
                for vi in pb.velocity(xb, 0.4):
                    assert np.abs(np.asarray(vi)).max() < 1e-14
    else:
        # the boundary data are the exact velocity
        xb = _points(dim, seed=2)
        for gi, vi in zip(pb.boundary(xb, 0.6), pb.velocity(xb, 0.6)):
            assert np.array_equal(np.asarray(gi), np.asarray(vi))


def test_fourier_forcing_is_a_curl_plus_a_gradient():
    """f = curl(psi) + grad(phi), each field drawn from its own seed.  Two forcings that
    share the phi seed differ by a pure curl, whose divergence vanishes; two that share
    the psi seed differ by a pure gradient, whose 2D curl vanishes.  A sign slip in
    either part breaks one of the two.  The draw is reproducible by seed."""
    t = 0.37
    x = _points(2, seed=3)
    pb = fourier_forcing_2d(seed_psi=1, seed_phi=2)

    def diff(other, c):
        return lambda y: np.asarray(pb.forcing(y, t)[c]) - np.asarray(other.forcing(y, t)[c])

    same_phi = fourier_forcing_2d(seed_psi=5, seed_phi=2)
    u, v = diff(same_phi, 0), diff(same_phi, 1)
    div = _d1(u, x, 0) + _d1(v, x, 1)
    assert np.abs(div).max() < 1e-6 * (np.abs(u(x)).max() + 1.0)
    same_psi = fourier_forcing_2d(seed_psi=1, seed_phi=7)
    u, v = diff(same_psi, 0), diff(same_psi, 1)
    curl = _d1(v, x, 0) - _d1(u, x, 1)
    assert np.abs(curl).max() < 1e-5 * (np.abs(u(x)).max() + 1.0)
    f1 = pb.forcing(x, t)
    g1 = fourier_forcing_2d(seed_psi=1, seed_phi=2).forcing(x, t)
    assert all(np.array_equal(a, b) for a, b in zip(f1, g1))
    assert not np.allclose(f1[0], same_phi.forcing(x, t)[0])


def test_lid_data_and_random_vectors():
    pb = lid_driven_3d()
    X = (np.array([0.3, 0.5, 0.0]), np.array([0.2, 1.0, 0.4]), np.array([1.0, 1.0, 0.5]))
    u, v, w = pb.boundary(X, 2.0)                    # sin(pi 2 / 4) = 1 on the lid z = 1
    assert np.allclose(u, [1.0, 1.0, 0.0]) and not v.any() and not w.any()
    assert all(not np.asarray(c).any() for c in pb.forcing(X, 1.0))
    a, b = random_vector(1000, 3), random_vector(1000, 3)
    assert np.array_equal(a, b) and a.min() >= -1.0 and a.max() <= 1.0
    assert abs(a.mean()) < 0.1 and not np.array_equal(a, random_vector(1000, 4))
