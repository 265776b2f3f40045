"""Pins of the warm-start oracle (oracle/warmstart.py) against what mathematics fixes:
library convolution, finite differences, closed forms and exact invariants."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import warmstart as ws
from oracle.fe import radau_right
from oracle.stokes import SlabGeometry
from workloads import random_vector


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 7, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = ws.conv3x3(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[bi, :, :, c], W[o, :, :, c], mode="same") for c in range(3))
            assert np.allclose(y[bi, :, :, o], ref, atol=1e-13)


def test_conv_adjoint_identity():
    """<g, conv(x)> - <g, bias> = <conv^T g, x> and = <dW, W> (bilinearity)."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 3))
    W = rng.standard_normal((5, 3, 3, 3))
    g = rng.standard_normal((2, 4, 6, 5))
    lin = float((g * ws.conv3x3(x, W, np.zeros(5))).sum())
    assert np.isclose(lin, float((ws.conv3x3_grad_input(g, W) * x).sum()), rtol=1e-13)
    dW, db = ws.conv3x3_grad_weights(x, g)
    assert np.isclose(lin, float((dW * W).sum()), rtol=1e-13)
    assert np.allclose(db, g.sum(axis=(0, 1, 2)))


@pytest.mark.parametrize("skip", [False, True])
def test_backward_matches_finite_differences(skip):
    rng = np.random.default_rng(3)
    dims = (3, 5, 2, 4)
    theta = rng.standard_normal(ws.n_params(*dims, skip=skip)) * 0.4
    x = rng.standard_normal((2, 4, 5, dims[0]))
    tgt = rng.standard_normal((2, 4, 5, dims[2]))

    def loss(th):
        return ws.mse(ws.forward(th, x, *dims, skip=skip)[0], tgt)[0]

    pred, acts = ws.forward(theta, x, *dims, skip=skip)
    _, g = ws.mse(pred, tgt)
    grad = ws.backward(theta, acts, g, *dims, skip=skip)
    h = 1e-6
    for i in rng.choice(len(theta), 60, replace=False):
        e = np.zeros_like(theta)
        e[i] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_mse_gradient_and_value():
    rng = np.random.default_rng(4)
    p, t = rng.standard_normal((3, 4)), rng.standard_normal((3, 4))
    L, g = ws.mse(p, t)
    assert np.isclose(L, ((p - t) ** 2).sum() / 12)
    h = 1e-7
    e = np.zeros_like(p)
    e[1, 2] = h
    assert np.isclose((ws.mse(p + e, t)[0] - ws.mse(p - e, t)[0]) / (2 * h), g[1, 2], rtol=1e-6)


def test_adam_first_step_closed_form_and_convergence():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = ws.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8)
    # at step 1 the bias-corrected moments are g and g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    x, m, v = np.array([5.0]), np.zeros(1), np.zeros(1)
    for s in range(1, 3001):
        x, m, v = ws.adam_step(x, 2 * (x - 1.5), m, v, s, lr=0.05)
    assert abs(x[0] - 1.5) < 1e-3


def test_extrapolation_matrix_dg1_closed_form():
    # nodes -1/3, 1: phi_0 = 3/4 (1 - s), phi_1 = 3/4 (s + 1/3) at s = 5/3 and s = 3
    assert np.allclose(ws.extrapolation_matrix(1), [[-0.5, 1.5], [-1.5, 2.5]], atol=1e-14)
    assert np.allclose(ws.extrapolation_matrix(0), [[1.0]])


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_extrapolation_exact_on_polynomials(k):
    s, _ = radau_right(k)
    E = ws.extrapolation_matrix(k)
    for deg in range(k + 1):
        assert np.allclose(E @ (s ** deg), (s + 2.0) ** deg, atol=1e-11)


@pytest.mark.parametrize("dim,n,r,k", [(2, 3, 2, 1), (2, 2, 1, 0), (3, 2, 1, 1)])
def test_gather_scatter_round_trip(dim, n, r, k):
    geo = SlabGeometry(dim, n, r, k, 1.0, 0.1)
    x = random_vector(geo.size, 5)
    x[geo.dirichlet] = 0.0
    cells = ws.cells_gather(geo, x)
    assert cells.shape == (n ** dim, ws.n_channels(dim, r, k))
    assert np.allclose(ws.cells_scatter_add(geo, cells, np.zeros(geo.size)), x, atol=1e-15)
    # every slab entry is covered; interior velocity nodes shared by 2^dim cells
    idx = ws.cell_index_map(geo)
    assert len(np.unique(idx)) == geo.size
    if n >= 2:
        shared = (np.bincount(idx.ravel(), minlength=geo.size)).max()
        assert shared == 2 ** dim


def test_gather_of_a_smooth_field_agrees_across_cells():
    """A global velocity node's value is the same in every cell that holds a copy."""
    geo = SlabGeometry(2, 3, 2, 1, 1.0, 0.1)
    x = random_vector(geo.size, 9)
    idx = ws.cell_index_map(geo)
    cells = ws.cells_gather(geo, x)
    assert np.array_equal(cells, x[idx])
    base = random_vector(geo.size, 10)
    inv = np.linspace(0.5, 2.0, idx.shape[1])
    assert np.allclose(ws.cells_gather(geo, x, base, inv), (x - base)[idx] * inv[None, :])


def test_extrapolate_slab_vector_linear_in_time():
    """DG(1): a slab vector holding u(t) = u0 + t u1 at the nodes is continued exactly."""
    geo = SlabGeometry(2, 2, 1, 1, 1.0, 0.25)
    s, _ = radau_right(1)
    u0, u1 = random_vector(geo.nv + geo.npr, 1), random_vector(geo.nv + geo.npr, 2)

    def slab(offset):
        X = np.zeros(geo.size)
        for a in range(2):
            u = u0 + (s[a] + offset) * u1
            X[a * geo.nv:(a + 1) * geo.nv] = u[:geo.nv]
            X[2 * geo.nv + a * geo.npr:2 * geo.nv + (a + 1) * geo.npr] = u[geo.nv:]
        return X

    assert np.allclose(ws.extrapolate(geo, slab(0.0)), slab(2.0), atol=1e-13)


def test_bypass_is_a_linear_convolution_added_to_the_output():
    """With every layer's weights and biases zero the network is its bypass alone."""
    rng = np.random.default_rng(11)
    dims = (3, 4, 2, 3)
    n_layers_params = ws.n_params(*dims)
    theta = np.zeros(ws.n_params(*dims, skip=True))
    Ws = rng.standard_normal((2, 3, 3, 3))
    theta[n_layers_params:] = Ws.ravel()
    x = rng.standard_normal((1, 4, 4, 3))
    assert np.allclose(ws.forward(theta, x, *dims, skip=True)[0], ws.conv3x3(x, Ws, np.zeros(2)))


def test_channel_rms():
    d = np.array([[[3.0, 0.0], [4.0, 1.0]]])
    assert np.allclose(ws.channel_rms(d), [np.sqrt(12.5), np.sqrt(0.5)])


def test_scatter_averages_the_copies_of_a_shared_node():
    """2D, 2x2 cells, Q2: the centre node (global (2, 2) on the 5x5 grid) lies in all four
    cells; one copy set to 4 and the rest 0 averages to 1."""
    geo = SlabGeometry(2, 2, 1, 0, 1.0, 0.1)
    idx = ws.cell_index_map(geo)
    centre = 2 * 5 + 2                                   # v_x of the centre node, a = 0
    copies = np.argwhere(idx == centre)
    assert len(copies) == 4
    cells = np.zeros(idx.shape)
    cells[tuple(copies[0])] = 4.0
    out = ws.cells_scatter_add(geo, cells, np.zeros(geo.size))
    assert out[centre] == 1.0 and np.count_nonzero(out) == 1


@pytest.mark.parametrize("dim,n,r,k", [(2, 3, 2, 1), (3, 2, 1, 1)])
def test_gather_adjoint_is_the_adjoint_of_the_scatter(dim, n, r, k):
    geo = SlabGeometry(dim, n, r, k, 1.0, 0.1)
    rng = np.random.default_rng(12)
    c = rng.standard_normal((n ** dim, ws.n_channels(dim, r, k)))
    x = rng.standard_normal(geo.size)
    s = rng.uniform(0.5, 2.0, c.shape[1])
    lhs = ws.cells_scatter_add(geo, c, np.zeros(geo.size), s) @ x
    rhs = (c * ws.cells_gather_adjoint(geo, x, s)).sum()
    assert np.isclose(lhs, rhs, rtol=1e-12)
