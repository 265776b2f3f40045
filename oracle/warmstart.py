"""Oracle of the learned warm start: cell tensors, temporal extrapolation, the convolutional
network (forward, backward, loss, Adam) in FP64 numpy.

Test infrastructure only (see oracle/__init__.py).  The paper has no learned warm start
(its slabs start from the previous slab's data through the coupling of Eq. InAlg only);
this part defines what the learned initial guess computes so that the GPU kernels can be
checked element by element.  Definitions:

* Cell tensor of a slab vector (layout of Eq. DefX, conventions of oracle/fe.py): one row
  per cell (cells lexicographic, x fastest), C = (k+1) (d (r+2)^d + dim P_r) channels:
  first the velocity values (temporal dof a, component, local node with x fastest), then
  the pressure modes (temporal dof a, mode).  Nodes shared by neighbouring cells appear in
  every cell that contains them.
* Scatter of a cell tensor back to a slab vector: the average over the copies of each
  velocity node; pressure modes have one copy.  Dirichlet entries are left alone.
* Temporal extrapolation: the DG(k) polynomial of the previous slab (Lagrange basis at the
  right Radau points, Eq. BasYk) evaluated at the next slab's nodes; on the reference
  interval the next slab's node s_a lies at s_a + 2.
* Network: L convolutions of size 3x3 with zero padding on the H x W grid of cells,
  channels c_in -> hidden -> ... -> hidden -> c_out, bias, ReLU after every layer except
  the last; optionally a linear bypass, one more 3x3 convolution (no bias) from the input
  straight to the output, added to the last layer's result.  Tensors are NHWC; weights
  W[o, ky, kx, c], then the bias; layer after layer in one flat parameter vector, the
  bypass weights last.
      y[b, i, j, o] = bias[o] + sum_{ky, kx, c} W[o, ky, kx, c] x[b, i + ky - 1, j + kx - 1, c]
* Loss: the mean of (pred - target)^2 over all elements.
* Adam (Kingma and Ba, 2015) with bias correction.

Pins (tests/test_oracle_warmstart.py): the convolution against scipy.signal.correlate2d,
the backward pass and the loss gradient against central finite differences, Adam's first
step against its closed form, scatter(gather(x)) = x, the adjoint identity
<scatter(c), x> = <c, adjoint(x)>, the extrapolation matrix of DG(1) against the
hand-derived values and exactness on polynomials of degree <= k.
"""
from __future__ import annotations

from math import comb

import numpy as np

from .fe import lagrange_values, radau_right


# ---------------------------------------------------------------------------
# Cell tensors
# ---------------------------------------------------------------------------
def n_channels(dim, r, k):
    return (k + 1) * (dim * (r + 2) ** dim + comb(r + dim, dim))


def cell_index_map(geo):
    """[n_cells, C] slab index of every (cell, channel) of the cell tensor."""
    sp_ = geo.space
    P = sp_.np1 ** geo.dim
    C = n_channels(geo.dim, geo.r, geo.k)
    idx = np.zeros((sp_.n_cells, C), dtype=np.int64)
    ch = 0
    for a in range(geo.kt):
        for comp in range(geo.dim):
            idx[:, ch:ch + P] = a * geo.nv + comp * sp_.n_nodes + sp_.cell_nodes
            ch += P
    o = geo.kt * geo.nv
    cells = np.arange(sp_.n_cells)
    for a in range(geo.kt):
        for m in range(sp_.n_pm):
            idx[:, ch] = o + a * geo.npr + cells * sp_.n_pm + m
            ch += 1
    assert ch == C
    return idx


def cells_gather(geo, x, base=None, inv_scale=None):
    """cells[c, ch] = (x - base)[map[c, ch]] * inv_scale[ch], computed in FP64."""
    idx = cell_index_map(geo)
    v = x[idx] - (base[idx] if base is not None else 0.0)
    if inv_scale is not None:
        v = v * np.asarray(inv_scale, dtype=np.float64)[None, :]
    return v


def cells_scatter_add(geo, cells, x, scale=None):
    """x + average over copies of scale * cells on every non-Dirichlet entry."""
    idx = cell_index_map(geo)
    v = cells * (np.asarray(scale, dtype=np.float64)[None, :] if scale is not None else 1.0)
    acc = np.zeros(geo.size)
    cnt = np.zeros(geo.size)
    np.add.at(acc, idx.ravel(), v.ravel())
    np.add.at(cnt, idx.ravel(), 1.0)
    out = x.copy()
    free = ~geo.dirichlet
    out[free] += acc[free] / cnt[free]
    return out


def cells_gather_adjoint(geo, x, scale=None):
    """The adjoint of cells_scatter_add (x -> cells): each copy of a non-Dirichlet entry g
    receives scale[ch] x[g] / (number of copies of g); copies of Dirichlet entries get 0."""
    idx = cell_index_map(geo)
    cnt = np.bincount(idx.ravel(), minlength=geo.size).astype(float)
    w = np.where(geo.dirichlet, 0.0, x / cnt)
    v = w[idx]
    if scale is not None:
        v = v * np.asarray(scale, dtype=np.float64)[None, :]
    return v


def channel_rms(data):
    """Root mean square of every channel (last axis) over all other axes."""
    d = np.asarray(data, dtype=np.float64)
    return np.sqrt((d.reshape(-1, d.shape[-1]) ** 2).mean(axis=0))


# ---------------------------------------------------------------------------
# Temporal extrapolation of the DG(k) polynomial
# ---------------------------------------------------------------------------
def extrapolation_matrix(k):
    """E[a, b] = phi_b(s_a + 2): the previous slab's basis at the next slab's nodes."""
    s, _ = radau_right(k)
    return lagrange_values(s, s + 2.0).T


def extrapolate(geo, x_prev):
    E = extrapolation_matrix(geo.k)
    out = np.zeros(geo.size)
    for blk, o in ((geo.nv, 0), (geo.npr, geo.kt * geo.nv)):
        X = x_prev[o:o + geo.kt * blk].reshape(geo.kt, blk)
        out[o:o + geo.kt * blk] = (E @ X).ravel()
    return out


# ---------------------------------------------------------------------------
# Convolutional network
# ---------------------------------------------------------------------------
def layer_shapes(c_in, hidden, c_out, n_layers):
    chans = [c_in] + [hidden] * (n_layers - 1) + [c_out]
    return [(chans[l + 1], chans[l]) for l in range(n_layers)]


def n_params(c_in, hidden, c_out, n_layers, skip=False):
    return sum(o * 9 * c + o for o, c in layer_shapes(c_in, hidden, c_out, n_layers)) + \
        (c_out * 9 * c_in if skip else 0)


def unpack(theta, c_in, hidden, c_out, n_layers, skip=False):
    """Flat parameter vector -> ([(W[o, 3, 3, c], bias[o])] per layer, bypass W or None)."""
    out, p = [], 0
    for o, c in layer_shapes(c_in, hidden, c_out, n_layers):
        W = theta[p:p + o * 9 * c].reshape(o, 3, 3, c)
        p += o * 9 * c
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    Ws = None
    if skip:
        Ws = theta[p:p + c_out * 9 * c_in].reshape(c_out, 3, 3, c_in)
        p += c_out * 9 * c_in
    assert p == len(theta)
    return out, Ws


def conv3x3(x, W, b):
    """Zero-padded 3x3 convolution (cross-correlation) of NHWC x with W[o, ky, kx, c]."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (B, H, Wd, W.shape[0])).copy()
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bijc,oc->bijo", xp[:, ky:ky + H, kx:kx + Wd, :], W[:, ky, kx, :])
    return y


def conv3x3_grad_input(g, W):
    """d(sum g * conv3x3(x)) / dx: the adjoint of the convolution applied to g."""
    B, H, Wd, _ = g.shape
    gx = np.zeros((B, H + 2, Wd + 2, W.shape[3]))
    for ky in range(3):
        for kx in range(3):
            gx[:, ky:ky + H, kx:kx + Wd, :] += np.einsum("bijo,oc->bijc", g, W[:, ky, kx, :])
    return gx[:, 1:H + 1, 1:Wd + 1, :]


def conv3x3_grad_weights(x, g):
    """(dW[o, ky, kx, c], dbias[o]) of sum g * conv3x3(x)."""
    B, H, Wd, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dW = np.zeros((g.shape[3], 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("bijo,bijc->oc", g, xp[:, ky:ky + H, kx:kx + Wd, :])
    return dW, g.sum(axis=(0, 1, 2))


def forward(theta, x, c_in, hidden, c_out, n_layers, skip=False):
    """Network output and the input of every layer (for the backward pass)."""
    layers, Ws = unpack(theta, c_in, hidden, c_out, n_layers, skip)
    acts = [x]
    h = x
    for l, (W, b) in enumerate(layers):
        h = conv3x3(h, W, b)
        if l < n_layers - 1:
            h = np.maximum(h, 0.0)
            acts.append(h)
    if skip:
        h = h + conv3x3(x, Ws, np.zeros(c_out))
    return h, acts


def backward(theta, acts, g_out, c_in, hidden, c_out, n_layers, skip=False):
    """Gradient of sum(g_out * network(x)) with respect to the flat parameters."""
    layers, _ = unpack(theta, c_in, hidden, c_out, n_layers, skip)
    grads = [None] * n_layers
    g = g_out
    for l in range(n_layers - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = conv3x3_grad_weights(acts[l], g)
        if l > 0:
            g = conv3x3_grad_input(g, W) * (acts[l] > 0.0)
    flat = [np.concatenate([dW.ravel(), db]) for dW, db in grads]
    if skip:
        flat.append(conv3x3_grad_weights(acts[0], g_out)[0].ravel())
    return np.concatenate(flat)


def mse(pred, target):
    """(loss, d loss / d pred) of the mean squared error."""
    d = pred - target
    return float((d * d).mean()), 2.0 * d / d.size


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) at step number `step` >= 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
