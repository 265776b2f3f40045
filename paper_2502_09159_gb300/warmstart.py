"""Learned initial guess for the slab solves (include/stmg_net.h).  Argument marshalling
and the training loop's bookkeeping only: gathers, the network, the loss, the optimiser
and the scatter all run in libstmg's kernels.

The guess for slab n from the solution x_{n-1} of slab n-1 is

    x_guess = E x_{n-1} + scatter( s_out * net( gather(x_{n-1}) * (1 / s_in) ) )

E the extrapolation of the DG(k) polynomial to the next slab, gather/scatter the
cell-tensor maps of the finest level, s_in and s_out per-channel RMS scales of the
training inputs and targets.  The network learns the part of x_n that extrapolation
misses, from pairs (x_{n-1}, x_n) of slabs the method itself has solved.  FGMRES with the
multigrid preconditioner always finishes the solve; the guess only changes where it
starts.

    ws = WarmStart(mg)                # mg: SpaceTimeMG, 2D
    ws.add_pair(x_prev, x_next)       # for the training slabs
    ws.fit(steps=600)
    x0 = ws.guess(x_prev)             # "net"; also "extrapolate" and "zero"
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import check, load


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class ConvNet:
    """The fully convolutional network of stmg_net.h on H x W grids (NHWC FP32)."""

    def __init__(self, H: int, W: int, c_in: int, c_out: int, hidden: int = 64, layers: int = 4,
                 max_batch: int = 8, seed: int = 0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("ConvNet needs a CUDA device (no CPU fallback)")
        self._lib = load()
        self.H, self.W, self.c_in, self.c_out, self.hidden, self.layers = H, W, c_in, c_out, hidden, layers
        self.max_batch = max_batch
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        check("stmg_net_create", self._lib.stmg_net_create(H, W, c_in, hidden, c_out, layers, max_batch,
                                                           C.c_ulonglong(seed), C.byref(h)))
        self._h = h
        n = C.c_longlong()
        check("stmg_net_num_params", self._lib.stmg_net_num_params(h, C.byref(n)))
        self.n_params = n.value
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stmg_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _s(self):
        self._lib.stmg_net_set_stream(self._h, _stream_ptr())

    def _chk(self, t, name, C_=None, dtype=None):
        torch = _torch()
        dtype = dtype or torch.float32
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {dtype} CUDA tensor")
        if C_ is not None and t.numel() % (self.H * self.W * C_) != 0:
            raise ValueError(f"{name}: size is not a multiple of H*W*{C_}")

    def _batch(self, x, C_, index):
        if index is not None:
            self._chk(index, "index", dtype=_torch().int32)
            return index.numel()
        return x.numel() // (self.H * self.W * C_)

    def params(self):
        torch = _torch()
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._s()
        check("stmg_net_get_params", self._lib.stmg_net_get_params(self._h, _ptr(p)))
        return p

    def set_params(self, p):
        self._chk(p, "params")
        if p.numel() != self.n_params:
            raise ValueError("params: wrong length")
        self._s()
        check("stmg_net_set_params", self._lib.stmg_net_set_params(self._h, _ptr(p)))

    def grads(self):
        torch = _torch()
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._s()
        check("stmg_net_get_grads", self._lib.stmg_net_get_grads(self._h, _ptr(g)))
        return g

    def forward(self, x, index=None, out=None):
        torch = _torch()
        self._chk(x, "x", self.c_in)
        B = self._batch(x, self.c_in, index)
        y = out if out is not None else torch.empty((B, self.H, self.W, self.c_out), dtype=torch.float32,
                                                    device=self.device)
        self._chk(y, "out", self.c_out)
        self._s()
        check("stmg_net_forward", self._lib.stmg_net_forward(self._h, B, _ptr(x), _ptr(index), _ptr(y)))
        return y

    def backward(self, x, grad_out, index=None):
        self._chk(x, "x", self.c_in)
        self._chk(grad_out, "grad_out", self.c_out)
        B = self._batch(x, self.c_in, index)
        self._s()
        check("stmg_net_backward", self._lib.stmg_net_backward(self._h, B, _ptr(x), _ptr(index), _ptr(grad_out)))
        return self.grads()

    def mse(self, pred, target, index=None):
        """(loss as a 1-element float64 CUDA tensor, d loss / d pred)."""
        torch = _torch()
        self._chk(pred, "pred", self.c_out)
        self._chk(target, "target", self.c_out)
        B = pred.numel() // (self.H * self.W * self.c_out)
        if index is not None and index.numel() != B:
            raise ValueError("index: one entry per prediction")
        g = torch.empty_like(pred)
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        self._s()
        check("stmg_net_mse", self._lib.stmg_net_mse(self._h, B, _ptr(pred), _ptr(target), _ptr(index), _ptr(g),
                                                     _ptr(loss)))
        return loss, g

    def adam(self, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8):
        self._s()
        check("stmg_net_adam", self._lib.stmg_net_adam(self._h, lr, beta1, beta2, eps, step))

    def train_step(self, inputs, targets, index, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8,
                   loss_out=None):
        self._chk(inputs, "inputs", self.c_in)
        self._chk(targets, "targets", self.c_out)
        B = self._batch(inputs, self.c_in, index)
        self._s()
        check("stmg_net_train_step", self._lib.stmg_net_train_step(
            self._h, B, _ptr(inputs), _ptr(targets), _ptr(index), lr, beta1, beta2, eps, step,
            _ptr(loss_out)))
        return loss_out


def channel_rms(data, C_: int):
    """(rms, 1/rms) per channel of a float32 CUDA tensor whose last axis has C_ entries."""
    torch = _torch()
    lib = load()
    rms = torch.empty(C_, dtype=torch.float32, device=data.device)
    inv = torch.empty_like(rms)
    check("stmg_channel_rms", lib.stmg_channel_rms(data.numel() // C_, C_, _ptr(data), _ptr(rms), _ptr(inv),
                                                   _stream_ptr()))
    return rms, inv


def scale_channels(data, s):
    lib = load()
    check("stmg_scale_channels", lib.stmg_scale_channels(data.numel() // s.numel(), s.numel(), _ptr(data), _ptr(s),
                                                         _stream_ptr()))
    return data


class WarmStart:
    """Learned initial guess on the finest level of a 2D SpaceTimeMG handle."""

    MODES = ("zero", "extrapolate", "net")

    def __init__(self, mg, hidden: int = 64, layers: int = 4, max_batch: int = 8, capacity: int = 128,
                 seed: int = 0):
        torch = _torch()
        if mg.dim != 2:
            raise NotImplementedError("the learned guess uses 2D convolutions (dim = 2 only)")
        self.mg = mg
        self.n = mg.levels[0]["n"]
        self.C = mg.n_channels(0)
        self.net = ConvNet(self.n, self.n, self.C, self.C, hidden, layers, max_batch, seed)
        self.capacity = capacity
        shape = (capacity, self.n, self.n, self.C)
        self.inputs = torch.empty(shape, dtype=torch.float32, device=mg.device)
        self.targets = torch.empty(shape, dtype=torch.float32, device=mg.device)
        self.count = 0
        self.inv_in = self.s_out = None
        self._ext = mg.empty(0)
        self._cells = torch.empty((self.n * self.n, self.C), dtype=torch.float32, device=mg.device)
        self._out = torch.empty((1, self.n, self.n, self.C), dtype=torch.float32, device=mg.device)

    def add_pair(self, x_prev, x_next):
        """Store one training pair: input gather(x_prev), target gather(x_next - E x_prev)."""
        if self.inv_in is not None:
            raise RuntimeError("add_pair after fit")
        if self.count >= self.capacity:
            raise RuntimeError("training set is full")
        i = self.count
        self.mg.cells_gather(x_prev, out=self.inputs[i].view(-1, self.C))
        self.mg.extrapolate(x_prev, out=self._ext)
        self.mg.cells_gather(x_next, base=self._ext, out=self.targets[i].view(-1, self.C))
        self.count += 1

    def fit(self, steps: int = 600, batch: int = 8, lr: float = 1e-3, lr_final: float = 1e-5, seed: int = 0):
        """Adam on minibatches of the stored pairs (cosine learning-rate decay from lr to
        lr_final); returns the per-step minibatch losses (host numpy array)."""
        torch = _torch()
        if self.count < 1:
            raise RuntimeError("no training pairs")
        n = self.count
        X, Y = self.inputs[:n], self.targets[:n]
        if self.inv_in is None:
            _, self.inv_in = channel_rms(X, self.C)
            self.s_out, inv_out = channel_rms(Y, self.C)
            scale_channels(X, self.inv_in)
            scale_channels(Y, inv_out)
        batch = min(batch, n, self.net.max_batch)
        rng = np.random.default_rng(seed)
        order = np.concatenate([rng.permutation(n) for _ in range((steps * batch) // n + 2)]).astype(np.int32)
        idx = torch.from_numpy(order[:steps * batch].reshape(steps, batch)).to(self.mg.device)
        losses = torch.zeros(steps, dtype=torch.float64, device=self.mg.device)
        for s in range(steps):
            a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * s / max(1, steps - 1)))
            self.net.train_step(X, Y, idx[s], float(a), s + 1, loss_out=losses[s:s + 1])
        return losses.cpu().numpy()

    def guess(self, x_prev, mode: str = "net", out=None):
        """Initial guess for the next slab from the previous slab's solution."""
        torch = _torch()
        if mode not in self.MODES:
            raise ValueError(f"mode must be one of {self.MODES}")
        x = out if out is not None else self.mg.empty(0)
        if mode == "zero":
            return x.zero_()
        self.mg.extrapolate(x_prev, out=x)
        if mode == "extrapolate":
            return x
        if self.inv_in is None:
            raise RuntimeError("guess(mode='net') before fit")
        self.mg.cells_gather(x_prev, inv_scale=self.inv_in, out=self._cells)
        self.net.forward(self._cells, out=self._out)
        self.mg.cells_scatter_add(self._out, x, scale=self.s_out)
        return x
