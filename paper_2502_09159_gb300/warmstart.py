"""Learned initial guess for the slab solves (include/stmg_net.h).  Argument marshalling
and the training loop's bookkeeping only: gathers, the network, the loss, the optimiser
and the scatter all run in libstmg's kernels.

The guess for slab n from the solution x_{n-1} of slab n-1 is

    c = gather(x_{n-1}),   a = rms(c)
    x_guess = E x_{n-1} + scatter( a * s_out * net( c / (a * s_in) ) )

E the extrapolation of the DG(k) polynomial to the next slab, gather/scatter the
cell-tensor maps of the finest level, a the sample's own amplitude (the map from one
slab to the next is linear, so inputs and targets are divided by it: samples of any
amplitude weigh alike), s_in and s_out per-channel RMS scales of the amplitude-normalised
training inputs and targets.  The network learns the part e = x_n - E x_{n-1} that
extrapolation misses, from pairs (x_{n-1}, x_n) of slabs the method itself has solved:
first by the mean squared error in cell-tensor space (`fit`), then on what FGMRES sees,
the initial residual ||S (e - u)|| relative to ||S e||, u the network's correction
(`fit_residual`; gradients through S^T).  A correction that is small in L2 but rough
from cell to cell has a large residual; the second stage removes that.  FGMRES with the
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
                 max_batch: int = 8, seed: int = 0, skip: bool = False):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("ConvNet needs a CUDA device (no CPU fallback)")
        self._lib = load()
        self.H, self.W, self.c_in, self.c_out, self.hidden, self.layers = H, W, c_in, c_out, hidden, layers
        self.skip = bool(skip)
        self.max_batch = max_batch
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        check("stmg_net_create", self._lib.stmg_net_create(H, W, c_in, hidden, c_out, layers, int(skip), max_batch,
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


def tensor_rms(data):
    """(rms, 1/rms) of all entries of a float32 CUDA tensor, as 1-element device tensors."""
    torch = _torch()
    lib = load()
    rms = torch.empty(1, dtype=torch.float32, device=data.device)
    inv = torch.empty_like(rms)
    check("stmg_tensor_rms", lib.stmg_tensor_rms(data.numel(), _ptr(data), _ptr(rms), _ptr(inv), _stream_ptr()))
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
                 seed: int = 0, skip: bool = True, residual_pairs: bool = True, history: int = 1):
        torch = _torch()
        if mg.dim != 2:
            raise NotImplementedError("the learned guess uses 2D convolutions (dim = 2 only)")
        self.mg = mg
        self.n = mg.levels[0]["n"]
        self.C = mg.n_channels(0)
        if history not in (1, 2):
            raise ValueError("history: 1 (the previous slab) or 2 (the two previous slabs)")
        self.history = history
        self.Cin = history * self.C
        self.net = ConvNet(self.n, self.n, self.Cin, self.C, hidden, layers, max_batch, seed, skip)
        self.capacity = capacity
        self.inputs = torch.empty((capacity, self.n, self.n, self.Cin), dtype=torch.float32, device=mg.device)
        self.targets = torch.empty((capacity, self.n, self.n, self.C), dtype=torch.float32, device=mg.device)
        self.count = 0
        self.inv_in = self.s_out = None
        self._ext = mg.empty(0)
        self._cells = torch.empty((self.n * self.n, self.Cin), dtype=torch.float32, device=mg.device)
        self._out = torch.empty((1, self.n, self.n, self.C), dtype=torch.float32, device=mg.device)
        self._amp = torch.empty(1, dtype=torch.float32, device=mg.device)
        self._inv_amp = torch.empty(1, dtype=torch.float32, device=mg.device)
        # per pair, for the residual stage: S e (FP64), the amplitude a and ||S e||^2
        self.residual_pairs = residual_pairs
        self.Se = [] if residual_pairs else None
        self.amps = torch.empty(capacity, dtype=torch.float32, device=mg.device)
        self.dens = torch.empty(capacity, dtype=torch.float64, device=mg.device)
        self._tmp = mg.empty(0)

    def _gather_input(self, x_prev, x_prev2, out):
        """Input cell tensor: gather(x_prev), or [gather(x_prev2), gather(x_prev)] along the
        channels with history 2."""
        if self.history == 1:
            self.mg.cells_gather(x_prev, out=out)
        else:
            if x_prev2 is None:
                raise ValueError("history 2 needs the slab before the previous one (x_prev2)")
            self.mg.cells_gather_strided(x_prev2, out, self.Cin, 0)
            self.mg.cells_gather_strided(x_prev, out, self.Cin, self.C)

    def add_pair(self, x_prev, x_next, x_prev2=None):
        """Store one training pair: input gather(x_prev) (with history 2 stacked after
        gather(x_prev2)), target gather(x_next - E x_prev), both divided by the input's
        amplitude."""
        if self.inv_in is not None:
            raise RuntimeError("add_pair after fit")
        if self.count >= self.capacity:
            raise RuntimeError("training set is full")
        i = self.count
        xi, yi = self.inputs[i].view(-1, self.Cin), self.targets[i].view(-1, self.C)
        self._gather_input(x_prev, x_prev2, xi)
        lib = load()
        inv = self._inv_amp
        check("stmg_tensor_rms", lib.stmg_tensor_rms(xi.numel(), _ptr(xi), _ptr(self.amps[i:i + 1]), _ptr(inv),
                                                     _stream_ptr()))
        scale_channels(xi, inv)
        self.mg.extrapolate(x_prev, out=self._ext)
        self.mg.cells_gather(x_next, base=self._ext, out=yi)
        scale_channels(yi, inv)
        if self.residual_pairs:
            # S e = S x_next - S E x_prev, by an apply and a residual (no vector arithmetic)
            Se = self.mg.empty(0)
            self.mg.apply(x_next, 0, out=self._tmp)
            self.mg.residual(self._tmp, self._ext, 0, out=Se)
            self.mg.dot(Se, Se, out=self.dens[i:i + 1])
            self.Se.append(Se)
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
            _, self.inv_in = channel_rms(X, self.Cin)
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

    def fit_residual(self, steps: int = 200, batch: int = 4, lr: float = 3e-4, lr_final: float = 1e-5,
                     seed: int = 1, warmup: int = 50):
        """Fine-tune on L = mean_b ||S e_b - S u_b||^2 / ||S e_b||^2, u_b = a_b scatter(s_out *
        net(x_b)): the squared initial-residual ratio of the learned guess to the
        extrapolated one (1 = no gain).  Gradient dL/du_b = -2 S^T r_b / ||S e_b||^2, taken
        back to cell tensors by the scatter's adjoint.  The residual is stiff in the
        network's output (rough corrections are amplified by S), so the learning rate
        ramps up linearly over `warmup` steps before its cosine decay.  Returns the per-step
        losses."""
        torch = _torch()
        if not self.residual_pairs:
            raise RuntimeError("fit_residual needs residual_pairs=True")
        if self.inv_in is None:
            self.fit(steps=0)                               # normalisation statistics only
        n = self.count
        X = self.inputs[:n]
        batch = min(batch, n, self.net.max_batch)
        # per-pair scale vectors of the scatter (a_b s_out) and of the adjoint gather
        amps = self.amps[:n].double().cpu().numpy()
        dens = self.dens[:n].cpu().numpy()
        s_out = self.s_out.double().cpu().numpy()
        fs = torch.from_numpy(np.stack([a * s_out for a in amps]).astype(np.float32)).to(self.mg.device)
        gs = torch.from_numpy(np.stack([-2.0 * a / (batch * d) * s_out for a, d in zip(amps, dens)])
                              .astype(np.float32)).to(self.mg.device)
        self.net.set_params(self.net.params())              # fresh Adam moments
        rng = np.random.default_rng(seed)
        order = np.concatenate([rng.permutation(n) for _ in range((steps * batch) // n + 2)]).astype(np.int32)
        order = order[:steps * batch].reshape(steps, batch)
        idx = torch.from_numpy(order).to(self.mg.device)
        pred = torch.empty((batch, self.n, self.n, self.C), dtype=torch.float32, device=self.mg.device)
        gpred = torch.empty_like(pred)
        u, r, z = self.mg.empty(0), self.mg.empty(0), self.mg.empty(0)
        rr = torch.zeros((steps, batch), dtype=torch.float64, device=self.mg.device)
        for s in range(steps):
            self.net.forward(X, index=idx[s], out=pred)
            for j, b in enumerate(order[s]):
                u.zero_()
                self.mg.cells_scatter_add(pred[j].view(-1, self.C), u, scale=fs[b])
                self.mg.residual(self.Se[b], u, 0, out=r)
                self.mg.dot(r, r, out=rr[s, j:j + 1])
                self.mg.apply_transpose(r, 0, out=z)
                self.mg.cells_gather_adjoint(z, scale=gs[b], out=gpred[j].view(-1, self.C))
            self.net.backward(X, gpred, index=idx[s])
            if s < warmup:
                a = lr * (s + 1) / warmup
            else:
                a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * (s - warmup) / max(1, steps - warmup - 1)))
            self.net.adam(float(a), s + 1)
        return (rr.cpu().numpy() / dens[order]).mean(axis=1)

    def residual_ratio(self):
        """Mean over the stored pairs of ||S (e - u)||^2 / ||S e||^2 for the current network."""
        torch = _torch()
        n = self.count
        out = torch.empty((1, self.n, self.n, self.C), dtype=torch.float32, device=self.mg.device)
        u, r = self.mg.empty(0), self.mg.empty(0)
        amps = self.amps[:n].double().cpu().numpy()
        vals = torch.zeros(n, dtype=torch.float64, device=self.mg.device)
        for b in range(n):
            self.net.forward(self.inputs[b:b + 1], out=out)
            fs = (self.s_out * float(amps[b])).contiguous()
            u.zero_()
            self.mg.cells_scatter_add(out.view(-1, self.C), u, scale=fs)
            self.mg.residual(self.Se[b], u, 0, out=r)
            self.mg.dot(r, r, out=vals[b:b + 1])
        return float((vals.cpu().numpy() / self.dens[:n].cpu().numpy()).mean())

    def guess(self, x_prev, mode: str = "net", out=None, x_prev2=None):
        """Initial guess for the next slab from the previous slab's solution (and, with
        history 2, the one before it)."""
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
        self._gather_input(x_prev, x_prev2, self._cells)
        lib = load()
        check("stmg_tensor_rms", lib.stmg_tensor_rms(self._cells.numel(), _ptr(self._cells), _ptr(self._amp),
                                                     _ptr(self._inv_amp), _stream_ptr()))
        scale_channels(self._cells, self._inv_amp)
        scale_channels(self._cells, self.inv_in)
        self.net.forward(self._cells, out=self._out)
        scale_channels(self._out, self._amp)
        self.mg.cells_scatter_add(self._out, x, scale=self.s_out)
        return x
