"""GB300 hp space-time multigrid for the instationary Stokes equations.

Python face of libstmg (include/stmg.h): argument marshalling only.  Every step of the
method runs in the library's CUDA kernels; PyTorch supplies device memory and streams.
There is no CPU fallback: if libstmg.so has not been built, importing works but every
call raises.

    from paper_2502_09159_gb300 import SpaceTimeMG
    mg = SpaceTimeMG(dim=2, n_cells=64, r=2, k=2, n_slabs=16, precond_precision="fp32")
    b = mg.slab_rhs(mg.forcing(f, slab=0))
    x, info = mg.solve_slab(b)
"""
from __future__ import annotations

import ctypes as C
from typing import Callable, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import CELL, FP32, FP64, VSP, StmgError, check, load

__all__ = ["SpaceTimeMG", "StmgError", "FP64", "FP32", "CELL", "VSP", "host_default_hierarchy",
           "host_tables_1d", "host_time_tables", "host_patch", "host_valence", "host_coarse_inverse",
           "host_invert",
           "build"]

_PREC = {"fp64": FP64, "fp32": FP32, FP64: FP64, FP32: FP32}


def build(force: bool = False) -> str:
    from .builder import build as _b
    return _b(force=force)


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class SpaceTimeMG:
    """One slab system of the space-time Stokes discretisation plus its hp multigrid."""

    def __init__(self, dim: int = 2, n_cells: int = 8, r: int = 1, k: int = 1, nu: float = 1.0,
                 T: float = 1.0, n_slabs: int = 4, levels: Optional[Sequence[Sequence[int]]] = None,
                 smoothers: Optional[Sequence[int]] = None, omega: float = 0.7, nu1: int = 1,
                 nu2: int = 1, precond_precision="fp64", precisions=("fp64", "fp32"),
                 gmres_max_iter: int = 200, rel_tol: float = 1e-8, use_graphs: bool = True,
                 sweep_variant: int = 0, autotune: bool = True, coarse_n: int = 1, k_min: int = 1,
                 n_sub: int = 1, half_inverses: bool = False, transfer_variant: int = 0,
                 apply_variant: int = 0, persistent: int = 1, time_h: bool = False,
                 arnoldi_form: int = 0, fuse_transfers: bool = True):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("SpaceTimeMG needs a CUDA device (no CPU fallback)")
        lib = load()
        cfg = _lib.Config()
        check("stmg_default_config", lib.stmg_default_config(C.byref(cfg)))
        cfg.dim, cfg.n_cells, cfg.r, cfg.k = dim, n_cells, r, k
        cfg.nu, cfg.T, cfg.n_slabs = nu, T, n_slabs
        if levels:
            cfg.n_levels = len(levels)
            for i, lvl in enumerate(levels):
                cfg.level_n[i], cfg.level_r[i], cfg.level_k[i] = lvl[0], lvl[1], lvl[2]
                cfg.level_nsub[i] = lvl[3] if len(lvl) > 3 else 0        # (n, r, k[, n_sub])
        if smoothers is not None:
            for i, s in enumerate(smoothers):
                cfg.smoother[i] = s
        cfg.omega, cfg.nu1, cfg.nu2 = omega, nu1, nu2
        cfg.precond_precision = _PREC[precond_precision]
        cfg.precisions = sum(1 << _PREC[p] for p in precisions)
        cfg.gmres_max_iter, cfg.rel_tol = gmres_max_iter, rel_tol
        cfg.use_graphs = int(use_graphs)
        cfg.sweep_variant = int(sweep_variant)
        cfg.autotune = int(autotune)
        cfg.coarse_n = int(coarse_n)
        cfg.k_min = int(k_min)
        cfg.n_sub = int(n_sub)
        cfg.half_inverses = int(half_inverses)
        cfg.transfer_variant = int(transfer_variant)
        cfg.apply_variant = int(apply_variant)
        cfg.persistent = int(persistent)
        cfg.time_h = int(time_h)
        cfg.arnoldi_form = int(arnoldi_form)
        cfg.fuse_transfers = int(fuse_transfers)
        self.cfg = cfg
        self.dim, self.r, self.k, self.n_sub = dim, r, k, int(n_sub)
        self.kt = self.n_sub * (k + 1)
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        check("stmg_create", lib.stmg_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._lib = lib
        n = C.c_int()
        check("stmg_num_levels", lib.stmg_num_levels(h, C.byref(n)))
        self.levels = []
        for l in range(n.value):
            li = _lib.LevelInfo()
            check("stmg_level_info", lib.stmg_level_info(h, l, C.byref(li)))
            self.levels.append({"n": li.n, "r": li.r, "k": li.k, "n_sub": li.n_sub, "size": li.size, "n_vel": li.n_vel,
                                "n_pres": li.n_pres, "smoother": li.smoother, "patch_size": li.patch_size,
                                "n_patches": li.n_patches, "n_patch_classes": li.n_patch_classes,
                                "inverse_bytes": tuple(li.inverse_bytes),
                                "sweep_variant": tuple(li.sweep_variant),
                                "patches_per_block": tuple(li.patches_per_block),
                                "apply_cells_per_block": tuple(li.apply_cells_per_block),
                                "transfer_cells_per_block": tuple(li.transfer_cells_per_block),
                                "streaming": li.streaming,
                                "apply_variant": tuple(li.apply_variant),
                                "apply_tile": tuple(tuple(t) for t in li.apply_tile),
                                "persistent": tuple(li.persistent),
                                "sweep_unroll": tuple(li.sweep_unroll)})

    # ---------------------------------------------------------------- plumbing
    def close(self):
        if getattr(self, "_h", None):
            self._lib.stmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        torch = _torch()
        self._lib.stmg_set_stream(self._h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def _vec(self, t, lvl, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: need a contiguous CUDA tensor")
        if t.dtype not in (torch.float64, torch.float32):
            raise ValueError(f"{name}: dtype must be float64 or float32")
        if t.numel() != self.levels[lvl]["size"]:
            raise ValueError(f"{name}: length {t.numel()} != level size {self.levels[lvl]['size']}")
        return FP64 if t.dtype == torch.float64 else FP32

    def size(self, lvl: int = 0) -> int:
        return self.levels[lvl]["size"]

    def empty(self, lvl: int = 0, dtype=None):
        torch = _torch()
        return torch.empty(self.size(lvl), dtype=dtype or torch.float64, device=self.device)

    def zeros(self, lvl: int = 0, dtype=None):
        torch = _torch()
        return torch.zeros(self.size(lvl), dtype=dtype or torch.float64, device=self.device)

    # ---------------------------------------------------------------- hot path
    def apply(self, x, lvl: int = 0, out=None):
        """y = S_lvl x (matrix-free)."""
        p = self._vec(x, lvl, "x")
        y = out if out is not None else self.empty(lvl, x.dtype)
        self._stream()
        check("stmg_apply", self._lib.stmg_apply(self._h, lvl, p, _ptr(x), _ptr(y)))
        return y

    def apply_transpose(self, x, lvl: int = 0, out=None):
        """y = S_lvl^T x (matrix-free)."""
        p = self._vec(x, lvl, "x")
        y = out if out is not None else self.empty(lvl, x.dtype)
        self._stream()
        check("stmg_apply_transpose", self._lib.stmg_apply_transpose(self._h, lvl, p, _ptr(x), _ptr(y)))
        return y

    def residual(self, b, x, lvl: int = 0, out=None):
        """r = b - S_lvl x."""
        p = self._vec(x, lvl, "x")
        self._vec(b, lvl, "b")
        r = out if out is not None else self.empty(lvl, x.dtype)
        self._stream()
        check("stmg_residual", self._lib.stmg_residual(self._h, lvl, p, _ptr(b), _ptr(x), _ptr(r)))
        return r

    def smooth(self, b, x, lvl: int = 0, steps: int = 1):
        """x <- x + omega W (b - S x), `steps` times, in place."""
        p = self._vec(x, lvl, "x")
        self._vec(b, lvl, "b")
        self._stream()
        check("stmg_smooth", self._lib.stmg_smooth(self._h, lvl, p, _ptr(b), _ptr(x), steps))
        return x

    def vanka_sweep(self, res, x, lvl: int = 0):
        """x += omega W res (one additive Vanka correction), in place."""
        p = self._vec(x, lvl, "x")
        self._vec(res, lvl, "res")
        self._stream()
        check("stmg_vanka_sweep", self._lib.stmg_vanka_sweep(self._h, lvl, p, _ptr(res), _ptr(x)))
        return x

    def restrict(self, r_f, lvl_fine: int, out=None):
        p = self._vec(r_f, lvl_fine, "r_f")
        b_c = out if out is not None else self.empty(lvl_fine + 1, r_f.dtype)
        self._stream()
        check("stmg_restrict", self._lib.stmg_restrict(self._h, lvl_fine, p, _ptr(r_f), _ptr(b_c)))
        return b_c

    def prolongate_add(self, y_c, x_f, lvl_fine: int):
        p = self._vec(x_f, lvl_fine, "x_f")
        self._vec(y_c, lvl_fine + 1, "y_c")
        self._stream()
        check("stmg_prolongate_add", self._lib.stmg_prolongate_add(self._h, lvl_fine, p, _ptr(y_c), _ptr(x_f)))
        return x_f

    def coarse_solve(self, b, out=None):
        lvl = len(self.levels) - 1
        p = self._vec(b, lvl, "b")
        x = out if out is not None else self.empty(lvl, b.dtype)
        self._stream()
        check("stmg_coarse_solve", self._lib.stmg_coarse_solve(self._h, p, _ptr(b), _ptr(x)))
        return x

    def vcycle(self, b, prec="fp64", out=None):
        """x = V(b), one hp space-time V-cycle from zero; b, x FP64."""
        torch = _torch()
        if b.dtype != torch.float64:
            raise ValueError("vcycle: b must be float64")
        self._vec(b, 0, "b")
        x = out if out is not None else self.empty(0)
        self._stream()
        check("stmg_vcycle", self._lib.stmg_vcycle(self._h, _PREC[prec], _ptr(b), _ptr(x)))
        return x

    def slab_rhs(self, F, x_prev=None, out=None):
        """b = F + (C_tau (x) M_h) V_prev^{k+1}."""
        self._vec(F, 0, "F")
        if x_prev is not None:
            self._vec(x_prev, 0, "x_prev")
        b = out if out is not None else self.empty(0)
        self._stream()
        check("stmg_slab_rhs", self._lib.stmg_slab_rhs(
            self._h, _ptr(F), _ptr(x_prev) if x_prev is not None else None, _ptr(b)))
        return b

    def dirichlet_lift(self, g, b, out=None):
        """y = b - S_{.,D} g on interior rows, y = g on boundary rows (non-homogeneous
        Dirichlet data g moved to the right-hand side)."""
        self._vec(g, 0, "g")
        self._vec(b, 0, "b")
        y = out if out is not None else self.empty(0)
        self._stream()
        check("stmg_dirichlet_lift", self._lib.stmg_dirichlet_lift(self._h, _ptr(g), _ptr(b), _ptr(y)))
        return y

    def boundary_vector(self, fn: Callable, slab: int):
        """Slab vector (device FP64) holding fn(x, t) -> tuple of dim velocity arrays at the
        boundary velocity nodes for the slab's Radau times t_n^a, zero elsewhere (input
        preparation on the host: node coordinates from the Gauss-Lobatto nodes)."""
        torch = _torch()
        n, r, dim = self.levels[0]["n"], self.r, self.dim
        xi = host_tables_1d(r)["xi"]
        G = (r + 1) * n + 1
        i = np.arange(G)
        cell = np.minimum(i // (r + 1), n - 1)
        coord = (cell + xi[i - cell * (r + 1)]) / n
        idx = np.indices((G,) * dim).reshape(dim, -1)[::-1]          # x fastest
        on_b = np.any((idx == 0) | (idx == G - 1), axis=0)
        nodes = np.nonzero(on_b)[0]
        X = tuple(coord[idx[d, nodes]] for d in range(dim))
        nn = G ** dim
        nv = dim * nn
        out = np.zeros(self.size(0))
        for a, t in enumerate(self.slab_times(slab)):
            vals = fn(X, t)
            for comp in range(dim):
                out[a * nv + comp * nn + nodes] = np.broadcast_to(vals[comp], nodes.shape)
        return torch.from_numpy(out).to(self.device)

    def solve_slab(self, b, x0=None, out=None):
        """FGMRES + V-cycle solve of S x = b; returns (x, info dict)."""
        self._vec(b, 0, "b")
        x = out if out is not None else (x0.clone() if x0 is not None else self.zeros(0))
        if out is not None and x0 is not None and out.data_ptr() != x0.data_ptr():
            x.copy_(x0)
        self._stream()
        info = _lib.SolveInfo()
        st = self._lib.stmg_solve_slab(self._h, _ptr(b), _ptr(x), C.byref(info))
        if st not in (_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_BREAKDOWN):
            raise StmgError("stmg_solve_slab", st)
        return x, {"iterations": info.iterations, "rel_residual": info.rel_residual,
                   "status": info.status, "seconds": info.seconds}

    def solve_slab_host(self, b: np.ndarray, x: np.ndarray):
        """Same with host arrays (float64, contiguous); x is overwritten with the solution."""
        if b.dtype != np.float64 or x.dtype != np.float64 or not b.flags.c_contiguous or not x.flags.c_contiguous:
            raise ValueError("solve_slab_host: contiguous float64 arrays")
        if b.size != self.size(0) or x.size != self.size(0):
            raise ValueError("solve_slab_host: wrong length")
        self._stream()
        info = _lib.SolveInfo()
        st = self._lib.stmg_solve_slab_host(self._h, b.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p),
                                            C.byref(info))
        if st not in (_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_BREAKDOWN):
            raise StmgError("stmg_solve_slab_host", st)
        return {"iterations": info.iterations, "rel_residual": info.rel_residual, "status": info.status,
                "seconds": info.seconds}

    def march_host(self, inputs: np.ndarray, out: np.ndarray, boundary_data: bool = False):
        """Whole time march through stmg_march_host with host arrays: inputs[s] is slab s's
        forcing F_s (or, with boundary_data, its Dirichlet values g_s); out[s] receives x_s.
        Both (n_slabs, D) float64, C-contiguous (pinned memory lets the copies overlap the
        solves).  Returns the per-slab info dicts."""
        for a, name in ((inputs, "inputs"), (out, "out")):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.ndim != 2 or a.shape[1] != self.size(0):
                raise ValueError(f"march_host: {name} must be a C-contiguous float64 (n_slabs, D) array")
        if inputs.shape != out.shape:
            raise ValueError("march_host: inputs and out differ in shape")
        n = inputs.shape[0]
        infos = (_lib.SolveInfo * n)()
        self._stream()
        st = self._lib.stmg_march_host(self._h, n, _lib.MARCH_BOUNDARY if boundary_data else _lib.MARCH_FORCING,
                                       inputs.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p), infos)
        if st != _lib.OK:
            raise StmgError("stmg_march_host", st)
        return [{"iterations": i.iterations, "rel_residual": i.rel_residual, "status": i.status,
                 "seconds": i.seconds} for i in infos]

    # ---------------------------------------------------------------- cell tensors
    def n_channels(self, lvl: int = 0) -> int:
        c = C.c_int()
        check("stmg_cells_channels", self._lib.stmg_cells_channels(self._h, lvl, C.byref(c)))
        return c.value

    def _f32(self, t, n, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() \
                or t.numel() != n:
            raise ValueError(f"{name}: need a contiguous float32 CUDA tensor of {n} entries")

    def cells_gather(self, x, base=None, inv_scale=None, out=None, lvl: int = 0):
        """Cell tensor [n^d, C] (FP32) of (x - base) * inv_scale."""
        torch = _torch()
        if x.dtype != torch.float64:
            raise ValueError("x: float64")
        self._vec(x, lvl, "x")
        if base is not None:
            self._vec(base, lvl, "base")
        Cn = self.n_channels(lvl)
        if inv_scale is not None:
            self._f32(inv_scale, Cn, "inv_scale")
        ncell = self.levels[lvl]["n"] ** self.dim
        cells = out if out is not None else torch.empty((ncell, Cn), dtype=torch.float32, device=self.device)
        self._f32(cells, ncell * Cn, "out")
        self._stream()
        check("stmg_cells_gather", self._lib.stmg_cells_gather(
            self._h, lvl, _ptr(x), _ptr(base) if base is not None else None,
            _ptr(inv_scale) if inv_scale is not None else None, _ptr(cells)))
        return cells

    def cells_gather_strided(self, x, out, row_stride: int, offset: int, base=None, inv_scale=None, lvl: int = 0):
        """Gather into columns offset .. offset + C - 1 of out (rows of row_stride floats)."""
        torch = _torch()
        if x.dtype != torch.float64:
            raise ValueError("x: float64")
        self._vec(x, lvl, "x")
        if base is not None:
            self._vec(base, lvl, "base")
        Cn = self.n_channels(lvl)
        ncell = self.levels[lvl]["n"] ** self.dim
        self._f32(out, ncell * row_stride, "out")
        if inv_scale is not None:
            self._f32(inv_scale, Cn, "inv_scale")
        self._stream()
        check("stmg_cells_gather_strided", self._lib.stmg_cells_gather_strided(
            self._h, lvl, _ptr(x), _ptr(base) if base is not None else None,
            _ptr(inv_scale) if inv_scale is not None else None, _ptr(out), row_stride, offset))
        return out

    def cells_scatter_add(self, cells, x, scale=None, lvl: int = 0):
        """x += average over copies of scale * cells (boundary entries untouched)."""
        self._vec(x, lvl, "x")
        Cn = self.n_channels(lvl)
        self._f32(cells, self.levels[lvl]["n"] ** self.dim * Cn, "cells")
        if scale is not None:
            self._f32(scale, Cn, "scale")
        self._stream()
        check("stmg_cells_scatter_add", self._lib.stmg_cells_scatter_add(
            self._h, lvl, _ptr(cells), _ptr(scale) if scale is not None else None, _ptr(x)))
        return x

    def cells_gather_adjoint(self, x, scale=None, out=None, lvl: int = 0):
        """Adjoint of cells_scatter_add: copies of x divided by their multiplicity."""
        torch = _torch()
        if x.dtype != torch.float64:
            raise ValueError("x: float64")
        self._vec(x, lvl, "x")
        Cn = self.n_channels(lvl)
        if scale is not None:
            self._f32(scale, Cn, "scale")
        ncell = self.levels[lvl]["n"] ** self.dim
        cells = out if out is not None else torch.empty((ncell, Cn), dtype=torch.float32, device=self.device)
        self._f32(cells, ncell * Cn, "out")
        self._stream()
        check("stmg_cells_gather_adjoint", self._lib.stmg_cells_gather_adjoint(
            self._h, lvl, _ptr(x), _ptr(scale) if scale is not None else None, _ptr(cells)))
        return cells

    def dot(self, x, y, out=None):
        """Deterministic FP64 dot product into a 1-element device tensor."""
        torch = _torch()
        if x.dtype != torch.float64 or y.dtype != torch.float64 or x.numel() != y.numel():
            raise ValueError("dot: two float64 tensors of one length")
        o = out if out is not None else torch.empty(1, dtype=torch.float64, device=self.device)
        self._stream()
        check("stmg_dot", self._lib.stmg_dot(self._h, x.numel(), _ptr(x), _ptr(y), _ptr(o)))
        return o

    def extrapolate(self, x_prev, out=None, lvl: int = 0):
        """The previous slab's DG(k) polynomial at the next slab's Radau points."""
        self._vec(x_prev, lvl, "x_prev")
        x = out if out is not None else self.empty(lvl)
        self._stream()
        check("stmg_extrapolate", self._lib.stmg_extrapolate(self._h, lvl, _ptr(x_prev), _ptr(x)))
        return x

    def remove_pressure_mean(self, x, lvl: int = 0):
        self._vec(x, lvl, "x")
        self._stream()
        check("stmg_remove_pressure_mean", self._lib.stmg_remove_pressure_mean(self._h, lvl, _ptr(x)))
        return x

    # ---------------------------------------------------------------- forcing
    def forcing_points(self):
        torch = _torch()
        nq = C.c_int()
        check("stmg_forcing_npoints", self._lib.stmg_forcing_npoints(self._h, C.byref(nq)))
        ncell = self.levels[0]["n"] ** self.dim
        pts = torch.empty((ncell, nq.value, self.dim), dtype=torch.float64, device=self.device)
        check("stmg_forcing_points", self._lib.stmg_forcing_points(self._h, _ptr(pts)))
        return pts

    def slab_times(self, slab: int):
        t = (C.c_double * self.kt)()
        check("stmg_slab_times", self._lib.stmg_slab_times(self._h, slab, t))
        return list(t)

    def assemble_forcing(self, fq, out=None):
        """F from samples fq[a][cell][q][dim] of f at forcing_points() and slab_times()."""
        torch = _torch()
        if fq.dtype != torch.float64 or not fq.is_cuda or not fq.is_contiguous():
            raise ValueError("fq: contiguous float64 CUDA tensor")
        F = out if out is not None else self.empty(0)
        self._stream()
        check("stmg_assemble_forcing", self._lib.stmg_assemble_forcing(self._h, _ptr(fq), _ptr(F)))
        return F

    def sample_forcing(self, f: Callable, slab: int, points=None):
        """Evaluate f(x_tuple, t) -> tuple of dim arrays at the forcing points of `slab`
        (input preparation on the host); returns fq ready for assemble_forcing."""
        torch = _torch()
        pts = (points if points is not None else self.forcing_points()).cpu().numpy()
        X = tuple(pts[..., d] for d in range(self.dim))
        fq = np.stack([np.stack(f(X, t), axis=-1) for t in self.slab_times(slab)])
        return torch.from_numpy(np.ascontiguousarray(fq)).to(self.device)

    def forcing(self, f: Callable, slab: int, points=None):
        return self.assemble_forcing(self.sample_forcing(f, slab, points))

    # ---------------------------------------------------------------- instrumentation
    def set_profiling(self, level: int):
        check("stmg_set_profiling", self._lib.stmg_set_profiling(self._h, level))

    def profile(self, reset: bool = False):
        ms = (C.c_double * _lib.PROF_N)()
        n = (C.c_longlong * _lib.PROF_N)()
        check("stmg_get_profile", self._lib.stmg_get_profile(self._h, ms, n, int(reset)))
        names = ["smoother", "mg_other", "operator", "other", "fine_sweep"]
        return {nm: {"ms": ms[i], "launches": n[i]} for i, nm in enumerate(names)}

    def device_status(self):
        """Synchronise; raise StmgError if a bounded device-side wait expired."""
        check("stmg_device_status", self._lib.stmg_device_status(self._h))

    def inject_wait_fault(self):
        """Testing hook: the next solve's grid barrier cannot complete and times out."""
        check("stmg_inject_wait_fault", self._lib.stmg_inject_wait_fault(self._h))

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.stmg_kernel_launches(self._h))

    def sweep_bytes(self, lvl: int = 0, prec="fp32") -> float:
        b = C.c_double()
        check("stmg_sweep_bytes", self._lib.stmg_sweep_bytes(self._h, lvl, _PREC[prec], C.byref(b)))
        return b.value


# -------------------------------------------------------------------- host introspection
def host_default_hierarchy(n: int, r: int, k: int, coarse_n: int = 1, k_min: int = 1):
    lib = load()
    buf = (C.c_int * (3 * _lib.MAX_LEVELS))()
    cnt = C.c_int()
    check("stmg_host_default_hierarchy", lib.stmg_host_default_hierarchy(n, r, k, coarse_n, k_min, buf,
                                                                                   C.byref(cnt)))
    return [tuple(buf[3 * i:3 * i + 3]) for i in range(cnt.value)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def host_tables_1d(r: int):
    lib = load()
    np1 = r + 2
    xi, M1, K1 = np.zeros(np1), np.zeros(np1 * np1), np.zeros(np1 * np1)
    G1, N1 = np.zeros((r + 1) * np1), np.zeros((r + 1) * np1)
    check("stmg_host_tables_1d", lib.stmg_host_tables_1d(r, _dp(xi), _dp(M1), _dp(K1), _dp(G1), _dp(N1)))
    return {"xi": xi, "M1": M1.reshape(np1, np1), "K1": K1.reshape(np1, np1),
            "G1": G1.reshape(r + 1, np1), "N1": N1.reshape(r + 1, np1)}


def host_time_tables(k: int, tau: float):
    lib = load()
    kt = k + 1
    nodes, w, K, M, phi = np.zeros(kt), np.zeros(kt), np.zeros(kt * kt), np.zeros(kt), np.zeros(kt)
    check("stmg_host_time_tables", lib.stmg_host_time_tables(k, tau, _dp(nodes), _dp(w), _dp(K), _dp(M), _dp(phi)))
    return {"nodes": nodes, "weights": w, "K": K.reshape(kt, kt), "M": M, "phi_left": phi}


def host_patch(dim, n, r, k, nu, tau, kind, patch, with_inverse=True):
    lib = load()
    B, npat, ncls = C.c_int(), C.c_longlong(), C.c_int()
    check("stmg_host_patch", lib.stmg_host_patch(dim, n, r, k, nu, tau, kind, 0, None, None, C.byref(B),
                                                 C.byref(npat), C.byref(ncls)))
    dofs = np.zeros(B.value, dtype=np.int32)
    inv = np.zeros((B.value, B.value)) if with_inverse else None
    check("stmg_host_patch", lib.stmg_host_patch(dim, n, r, k, nu, tau, kind, patch,
                                                 dofs.ctypes.data_as(C.POINTER(C.c_int)),
                                                 _dp(inv) if with_inverse else None, C.byref(B),
                                                 C.byref(npat), C.byref(ncls)))
    return {"dofs": dofs, "inverse": inv, "B": B.value, "n_patches": npat.value, "n_classes": ncls.value}


def host_valence(dim, n, r, k, kind):
    lib = load()
    size = C.c_longlong()
    check("stmg_host_valence", lib.stmg_host_valence(dim, n, r, k, kind, None, C.byref(size)))
    v = np.zeros(size.value, dtype=np.int32)
    check("stmg_host_valence", lib.stmg_host_valence(dim, n, r, k, kind, v.ctypes.data_as(C.POINTER(C.c_int)),
                                                     C.byref(size)))
    return v


def host_coarse_inverse(dim, n, r, k, nu, tau):
    lib = load()
    D = C.c_longlong()
    check("stmg_host_coarse_inverse", lib.stmg_host_coarse_inverse(dim, n, r, k, nu, tau, None, C.byref(D)))
    G = np.zeros(D.value * D.value)
    check("stmg_host_coarse_inverse", lib.stmg_host_coarse_inverse(dim, n, r, k, nu, tau, _dp(G), C.byref(D)))
    return G.reshape(D.value, D.value).T.copy()     # column-major -> row-major


def host_invert(A, threads=0):
    """Inverse of the square FP64 matrix A by the library's setup routine (host only)."""
    lib = load()
    M = np.ascontiguousarray(A, dtype=np.float64).copy()
    n = M.shape[0]
    if M.ndim != 2 or M.shape[1] != n:
        raise ValueError("host_invert: A must be square")
    check("stmg_host_invert", lib.stmg_host_invert(_dp(M), n, threads))
    return M
