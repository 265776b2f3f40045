"""ctypes declarations of libstmg (include/stmg.h, include/stmg_net.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

MAX_LEVELS = 24
OK, ERR_ARG, ERR_OOM, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_NONFINITE, ERR_CUDA, \
    ERR_UNIMPLEMENTED, ERR_SINGULAR, ERR_TOO_LARGE, ERR_TIMEOUT = range(11)
NOALLOC_MAX_ENTRIES = 1 << 20
FP64, FP32 = 0, 1
CELL, VSP = 0, 1
MARCH_FORCING, MARCH_BOUNDARY = 0, 1
PROF_SMOOTHER, PROF_MG_OTHER, PROF_OPERATOR, PROF_OTHER, PROF_FINE_SWEEP, PROF_N = range(6)


class Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_cells", C.c_int), ("r", C.c_int), ("k", C.c_int),
                ("nu", C.c_double), ("T", C.c_double), ("n_slabs", C.c_int),
                ("n_levels", C.c_int),
                ("level_n", C.c_int * MAX_LEVELS), ("level_r", C.c_int * MAX_LEVELS),
                ("level_k", C.c_int * MAX_LEVELS), ("smoother", C.c_int * MAX_LEVELS),
                ("omega", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
                ("precond_precision", C.c_int), ("precisions", C.c_int),
                ("gmres_max_iter", C.c_int), ("rel_tol", C.c_double), ("use_graphs", C.c_int),
                ("sweep_variant", C.c_int), ("autotune", C.c_int), ("coarse_n", C.c_int),
                ("k_min", C.c_int), ("n_sub", C.c_int), ("half_inverses", C.c_int),
                ("transfer_variant", C.c_int), ("apply_variant", C.c_int), ("persistent", C.c_int),
                ("level_nsub", C.c_int * MAX_LEVELS), ("time_h", C.c_int), ("arnoldi_form", C.c_int), ("fuse_transfers", C.c_int)]


class LevelInfo(C.Structure):
    _fields_ = [("n", C.c_int), ("r", C.c_int), ("k", C.c_int), ("n_sub", C.c_int),
                ("size", C.c_longlong), ("n_vel", C.c_longlong), ("n_pres", C.c_longlong),
                ("smoother", C.c_int), ("patch_size", C.c_int), ("n_patches", C.c_longlong),
                ("n_patch_classes", C.c_int), ("inverse_bytes", C.c_longlong * 2),
                ("sweep_variant", C.c_int * 2), ("patches_per_block", C.c_int * 2),
                ("apply_cells_per_block", C.c_int * 2), ("transfer_cells_per_block", C.c_int * 2),
                ("streaming", C.c_int), ("apply_variant", C.c_int * 2), ("apply_tile", (C.c_int * 2) * 2),
                ("persistent", C.c_int * 2), ("sweep_unroll", C.c_int * 2)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("status", C.c_int),
                ("seconds", C.c_double)]


_VP, _I, _D, _LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
_SIGS = {
    "stmg_default_config": (_I, [C.POINTER(Config)]),
    "stmg_create": (_I, [C.POINTER(Config), C.POINTER(_VP)]),
    "stmg_destroy": (None, [_VP]),
    "stmg_set_stream": (_I, [_VP, _VP]),
    "stmg_num_levels": (_I, [_VP, C.POINTER(_I)]),
    "stmg_level_info": (_I, [_VP, _I, C.POINTER(LevelInfo)]),
    "stmg_apply": (_I, [_VP, _I, _I, _VP, _VP]),
    "stmg_residual": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "stmg_apply_transpose": (_I, [_VP, _I, _I, _VP, _VP]),
    "stmg_smooth": (_I, [_VP, _I, _I, _VP, _VP, _I]),
    "stmg_smooth_noalloc": (_I, [_VP, _I, _I, _VP, _VP, _I]),
    "stmg_vanka_sweep": (_I, [_VP, _I, _I, _VP, _VP]),
    "stmg_restrict": (_I, [_VP, _I, _I, _VP, _VP]),
    "stmg_prolongate_add": (_I, [_VP, _I, _I, _VP, _VP]),
    "stmg_coarse_solve": (_I, [_VP, _I, _VP, _VP]),
    "stmg_vcycle": (_I, [_VP, _I, _VP, _VP]),
    "stmg_slab_rhs": (_I, [_VP, _VP, _VP, _VP]),
    "stmg_dirichlet_lift": (_I, [_VP, _VP, _VP, _VP]),
    "stmg_solve_slab": (_I, [_VP, _VP, _VP, C.POINTER(SolveInfo)]),
    "stmg_solve_slab_host": (_I, [_VP, _VP, _VP, C.POINTER(SolveInfo)]),
    "stmg_march_host": (_I, [_VP, _I, _I, _VP, _VP, C.POINTER(SolveInfo)]),
    "stmg_forcing_npoints": (_I, [_VP, C.POINTER(_I)]),
    "stmg_forcing_points": (_I, [_VP, _VP]),
    "stmg_slab_times": (_I, [_VP, _I, C.POINTER(_D)]),
    "stmg_assemble_forcing": (_I, [_VP, _VP, _VP]),
    "stmg_set_profiling": (_I, [_VP, _I]),
    "stmg_get_profile": (_I, [_VP, C.POINTER(_D), C.POINTER(_LL), _I]),
    "stmg_kernel_launches": (_LL, [_VP]),
    "stmg_inject_wait_fault": (_I, [_VP]),
    "stmg_device_status": (_I, [_VP]),
    "stmg_autotune": (_I, [_VP]),
    "stmg_sweep_bytes": (_I, [_VP, _I, _I, C.POINTER(_D)]),
    "stmg_status_string": (C.c_char_p, [_I]),
    "stmg_cells_channels": (_I, [_VP, _I, C.POINTER(_I)]),
    "stmg_cells_gather": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "stmg_cells_scatter_add": (_I, [_VP, _I, _VP, _VP, _VP]),
    "stmg_cells_gather_strided": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _LL, _I]),
    "stmg_cells_gather_adjoint": (_I, [_VP, _I, _VP, _VP, _VP]),
    "stmg_dot": (_I, [_VP, _LL, _VP, _VP, _VP]),
    "stmg_extrapolate": (_I, [_VP, _I, _VP, _VP]),
    "stmg_remove_pressure_mean": (_I, [_VP, _I, _VP]),
    "stmg_net_create": (_I, [_I, _I, _I, _I, _I, _I, _I, _I, C.c_ulonglong, C.POINTER(_VP)]),
    "stmg_net_destroy": (None, [_VP]),
    "stmg_net_set_stream": (_I, [_VP, _VP]),
    "stmg_net_num_params": (_I, [_VP, C.POINTER(_LL)]),
    "stmg_net_set_params": (_I, [_VP, _VP]),
    "stmg_net_get_params": (_I, [_VP, _VP]),
    "stmg_net_get_grads": (_I, [_VP, _VP]),
    "stmg_net_forward": (_I, [_VP, _I, _VP, _VP, _VP]),
    "stmg_net_backward": (_I, [_VP, _I, _VP, _VP, _VP]),
    "stmg_net_mse": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP]),
    "stmg_net_adam": (_I, [_VP, C.c_float, C.c_float, C.c_float, C.c_float, _I]),
    "stmg_net_train_step": (_I, [_VP, _I, _VP, _VP, _VP, C.c_float, C.c_float, C.c_float, C.c_float, _I,
                                 _VP]),
    "stmg_channel_rms": (_I, [_LL, _I, _VP, _VP, _VP, _VP]),
    "stmg_tensor_rms": (_I, [_LL, _VP, _VP, _VP, _VP]),
    "stmg_scale_channels": (_I, [_LL, _I, _VP, _VP, _VP]),
    "stmg_host_default_hierarchy": (_I, [_I, _I, _I, _I, _I, C.POINTER(_I), C.POINTER(_I)]),
    "stmg_host_tables_1d": (_I, [_I] + [C.POINTER(_D)] * 5),
    "stmg_host_time_tables": (_I, [_I, _D] + [C.POINTER(_D)] * 5),
    "stmg_host_patch": (_I, [_I, _I, _I, _I, _D, _D, _I, _LL, C.POINTER(_I), C.POINTER(_D),
                             C.POINTER(_I), C.POINTER(_LL), C.POINTER(_I)]),
    "stmg_host_valence": (_I, [_I, _I, _I, _I, _I, C.POINTER(_I), C.POINTER(_LL)]),
    "stmg_host_coarse_inverse": (_I, [_I, _I, _I, _I, _D, _D, C.POINTER(_D), C.POINTER(_LL)]),
    "stmg_host_invert": (_I, [C.POINTER(_D), _I, _I]),
}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstmg.so")
_lib = None


class StmgError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        msg = load().stmg_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{fn} failed: {msg} ({status})")


def load():
    """Load libstmg.so from the package directory; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libstmg.so is missing ({LIB_PATH}): build it with "
                           "`python -m paper_2502_09159_gb300.builder` (there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(fn, status):
    if status != OK:
        raise StmgError(fn, status)
    return status
