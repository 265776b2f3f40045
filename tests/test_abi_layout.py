"""The ctypes mirror of the C ABI's structs (paper_2502_09159_gb300/_lib.py) against
include/stmg.h itself: a small C program compiled with gcc prints every field's offset
and each struct's size, and the defaults that stmg_default_config writes are read back
through the mirror (CPU only: stmg_default_config is host code)."""
import ctypes
import json
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "stmg_config": ["dim", "n_cells", "r", "k", "nu", "T", "n_slabs", "n_levels", "level_n", "level_r", "level_k",
                    "smoother", "omega", "nu1", "nu2", "precond_precision", "precisions", "gmres_max_iter",
                    "rel_tol", "use_graphs", "sweep_variant", "autotune", "coarse_n", "k_min", "n_sub",
                    "half_inverses", "transfer_variant", "apply_variant", "persistent", "level_nsub",
                    "time_h", "arnoldi_form", "fuse_transfers"],
    "stmg_level_info_t": ["n", "r", "k", "n_sub", "size", "n_vel", "n_pres", "smoother", "patch_size", "n_patches",
                          "n_patch_classes", "inverse_bytes", "sweep_variant", "patches_per_block",
                          "apply_cells_per_block", "transfer_cells_per_block", "streaming", "apply_variant",
                          "apply_tile", "persistent", "sweep_unroll"],
    "stmg_solve_info": ["iterations", "rel_residual", "status", "seconds"],
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    d = tmp_path_factory.mktemp("abi")
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "stmg.h"', "int main(void) {", 'printf("{");']
    first = True
    for s, fields in STRUCTS.items():
        sep = "" if first else ","
        first = False
        src.append(f'printf("{sep}\\"{s}\\": {{\\"sizeof\\": %zu", sizeof({s}));')
        for f in fields:
            src.append(f'printf(", \\"{f}\\": %zu", offsetof({s}, {f}));')
        src.append('printf("}");')
    src += ['printf("}\\n");', "return 0;", "}"]
    c_file, exe = d / "layout.c", d / "layout"
    c_file.write_text("\n".join(src) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(c_file), "-o", str(exe)],
                   check=True, capture_output=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


def _mirror(name):
    from paper_2502_09159_gb300 import _lib
    return {"stmg_config": _lib.Config, "stmg_level_info_t": _lib.LevelInfo, "stmg_solve_info": _lib.SolveInfo}[name]


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_ctypes_mirror_matches_the_header(c_layout, name):
    cls = _mirror(name)
    assert [f[0] for f in cls._fields_] == STRUCTS[name]       # same fields, same order
    assert ctypes.sizeof(cls) == c_layout[name]["sizeof"]
    for f in STRUCTS[name]:
        assert getattr(cls, f).offset == c_layout[name][f], f


def test_default_config_read_through_the_mirror():
    import paper_2502_09159_gb300 as pkg
    from paper_2502_09159_gb300 import _lib
    pkg.build()
    lib = _lib.load()
    cfg = _lib.Config()
    ctypes.memset(ctypes.byref(cfg), 0x55, ctypes.sizeof(cfg))
    assert lib.stmg_default_config(ctypes.byref(cfg)) == _lib.OK
    assert (cfg.dim, cfg.n_cells, cfg.r, cfg.k, cfg.n_slabs) == (2, 8, 1, 1, 4)
    assert (cfg.nu, cfg.T, cfg.omega, cfg.rel_tol) == (1.0, 1.0, 0.7, 1e-8)
    assert (cfg.nu1, cfg.nu2, cfg.gmres_max_iter, cfg.precisions) == (1, 1, 200, 3)
    assert (cfg.use_graphs, cfg.sweep_variant, cfg.autotune, cfg.coarse_n, cfg.k_min) == (1, 0, 1, 1, 1)
    assert (cfg.n_sub, cfg.half_inverses, cfg.transfer_variant, cfg.n_levels) == (1, 0, 0, 0)
    assert cfg.apply_variant == 0 and cfg.persistent == 1 and cfg.time_h == 0 and cfg.arnoldi_form == 0 and cfg.fuse_transfers == 1
    assert list(cfg.level_nsub) == [0] * len(cfg.level_nsub)
    assert list(cfg.smoother) == [_lib.CELL] * len(cfg.smoother)
