"""stmg_smooth_noalloc, the smoothing step for callers that must not have device memory
allocated for them while they run, checked through the C ABI against stmg_smooth.

Collected last on purpose (file name), so that a run stopping at the first failure has
already run every other test.  Works alone in a fresh process and after the others.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2502_09159_gb300 as stmg  # noqa: E402
from paper_2502_09159_gb300 import _lib  # noqa: E402
from workloads import random_vector  # noqa: E402

stmg.build()
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}     # the smoothing-step tolerances of the parity tests


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_smooth_noalloc_matches_smooth_twice(dtype):
    g = stmg.SpaceTimeMG(dim=2, n_cells=16, r=2, k=2, nu=1.0, T=1.0, n_slabs=16, use_graphs=False)
    lib = _lib.load()
    prec = stmg.FP64 if dtype == torch.float64 else stmg.FP32
    for lvl in (0, 1):
        D = g.size(lvl)
        b = torch.from_numpy(random_vector(D, 5 + lvl)).to("cuda", dtype)
        x0 = torch.from_numpy(random_vector(D, 9 + lvl)).to("cuda", dtype)
        ref = x0.clone()
        g._stream()
        assert lib.stmg_smooth(g._h, lvl, prec, C.c_void_p(b.data_ptr()), C.c_void_p(ref.data_ptr()), 2) == 0
        for _ in range(2):                                   # two calls in a row share the scratch
            x = x0.clone()
            st = lib.stmg_smooth_noalloc(g._h, lvl, prec, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), 2)
            assert st == 0, lib.stmg_status_string(st)
            torch.cuda.synchronize()
            err = ((x - ref).abs().max() / ref.abs().max()).item()
            assert err < TOL[dtype], err
    g.device_status()                                        # no bounded device-side wait expired
    g.close()


def test_smooth_noalloc_rejects_levels_beyond_its_scratch():
    # 2D 128x128, Q3/P2, DG(2): 1,184,262 dofs > 2^20 on the finest level; the next level fits
    g = stmg.SpaceTimeMG(dim=2, n_cells=128, r=2, k=2, precisions=("fp32",), precond_precision="fp32",
                         use_graphs=False)
    lib = _lib.load()
    assert g.size(0) > _lib.NOALLOC_MAX_ENTRIES >= g.size(1)
    b = torch.zeros(g.size(0), dtype=torch.float32, device="cuda")
    x = torch.zeros_like(b)
    st = lib.stmg_smooth_noalloc(g._h, 0, stmg.FP32, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), 1)
    assert st == _lib.ERR_TOO_LARGE
    assert b"scratch" in lib.stmg_status_string(st)
    b1 = torch.from_numpy(random_vector(g.size(1), 3)).to("cuda", torch.float32)
    x1, ref = torch.zeros_like(b1), torch.zeros_like(b1)
    assert lib.stmg_smooth_noalloc(g._h, 1, stmg.FP32, C.c_void_p(b1.data_ptr()), C.c_void_p(x1.data_ptr()), 1) == 0
    g.smooth(b1, ref, 1, steps=1)
    torch.cuda.synchronize()
    assert ((x1 - ref).abs().max() / ref.abs().max()).item() < 1e-5
    g.device_status()
    g.close()
