"""Time one hot-path kernel of libstmg in isolation on a chosen configuration.

    python -m paper_2502_09159_gb300.kernel_bench --kernel sweep --prec fp32 \
        --dim 2 --n 64 --r 2 --k 2 --level 0 --reps 20

Kernels: apply, residual, sweep, smooth (residual + sweep), restrict, prolong, vcycle.
`--grid` runs the (dim, r, k) x precision throughput table of the 2D 256^2 / 3D 16^3 meshes.
Prints one JSON line with the mean time per call (CUDA events after warm-up), dofs/s,
and for the sweep its algorithmic bytes and GB/s.  Used for profiler captures and by the
launch-parameter tuner.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import SpaceTimeMG


def run(kernel="sweep", prec="fp32", dim=2, n=64, r=2, k=2, level=0, reps=20, warmup=3, smoother=0,
        mg: SpaceTimeMG | None = None, variant=0, autotune=True, coarse_n=1, k_min=1, profile_range=False,
        graphs=False):
    dtype = torch.float64 if prec == "fp64" else torch.float32
    own = mg is None
    if own:
        mg = SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, precisions=(prec,), precond_precision=prec,
                         smoothers=[smoother] * 24, sweep_variant=variant, autotune=autotune,
                         coarse_n=coarse_n, k_min=k_min, use_graphs=graphs)
    D = mg.size(level)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(D, generator=g, device="cuda", dtype=dtype)
    b = torch.rand(D, generator=g, device="cuda", dtype=dtype)
    y = torch.empty_like(x)
    if kernel in ("restrict", "prolong"):
        xc = torch.rand(mg.size(level + 1), generator=g, device="cuda", dtype=dtype)
    fns = {
        "apply": lambda: mg.apply(x, level, out=y),
        "residual": lambda: mg.residual(b, x, level, out=y),
        "sweep": lambda: mg.vanka_sweep(b, y, level),
        "smooth": lambda: mg.smooth(b, y, level),
        "restrict": lambda: mg.restrict(x, level, out=xc),
        "prolong": lambda: mg.prolongate_add(xc, y, level),
        "vcycle": lambda: mg.vcycle(b.double(), prec, out=y.double() if dtype != torch.float64 else y),
    }
    if kernel == "vcycle":
        b64, y64 = b.double(), torch.empty(D, dtype=torch.float64, device="cuda")
        fns["vcycle"] = lambda: mg.vcycle(b64, prec, out=y64)
    y.zero_()
    fn = fns[kernel]
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if profile_range:                       # limits an `ncu --profile-from-start off` capture
        torch.cuda.profiler.start()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    if profile_range:
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / reps
    out = {"kernel": kernel, "prec": prec, "variant": variant, "dim": dim, "n": mg.levels[level]["n"], "r": mg.levels[level]["r"],
           "k": mg.levels[level]["k"], "level": level, "dofs": D, "ms": ms, "dofs_per_s": D / (ms / 1e3)}
    if kernel == "sweep":
        sb = mg.sweep_bytes(level, prec)
        out.update({"bytes": sb, "GBs": sb / (ms / 1e3) / 1e9})
    if own:
        mg.close()
    return out


def table(prec="fp32", dim=2, n=64, r=2, k=2, coarse_n=8, k_min=2, reps=50):
    """Mean time of every V-cycle kernel on every level of one tuned handle (CUDA events)."""
    mg = SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, precisions=(prec,), precond_precision=prec,
                     coarse_n=coarse_n, k_min=k_min, use_graphs=False)
    rows = []
    last = len(mg.levels) - 1
    for l in range(len(mg.levels)):
        kernels = ["residual"] + (["sweep", "restrict", "prolong"] if l < last else [])
        for kname in kernels:
            o = run(kname, prec, level=l, reps=reps, mg=mg)
            rows.append({"level": l, "n": o["n"], "r": o["r"], "k": o["k"], "kernel": kname,
                         "us": round(o["ms"] * 1e3, 2), **({"GBs": round(o["GBs"])} if "GBs" in o else {})})
    o = run("vcycle", prec, level=0, reps=reps, mg=mg)
    rows.append({"level": 0, "kernel": "vcycle (graph)", "us": round(o["ms"] * 1e3, 2)})
    mg.close()
    return rows


def _hbm_peak():
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def grid(dims=(2, 3), rs=(1, 2, 3, 4), ks=(0, 1, 2, 3), reps=10, mem_limit_gb=200.0, out=None):
    """Apply, sweep and V-cycle throughput per (dim, r, k) and precision on the 2D 256^2 and
    3D 16^3 meshes (random inputs; cost is data-independent).  One handle per point holds both
    precisions when their inverses fit `mem_limit_gb` together, else one handle per precision
    that fits alone; a precision that fits in neither way is reported as not fitting.  Launch shapes are autotuned and the V-cycle runs as a graph."""
    import time
    peak, peak_kind = _hbm_peak()
    rows = []
    for dim in dims:
        n = 256 if dim == 2 else 16
        for r in rs:
            for k in ks:
                from math import comb
                B = (k + 1) * (dim * (r + 2) ** dim + comb(r + dim, dim))
                inv64 = n ** dim * B * B * 8 * 1.15 / 1e9
                if 1.5 * inv64 <= mem_limit_gb:
                    handles = [("fp64", "fp32")]
                else:
                    handles = [(p,) for p, gb in (("fp64", inv64), ("fp32", 0.5 * inv64)) if gb <= mem_limit_gb]
                base = {"dim": dim, "n": n, "r": r, "k": k, "B": B}
                done = set()
                for precs in handles:
                    t0 = time.time()
                    mg = SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, precisions=precs, precond_precision=precs[-1],
                                     use_graphs=True)
                    setup = time.time() - t0
                    for prec in precs:
                        a = run("apply", prec, level=0, reps=reps, mg=mg)
                        s = run("sweep", prec, level=0, reps=reps, mg=mg)
                        v = run("vcycle", prec, level=0, reps=reps, mg=mg)
                        lv = mg.levels[0]
                        pi = 0 if prec == "fp64" else 1
                        row = {**base, "prec": prec, "D": a["dofs"], "levels": len(mg.levels),
                               "setup_s": round(setup, 1),
                               "apply_Gdofs": round(a["dofs_per_s"] / 1e9, 3),
                               "sweep_Gdofs": round(s["dofs_per_s"] / 1e9, 3),
                               "sweep_GBs": round(s["GBs"], 1), "sweep_frac": round(s["GBs"] / peak, 3),
                               "vcycle_Gdofs": round(v["dofs_per_s"] / 1e9, 3),
                               "apply_us": round(a["ms"] * 1e3, 1), "sweep_us": round(s["ms"] * 1e3, 1),
                               "vcycle_us": round(v["ms"] * 1e3, 1),
                               "sweep_variant": lv["sweep_variant"][pi],
                               "patches_per_block": lv["patches_per_block"][pi],
                               "apply_cells_per_block": lv["apply_cells_per_block"][pi],
                               "peak_GBs": peak, "peak_kind": peak_kind}
                        rows.append(row)
                        done.add(prec)
                        if out:
                            print(json.dumps(row), file=out, flush=True)
                    mg.close()
                    del mg
                    import torch
                    torch.cuda.empty_cache()
                for prec in ("fp64", "fp32"):
                    if prec not in done:
                        row = {**base, "prec": prec, "status": "does not fit",
                               "inverse_GB": round(inv64 * (1 if prec == "fp64" else 0.5), 1)}
                        rows.append(row)
                        if out:
                            print(json.dumps(row), file=out, flush=True)
    return rows


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--kernel", default="sweep")
    p.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--dim", type=int, default=2)
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--r", type=int, default=2)
    p.add_argument("--k", type=int, default=2)
    p.add_argument("--level", type=int, default=0)
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--vsp", action="store_true")
    p.add_argument("--variant", type=int, default=0, help="sweep kernel: 0 tuned, 1 block per patches, 2 TMA")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--coarse-n", type=int, default=1)
    p.add_argument("--k-min", type=int, default=1)
    p.add_argument("--table", action="store_true", help="every V-cycle kernel on every level")
    p.add_argument("--profile-range", action="store_true", help="wrap the timed calls in cudaProfilerStart/Stop")
    p.add_argument("--graphs", action="store_true", help="capture the V-cycle in a CUDA graph")
    p.add_argument("--grid", action="store_true",
                   help="apply/sweep/V-cycle over dim in {2,3} (256^2, 16^3), r in 1..4, k in 0..3")
    p.add_argument("--grid-dims", default="2,3")
    p.add_argument("--out", default=None, help="also write the grid rows (JSON lines) to this file")
    a = p.parse_args()
    if a.grid:
        import sys
        f = open(a.out, "w") if a.out else None
        grid(tuple(int(d) for d in a.grid_dims.split(",")), reps=a.reps, out=f or sys.stdout)
        return
    if a.table:
        for row in table(a.prec, a.dim, a.n, a.r, a.k, a.coarse_n, a.k_min, a.reps):
            print(json.dumps(row))
        return
    print(json.dumps(run(a.kernel, a.prec, a.dim, a.n, a.r, a.k, a.level, a.reps, a.warmup, int(a.vsp),
                         variant=a.variant, autotune=not a.no_autotune, coarse_n=a.coarse_n, k_min=a.k_min,
                         profile_range=a.profile_range, graphs=a.graphs)))


if __name__ == "__main__":
    main()
