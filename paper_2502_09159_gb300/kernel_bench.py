"""Time one hot-path kernel of libstmg in isolation on a chosen configuration.

    python -m paper_2502_09159_gb300.kernel_bench --kernel sweep --prec fp32 \
        --dim 2 --n 64 --r 2 --k 2 --level 0 --reps 20

Kernels: apply, residual, sweep, smooth (residual + sweep), restrict, prolong, vcycle.
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
    a = p.parse_args()
    if a.table:
        for row in table(a.prec, a.dim, a.n, a.r, a.k, a.coarse_n, a.k_min, a.reps):
            print(json.dumps(row))
        return
    print(json.dumps(run(a.kernel, a.prec, a.dim, a.n, a.r, a.k, a.level, a.reps, a.warmup, int(a.vsp),
                         variant=a.variant, autotune=not a.no_autotune, coarse_n=a.coarse_n, k_min=a.k_min,
                         profile_range=a.profile_range, graphs=a.graphs)))


if __name__ == "__main__":
    main()
