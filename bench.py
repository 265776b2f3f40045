"""Benchmark: space-time dofs/s of the hp space-time multigrid solve on one GB300.

Workload (default, the 2D configuration the headline metric is quoted on): unit square
x [0,1], 64x64 cells, Q3/P2disc (r=2) in space, DG(2) in time, 16 slabs, nu = 1,
forcing = seeded random Fourier modes (8 modes per potential, c ~ N(0,1), a,b ~ U{1..4},
theta ~ U[0,2pi), numpy PCG64 seeds 1 and 2), hp hierarchy 64^2 Q3 -> 64^2 Q2 -> 32^2 ->
16^2 -> 8^2 (direct solve) with DG(2) on every level (Alg. 2/3 with h_0 = 1/8; the Table
2(b) hierarchy and the r:2->1, k:2->0 hierarchy are reported beside it), cell Vanka with
omega = 0.7, FGMRES to ||b - S x|| <= 1e-8 ||b||.
One step = one time march over all 16 slabs (slab right-hand side with the coupling to
the previous slab, FGMRES + one V-cycle per iteration).  value = 16 * D / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --only-kernel sweep|residual|apply|vcycle|restrict|prolong|cgs2 [--level L] [--prec fp32]
        (one kernel of the headline handle in a loop inside cudaProfilerStart/Stop, for ncu)

The headline runs the V-cycle in FP32 (FGMRES, true residual and coarse solve in FP64);
the timed march carries no instrumentation.  A second, instrumented march times the
dominant kernel (the finest-level Vanka sweep) for the roofline.  Reported beside it: the
end-to-end march through the host-buffer C call, the FP64-preconditioner solve, the
apply / sweep / V-cycle rates, the error of slab 1 against the FP64 oracle, a subset of
the (dim, r, k) throughput grid, and the one-time setup.  --impl reference times the FP64
CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c2": (dict(dim=2, n_cells=64, r=2, k=2, nu=1.0, T=1.0, n_slabs=16),
           "2D 64x64 Q3/P2disc DG(2), 16 slabs, Fourier forcing (seeds 1,2), cell Vanka", "fourier"),
    "c3": (dict(dim=3, n_cells=32, r=2, k=1, nu=1e-2, T=1.0, n_slabs=8),
           "3D 32^3 Q3/P2disc DG(1), 8 slabs, Taylor-Green-like field, nu = 1e-2, cell Vanka", "taylor_green"),
    "lid": (dict(dim=3, n_cells=16, r=2, k=2, nu=1.0, T=8.0, n_slabs=256),
            "3D lid-driven cavity (Sec. 5.2, c = 4): 16^3 Q3/P2disc DG(2), 256 slabs on [0, 8], lid velocity "
            "sin(pi t / 4) in x on z = 1, no-slip walls, nu = 1, cell Vanka, n_sm = 1", "lid"),
    "lid5": (dict(dim=3, n_cells=32, r=2, k=2, nu=1.0, T=8.0, n_slabs=512),
             "3D lid-driven cavity (Sec. 5.2, c = 5): 32^3 Q3/P2disc DG(2), 512 slabs on [0, 8], lid velocity "
             "sin(pi t / 4) in x on z = 1, no-slip walls, nu = 1, cell Vanka, n_sm = 1", "lid"),
    "lid_r3": (dict(dim=3, n_cells=16, r=3, k=3, nu=1.0, T=8.0, n_slabs=256),
               "3D lid-driven cavity (Sec. 5.2, c = 4, r = 3): 16^3 Q4/P3disc DG(3), 256 slabs on [0, 8], lid "
               "velocity sin(pi t / 4) in x on z = 1, no-slip walls, nu = 1, cell Vanka, n_sm = 1", "lid"),
}
WORKLOADS_KIND = {name: kind for _, name, kind in WORKLOADS.values()}
# the paper's throughput on the same workloads (Table 3, n_sm = 1; 13,824 CPU ranks)
PAPER_THETA = {"lid": 302520576 / 149.4, "lid5": 4708913664 / 329.0, "lid_r3": 927534080 / 629.4}
WORKLOAD, WORKLOAD_NAME, _ = WORKLOADS["c2"]
METRIC = "space-time DoFs/s (apply, Vanka sweep, V-cycle); time-to-1e-8 mixed vs FP64"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-micro", action="store_true", help="skip the per-kernel rate measurements")
    p.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline (profiler runs)")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    p.add_argument("--coarse-n", type=int, default=0,
                   help="coarsest mesh of the hierarchy (Alg. 2's 1/h_0); 0: 8 in 2D, 1 in 3D")
    p.add_argument("--k-min", type=int, default=0, help="lowest temporal degree of the hierarchy; 0: k in 2D, 1 in 3D")
    p.add_argument("--levels", default="", help="explicit level list n:r:k,... fine -> coarse")
    p.add_argument("--half-inverses", action="store_true",
                   help="store the FP32 V-cycle's patch inverses in FP16 with row scales (timed march)")
    p.add_argument("--profile-range", action="store_true",
                   help="wrap the timed steps in cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    p.add_argument("--only-kernel", default="", choices=["", "sweep", "residual", "apply", "vcycle", "restrict",
                                                          "prolong", "cgs2"],
                   help="time one kernel of the headline handle in a loop (for ncu captures)")
    p.add_argument("--level", type=int, default=0, help="level of --only-kernel")
    p.add_argument("--prec", default="fp32", choices=["fp32", "fp64"], help="precision of --only-kernel")
    p.add_argument("--reps", type=int, default=3, help="launches of --only-kernel inside the profiler range")
    p.add_argument("--apply-variant", type=int, default=0, help="force the operator kernel (1 per-cell, 2 node-centred, 3 register, 4 pair-split register)")
    p.add_argument("--sweep-variant", type=int, default=0, help="force the sweep kernel (1 block, 2 TMA, 3 pipelined)")
    p.add_argument("--arnoldi-form", type=int, default=0,
                   help="Arnoldi step: 0 rows of w in registers where they fit (default), 1 split passes")
    p.add_argument("--persistent", type=int, default=1,
                   help="levels below the finest in one persistent kernel: 0 never, 1 tuner (default), 2 always")
    p.add_argument("--workload", default="c2", choices=sorted(WORKLOADS),
                   help="c2: the 2D headline configuration; c3: the 3D 32^3 configuration; "
                        "lid: the lid-driven cavity at c = 4 (lid5: c = 5; lid_r3: c = 4 with Q4/P3 DG(3))")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seeds(rank):
    """Forcing seeds of the problem rank `rank` solves: replicas run independent problems."""
    return 1 + 10 * rank, 2 + 10 * rank


def max_over_ranks(ms, world, device=None):
    """The slowest rank's time (the job's time) via an all-reduce; identity on one rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def aggregate_value(world, slabs, dofs_per_slab, ms_per_step):
    """Whole-job throughput: all ranks' space-time dofs per step over the slowest rank's time."""
    return world * slabs * dofs_per_slab / (ms_per_step / 1e3)


def slab_dofs(w):
    d, n, r, k = w["dim"], w["n_cells"], w["r"], w["k"]
    return (k + 1) * (d * ((r + 1) * n + 1) ** d + math.comb(r + d, d) * n ** d)


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        try:
            import tempfile
            self.path = os.path.join(tempfile.gettempdir(), f"stmg_clocks_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as f:
            return summarise_clocks(f)


def summarise_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in the rows of
    `nvidia-smi --query-gpu=<Clocks.Q> --format=csv,noheader,nounits` (index, clocks.sm,
    clocks.max.sm, power.draw, the reasons mask, then hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap as "Active" / "Not Active"); None without rows."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source(src, name):
    """Text of the __global__ definition of `name` (with its template line) up to its closing
    brace at column 0, or None."""
    lines = src.splitlines(keepends=True)
    for i, l in enumerate(lines):
        if "__global__" in l and f"{name}(" in l:
            start = i - 1 if i > 0 and lines[i - 1].startswith("template") else i
            j = i
            while j < len(lines) and not lines[j].startswith("}"):
                j += 1
            return "".join(lines[start:j + 1])
    return None


def ncu_traffic(kernel_file, kernel_name, key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    when the kernel's definition changed since the capture (the hash covers the kernel's
    own source text, so unrelated code added to the same file keeps the figure valid)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        with open(os.path.join(ROOT, "paper_2502_09159_gb300", "csrc", kernel_file)) as f:
            text = kernel_source(f.read(), kernel_name)
        if text is None:
            return None
        h = hashlib.sha256(text.encode()).hexdigest()[:16]
        e = tr.get(key)
        if e and e.get("source_sha256_16") == h:
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------- our arm
def sweep_alg_bytes(level, prec):
    """Algorithmic bytes of one Vanka sweep: every patch's B x B inverse once plus about
    three vectors (residual read, iterate read and written), n_patches B^2 s + 3 D s."""
    s = 8 if prec == "fp64" else 4
    return level["n_patches"] * level["patch_size"] ** 2 * s + 3 * level["size"] * s


def run_ours(args):
    import numpy as np
    import torch

    import paper_2502_09159_gb300 as stmg
    from workloads import fourier_forcing_2d, lid_driven_3d, taylor_green_3d
    global WORKLOAD, WORKLOAD_NAME
    WORKLOAD, WORKLOAD_NAME, forcing_kind = WORKLOADS[args.workload]
    if args.coarse_n == 0:
        args.coarse_n = 8 if WORKLOAD["dim"] == 2 else 1
    if args.k_min == 0:
        args.k_min = WORKLOAD["k"] if WORKLOAD["dim"] == 2 else 1

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    stmg.build()
    w = WORKLOAD
    D = slab_dofs(w)
    N = w["n_slabs"]
    # replicas: every rank solves its own problem (different forcing seeds), no data-path collective
    if forcing_kind == "fourier":
        sp, sf = replica_seeds(rank)
        pb = fourier_forcing_2d(nu=w["nu"], seed_psi=sp, seed_phi=sf)
    elif forcing_kind == "lid":
        pb = lid_driven_3d(nu=w["nu"], T=w["T"])
    else:
        pb = taylor_green_3d(nu=w["nu"])
    precisions = ("fp64", "fp32") if w["dim"] == 2 else ("fp32",)

    levels = [tuple(int(v) for v in t.split(":")) for t in args.levels.split(",")] if args.levels else None

    def make(prec, coarse_n=args.coarse_n, k_min=args.k_min, half=args.half_inverses, lv=levels, max_iter=None):
        return stmg.SpaceTimeMG(**w, precond_precision=prec, coarse_n=min(coarse_n, w["n_cells"]),
                                k_min=k_min, levels=lv, precisions=precisions if prec == "fp32" else (prec,),
                                gmres_max_iter=max_iter or (200 if w["dim"] == 2 else 80),
                                half_inverses=half and prec == "fp32", apply_variant=args.apply_variant,
                                sweep_variant=args.sweep_variant, persistent=args.persistent,
                                arnoldi_form=args.arnoldi_form)

    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    mg = make("fp32")                       # hierarchy, patch and coarse inverses, launch-shape tuning
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    if args.only_kernel:
        print(json.dumps(only_kernel(mg, args)), flush=True)
        return
    # resident per-slab inputs: the assembled forcing, or for the lid-driven cavity (no
    # forcing) the slab's boundary values
    # the forcing enters the timed march as its samples at the quadrature points of every
    # slab (the synthetic input, resident): the assembly of F_n (Eq. DefFn, the paper's
    # "other" work of a time step) runs inside each step
    if forcing_kind == "lid":
        F0 = mg.zeros()
        F = [mg.boundary_vector(pb.boundary, s) for s in range(N)]
        FQ = None
    else:
        F0 = None
        pts = mg.forcing_points()
        FQ = [mg.sample_forcing(pb.forcing, s, pts) for s in range(N)]
        F = [mg.assemble_forcing(FQ[s]) for s in range(N)]
    x_bufs = [mg.zeros() for _ in range(N)]
    b_buf = mg.empty()
    b_tmp = mg.empty()
    f_buf = mg.empty()

    def build_b(g, s, x_prev):
        if F0 is None:
            g.assemble_forcing(FQ[s], out=f_buf)
            g.slab_rhs(f_buf, x_prev, out=b_buf)
        else:
            g.slab_rhs(F0, x_prev, out=b_tmp)
            g.dirichlet_lift(F[s], b_tmp, out=b_buf)

    def step(g, iters, statuses=None):
        """One march; with `statuses` (a list) a slab that does not converge is recorded
        there instead of raising."""
        x_prev = None
        for s in range(N):
            build_b(g, s, x_prev)
            x_bufs[s].zero_()
            _, info = g.solve_slab(b_buf, out=x_bufs[s])
            if info["status"] != 0:
                if statuses is None:
                    raise RuntimeError(f"slab {s}: {info}")
                statuses.append({"slab": s, **info})
            iters.append(info["iterations"])
            x_prev = x_bufs[s]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    its = []
    for _ in range(args.warmup):
        step(mg, its)
    clocks = Clocks(local)
    its = []
    barrier()
    clocks.start()
    launches_before = mg.kernel_launches
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile_range:
        torch.cuda.profiler.start()
    ev0.record()
    for _ in range(args.steps):
        step(mg, its)
    ev1.record()
    barrier()
    if args.profile_range:
        torch.cuda.profiler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = mg.kernel_launches - launches_before
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, device="cuda")
    ms_step = ms / args.steps
    value = aggregate_value(world, N, D, ms_step)
    x1_fp32 = x_bufs[0].cpu().numpy()        # slab 1 of the timed march (parity against the oracle)
    # the one-time setup next to the march: the paper's theta divides by the total wall
    # time, which may or may not include its (CPU) smoother setup
    setup_ms = max_over_ranks(setup_ms, world, device="cuda")
    setup = {"seconds": round(setup_ms / 1e3, 3), "precisions": list(precisions),
             "value_incl_setup": aggregate_value(world, N, D, ms_step + setup_ms),
             "includes": "handle creation: level geometry, patch inverses (FP64 on the host, "
                         "stored per patch on the device), coarse inverse, launch-shape tuning"}

    # ---- roofline of the dominant kernel (finest-level FP32 Vanka sweep): one more march,
    # untimed, with CUDA events around every finest-level sweep on the stream it runs on
    mg.set_profiling(1)
    mg.profile(reset=True)
    step(mg, [])
    prof = mg.profile(reset=True)
    mg.set_profiling(0)
    lv0 = mg.levels[0]
    sweep_ms = prof["fine_sweep"]["ms"] / max(prof["fine_sweep"]["launches"], 1)
    alg_bytes = sweep_alg_bytes(lv0, "fp32") if not args.half_inverses else mg.sweep_bytes(0, "fp32")
    peaks, peak_kind = measured_peaks()
    achieved = alg_bytes / (sweep_ms / 1e3) / 1e9
    # the sweep kernel the tuner chose for the finest level (FP32)
    sv = lv0["sweep_variant"][1]
    kname = ("k_vanka_sweep_half" if args.half_inverses else
             {1: "k_vanka_sweep", 2: "k_vanka_sweep_tma", 3: "k_vanka_sweep_pipe"}.get(sv, "k_vanka_sweep"))
    traffic_key = ("vanka_sweep_fp32_finest" + ("" if args.workload == "c2" else "_" + args.workload) +
                   ("_half" if args.half_inverses else "") + ("_pipe" if sv == 3 and not args.half_inverses else ""))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "peak_kind": peak_kind,
                "traffic": ncu_traffic("k_vanka.cu", kname, traffic_key),
                "kernel": f"{kname}<float>, finest level, {lv0['patches_per_block'][1]} patches per block, "
                          f"rounds of {lv0['sweep_unroll'][1]} column chunks",
                "bytes_per_launch": alg_bytes,
                "bytes_rule": "n_patches * B^2 * 4 + 3 * D * 4 (stored inverses, residual, iterate)"
                              if not args.half_inverses else "stmg_sweep_bytes (FP16 inverses + row scales)",
                "stored_bytes_per_launch": mg.sweep_bytes(0, "fp32"),
                "avg_launch_ms": round(sweep_ms, 5), "launches_timed": prof["fine_sweep"]["launches"],
                "timed_in": "a separate instrumented march right after the timed region (events around each "
                            "finest-level sweep inside the V-cycle graph)",
                "redundancy": f"{lv0['n_patch_classes']} distinct patch matrices among {lv0['n_patches']} stored "
                              "per-patch inverses (uniform mesh); the stream is the paper's matrix-based smoother's"}

    # ---- end to end through the C ABI: stmg_march_host, host inputs in, host solutions out
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(mg, F, N, D, world, args, barrier, forcing_kind == "lid")

    # ---- per-kernel rates and FP64 vs mixed time-to-1e-8 (not part of the timed step)
    extra = {}
    x1_fp64 = None
    if not args.no_micro and rank == 0:
        extra, x1_fp64 = micro(mg, make, N, D, step, x_bufs)
        extra["time_split"] = guarded(lambda: time_split(mg, step))
        extra["paper_hierarchy"] = guarded(lambda: other_hierarchy(
            make, step, N, D, coarse_n=1, k_min=1,
            what="the Table 2(b) rule: coarsest mesh 1x1, DG(1) on the two coarsest levels"))
        if args.workload == "c2":
            k0 = [(64, 2, 2), (64, 1, 1), (64, 1, 0), (32, 1, 0), (16, 1, 0), (8, 1, 0), (4, 1, 0), (2, 1, 0),
                  (1, 1, 0)]
            extra["k0_hierarchy"] = guarded(lambda: other_hierarchy(
                make, step, N, D, lv=k0, max_iter=600,
                what="r:2->1 with k:2->1, then k:1->0, then geometric to 1x1 with DG(0)"))
            mg.close()
            torch.cuda.empty_cache()
            extra["warm_start"] = guarded(warm_start_bench)
            extra["throughput_grid"] = guarded(throughput_grid)
    line = {"metric": METRIC, "value": value, "unit": "space-time DoFs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (value / PAPER_THETA[args.workload]) if args.workload in PAPER_THETA else None,
            "dtype": "f64 FGMRES + f32 V-cycle", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "dofs_per_slab": D, "slabs_per_step": N,
                       "levels": [(l["n"], l["r"], l["k"]) for l in mg.levels],
                       "precond": "fp32" + (" (FP16 inverses)" if args.half_inverses else ""), "rel_tol": 1e-8,
                       "parallelism": f"replicas x{world}",
                       "hierarchy": f"Alg. 2/3 with h_0 = 1/{args.coarse_n}, lowest temporal degree "
                                    f"{args.k_min}" if not levels else "explicit",
                       "l2_policy": "inputs larger than L2 (finest FP32 patch inverses "
                                    f"{mg.levels[0]['inverse_bytes'][1] / 1e6:.0f} MB > 129 MB)",
                       "mean_gmres_iterations": statistics.mean(its) if its else None,
                       "step": ("per slab: the boundary lift of the slab's Dirichlet data, the coupling to the "
                                "previous slab, the FGMRES solve" if FQ is None else
                                "per slab: the assembly of F_n from the forcing's resident samples at the "
                                "quadrature points, the coupling to the previous slab, the FGMRES solve")},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk, "setup": setup}
    line.update(extra)
    if rank == 0:
        if not args.no_baseline:
            base, x1_oracle = cpu_baseline(coarse_n=args.coarse_n, k_min=args.k_min)
            line["cpu_baseline"] = base
            line["parity"] = parity_against_oracle(x1_oracle, x1_fp32, x1_fp64)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def guarded(fn):
    """A secondary measurement: its failure is reported in the line, not raised."""
    try:
        return fn()
    except Exception as e:
        return {"error": f"{type(e).__name__}: {str(e)[:400]}"}


def parity_against_oracle(x_oracle, x_fp32, x_fp64):
    """Slab 1 of the march: the GPU solutions (FP32 and FP64 V-cycle, FGMRES to 1e-8)
    against the FP64 oracle's solution of the same slab (FGMRES + V-cycle to 1e-12), after
    removing the pressure mean of every temporal dof (the pressure is determined up to these
    constants)."""
    if x_oracle is None:
        return {"slab": 1, "note": "the oracle sample is not the benched workload's size; see tests/"}
    import numpy as np
    w = WORKLOAD
    d, n, r, k = w["dim"], w["n_cells"], w["r"], w["k"]
    nv = d * ((r + 1) * n + 1) ** d
    npm = math.comb(r + d, d)
    kt = k + 1

    def center(x):
        x = x.copy()
        o = kt * nv
        npr = npm * n ** d
        for a in range(kt):
            p = x[o + a * npr:o + (a + 1) * npr]
            p[::npm] -= p[::npm].mean()
        return x

    ref = center(x_oracle)
    vel = slice(0, kt * nv)
    pre = slice(kt * nv, None)
    out = {"slab": 1, "reference": "FP64 oracle, FGMRES + V-cycle to 1e-12 (same hierarchy)",
           "tolerance_gpu": 1e-8}
    for tag, x in (("fp32_vcycle", x_fp32), ("fp64_vcycle", x_fp64)):
        if x is None:
            continue
        xc = center(x)
        out[tag] = {"rel_err_max": float(np.abs(xc - ref).max() / np.abs(ref).max()),
                    "rel_err_velocity_l2": float(np.linalg.norm(xc[vel] - ref[vel]) / np.linalg.norm(ref[vel])),
                    "rel_err_pressure_l2": float(np.linalg.norm(xc[pre] - ref[pre]) / np.linalg.norm(ref[pre]))}
    return out


def only_kernel(mg, args):
    """One kernel of the headline handle, `reps` launches inside cudaProfilerStart/Stop after
    three warm-up launches (for `ncu --profile-from-start off`); CUDA-event time per launch."""
    import torch
    prec = args.prec
    dt = torch.float64 if prec == "fp64" else torch.float32
    lvl = args.level
    D = mg.size(lvl)
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(D, generator=gen, device="cuda", dtype=dt)
    b = torch.rand(D, generator=gen, device="cuda", dtype=dt)
    y = torch.zeros_like(x)
    v64 = torch.rand(mg.size(0), generator=gen, device="cuda", dtype=torch.float64)
    z64 = torch.empty_like(v64)
    if args.only_kernel in ("restrict", "prolong"):
        xc = torch.rand(mg.size(lvl + 1), generator=gen, device="cuda", dtype=dt)
    fns = {"apply": lambda: mg.apply(x, lvl, out=y),
           "residual": lambda: mg.residual(b, x, lvl, out=y),
           "sweep": lambda: mg.vanka_sweep(b, y, lvl),
           "restrict": lambda: mg.restrict(x, lvl, out=xc),
           "prolong": lambda: mg.prolongate_add(xc, y, lvl),
           "vcycle": lambda: mg.vcycle(v64, prec, out=z64)}
    if args.only_kernel == "cgs2":
        # one FGMRES solve of slab 1's right-hand side: the Arnoldi steps are the k_cgs2 launches
        fb = torch.rand(mg.size(0), generator=gen, device="cuda", dtype=torch.float64)
        fns["cgs2"] = lambda: mg.solve_slab(fb, out=torch.zeros_like(fb))
    fn = fns[args.only_kernel]
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record()
    for _ in range(args.reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / args.reps
    out = {"kernel": args.only_kernel, "prec": prec, "level": lvl, "dofs": D, "ms": ms, "dofs_per_s": D / (ms / 1e3),
           "levels": [(l["n"], l["r"], l["k"]) for l in mg.levels],
           "launch_shapes": [{k: l[k] for k in ("apply_variant", "apply_tile", "apply_cells_per_block", "sweep_variant",
                                                "patches_per_block", "sweep_unroll", "transfer_cells_per_block",
                                                "persistent")} for l in mg.levels]}
    if args.only_kernel == "sweep":
        out["alg_bytes"] = sweep_alg_bytes(mg.levels[lvl], prec)
        out["GBs"] = out["alg_bytes"] / (ms / 1e3) / 1e9
    return out


def warm_start_bench():
    """The learned initial guess on its workload: 2D 128^2 Q3/P2disc DG(1), 256 slabs on
    [0, 1], Fourier forcing (seeds 4, 5) whose phases drift by 0.05 * 2 pi per unit time.
    Slabs 0-127 are solved from the extrapolated guess; pairs of slabs 16-127 (after the
    start-up transient) train the network on the initial-residual ratio; slabs 128-255 are
    then marched three times, from the zero, the extrapolated and the learned guess, each
    timed with CUDA events including the guess itself."""
    import numpy as np
    import torch

    import paper_2502_09159_gb300 as stmg
    from paper_2502_09159_gb300.warmstart import WarmStart
    from workloads import fourier_forcing_2d
    n, N = 128, 256
    pb = fourier_forcing_2d(nu=1.0, seed_psi=4, seed_phi=5, drift=0.05 * 2 * math.pi)
    g = stmg.SpaceTimeMG(dim=2, n_cells=n, r=2, k=1, nu=1.0, T=1.0, n_slabs=N, precond_precision="fp32",
                         coarse_n=8, k_min=1)
    D = g.size(0)
    pts = g.forcing_points()
    F = [g.forcing(pb.forcing, s, pts) for s in range(N)]
    ws = WarmStart(g, hidden=64, layers=4, capacity=N // 2, seed=1)
    b = g.empty()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x_prev = g.zeros()
    for s in range(N // 2):
        g.slab_rhs(F[s], x_prev if s else None, out=b)
        x, info = g.solve_slab(b, ws.guess(x_prev, "extrapolate") if s else None)
        g.remove_pressure_mean(x)
        if s >= 16:
            ws.add_pair(x_prev, x)
        x_prev = x
    e1.record()
    torch.cuda.synchronize()
    collect_ms = e0.elapsed_time(e1)
    start = x_prev
    e0.record()
    losses = ws.fit_residual(steps=800, batch=4, lr=1e-4, warmup=100)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    ratio = ws.residual_ratio()
    modes = {}
    guess_buf = g.empty()
    for m in WarmStart.MODES:
        its = []
        xp = start
        sols = [g.empty() for _ in range(2)]
        torch.cuda.synchronize()
        e0.record()
        for s in range(N // 2, N):
            g.slab_rhs(F[s], xp, out=b)
            ws.guess(xp, m, out=guess_buf)
            x = sols[s % 2]
            x.copy_(guess_buf)
            _, info = g.solve_slab(b, out=x)
            if info["status"] != 0:
                raise RuntimeError(f"warm start {m}: slab {s}: {info}")
            its.append(info["iterations"])
            xp = x
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        modes[m] = {"ms_per_slab": round(ms / (N // 2), 3), "mean_iterations": round(statistics.mean(its), 3),
                    "theta_dofs_per_s": (N // 2) * D / (ms / 1e3)}
    # the guess alone (gather, network, scatter, extrapolation) per slab
    torch.cuda.synchronize()
    e0.record()
    for _ in range(20):
        ws.guess(start, "net", out=guess_buf)
    e1.record()
    torch.cuda.synchronize()
    out = {"workload": "2D 128x128 Q3/P2disc DG(1), 256 slabs, drifting Fourier forcing (seeds 4, 5); "
                       "train on slabs 16-127, evaluate on 128-255",
           "dofs_per_slab": D, "network": "4 conv3x3 layers, 64 channels, linear 3x3 bypass, FP32",
           "train_pairs": ws.count, "collect_ms": round(collect_ms, 1), "train_ms": round(train_ms, 1),
           "train_steps": len(losses), "residual_ratio_sq_train": round(ratio, 4),
           "net_guess_ms": round(e0.elapsed_time(e1) / 20, 3), "modes": modes}
    g.close()
    return out


def run_e2e(mg, F, N, D, world, args, barrier, boundary_data):
    """The march end to end through the C ABI's host-buffer call (stmg_march_host): every
    step copies all slabs' inputs (forcing, or boundary values for the cavity) from pinned
    host memory and every solution back, inside the timed region (the library overlaps the
    copies with the solves on a copy stream)."""
    import torch
    Fh = torch.stack([f.cpu() for f in F]).pin_memory()
    Xh = torch.empty_like(Fh).pin_memory()
    Fn, Xn = Fh.numpy(), Xh.numpy()
    mg.march_host(Fn, Xn, boundary_data=boundary_data)          # warm-up
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        infos = mg.march_host(Fn, Xn, boundary_data=boundary_data)
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = max_over_ranks(e2e_ms, world, device="cuda")
    return {"value": world * N * D / (e2e_ms / 1e3), "unit": "space-time DoFs/s", "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": N * D * 8, "d2h_bytes_per_step": N * D * 8,
            "api": "stmg_march_host (C ABI, host FP64 buffers in pinned memory)",
            "mean_gmres_iterations": statistics.mean(i["iterations"] for i in infos)}


def time_split(mg, step_fn):
    """One more march with events around every category (the split of the paper's
    lid-cavity breakdown): smoother, MG without smoother, operator outside MG, other."""
    import torch
    mg.set_profiling(2)
    mg.profile(reset=True)
    torch.cuda.synchronize()
    t0 = time.time()
    step_fn(mg, [])
    torch.cuda.synchronize()
    wall = (time.time() - t0) * 1e3
    p = mg.profile(reset=True)
    mg.set_profiling(0)
    out = {k: round(v["ms"], 3) for k, v in p.items()}
    out["wall_ms"] = round(wall, 3)
    return out


def other_hierarchy(make, step_fn, N, D, coarse_n=None, k_min=None, lv=None, what="", max_iter=None):
    """The same workload and FP32 V-cycle on another level list: its march, timed once after
    one warm-up march.  Slabs that do not reach 1e-8 within the iteration budget are listed."""
    import torch
    kw = {}
    if max_iter is not None:
        kw["max_iter"] = max_iter
    if coarse_n is not None:
        kw["coarse_n"] = coarse_n
    if k_min is not None:
        kw["k_min"] = k_min
    if lv is not None:
        kw["lv"] = lv
    g = make("fp32", **kw)
    its, bad = [], []
    step_fn(g, its, bad)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its, bad = [], []
    e0.record()
    step_fn(g, its, bad)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"value": N * D / (ms / 1e3), "ms_per_step": ms, "mean_iterations": statistics.mean(its),
           "max_iterations": max(its), "levels": [(l["n"], l["r"], l["k"]) for l in g.levels], "hierarchy": what}
    if bad:
        out["not_converged"] = [{"slab": b["slab"], "iterations": b["iterations"],
                                 "rel_residual": b["rel_residual"]} for b in bad]
        out["value"] = None
    g.close()
    return out


def micro(mg, make, N, D, step_fn, x_bufs):
    """Per-kernel rates on the finest level (CUDA events, 20 back-to-back calls after 3
    warm-ups), and time-to-1e-8 of the FP64 vs the FP32 V-cycle (and FP16 inverses) over
    the same march.  Returns the report and slab 1's solution with the FP64 V-cycle."""
    import torch
    out = {}

    def timeit(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    x64 = torch.randn(D, dtype=torch.float64, device="cuda")
    x32 = x64.float()
    y64, y32 = torch.empty_like(x64), torch.empty_like(x32)
    rates = {}
    have = [("fp64", x64, y64)] if mg.levels[0]["inverse_bytes"][0] else []
    for tag, x, y in have + [("fp32", x32, y32)]:
        t = timeit(lambda: mg.apply(x, 0, out=y))
        rates[f"apply_{tag}"] = D / (t / 1e3)
        t = timeit(lambda: mg.vanka_sweep(x, y, 0))
        rates[f"vanka_sweep_{tag}"] = D / (t / 1e3)
        rates[f"vanka_sweep_{tag}_GBs"] = sweep_alg_bytes(mg.levels[0], tag) / (t / 1e3) / 1e9
        t = timeit(lambda: (mg.residual(x, y, 0, out=y), mg.vanka_sweep(y, x, 0)))
        rates[f"smoothing_step_{tag}"] = D / (t / 1e3)
        b = x64.clone()
        z = torch.empty_like(b)
        t = timeit(lambda: mg.vcycle(b, tag, out=z))
        rates[f"vcycle_{tag}"] = D / (t / 1e3)
        rates[f"vcycle_{tag}_us"] = t * 1e3
    out["rates_dofs_per_s"] = {k: float(f"{v:.4g}") for k, v in rates.items()}
    # time-to-1e-8: FP64 preconditioner vs FP32 preconditioner, same march
    tt = {}
    x1_fp64 = None
    for prec in ("fp64", "fp32"):
        g = mg if prec == "fp32" else make("fp64")     # FP64 V-cycle (FP64 inverses)
        its = []
        step_fn(g, its)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record()
        step_fn(g, its)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tt[prec] = {"ms_per_slab": ms / N, "mean_iterations": statistics.mean(its), "theta_dofs_per_s": N * D / (ms / 1e3)}
        if g is not mg:
            x1_fp64 = x_bufs[0].cpu().numpy()
            g.close()
    # the same march with half-precision patch inverses in the FP32 V-cycle
    g = make("fp32", half=True)
    its = []
    step_fn(g, its)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its = []
    e0.record()
    step_fn(g, its)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    x = torch.randn(D, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    t = timeit(lambda: g.vanka_sweep(x, y, 0))
    tt["fp32_half_inverses"] = {"ms_per_slab": ms / N, "mean_iterations": statistics.mean(its),
                                "theta_dofs_per_s": N * D / (ms / 1e3),
                                "finest_sweep_GBs": g.sweep_bytes(0, "fp32") / (t / 1e3) / 1e9,
                                "finest_inverse_bytes": g.levels[0]["inverse_bytes"][1]}
    g.close()
    out["time_to_1e-8"] = tt
    return out, x1_fp64


def throughput_grid(reps=10):
    """A subset of the (dim, r, k) throughput grid: 2D 256^2 and 3D 16^3, r = 1, 2, 4,
    k = 0, 2, FP32 and FP64, random inputs U[0,1) (cost is data independent), launch shapes
    autotuned, V-cycle as a CUDA graph.  Per point: the finest level's apply, Vanka sweep and
    V-cycle in dofs/s (CUDA events, `reps` back-to-back calls after 3 warm-ups) and the
    sweep's and apply's fraction of the measured HBM bandwidth (sweep: n_patches B^2 s +
    3 D s bytes; apply: 2 D s, x in and y out)."""
    import torch

    import paper_2502_09159_gb300 as stmg
    peaks, peak_kind = measured_peaks()
    peak = peaks["hbm_gbs"]
    rows = []

    def timeit(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_all = time.perf_counter()
    for dim in (2, 3):
        n = 256 if dim == 2 else 16
        for r in (1, 2, 4):
            for k in (0, 2):
                t0 = time.perf_counter()
                g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, precisions=("fp64", "fp32"),
                                     precond_precision="fp32", use_graphs=True)
                setup_s = time.perf_counter() - t0
                D = g.size(0)
                lv = g.levels[0]
                for prec in ("fp32", "fp64"):
                    dt = torch.float32 if prec == "fp32" else torch.float64
                    sz = 4 if prec == "fp32" else 8
                    gen = torch.Generator(device="cuda").manual_seed(3)
                    x = torch.rand(D, generator=gen, device="cuda", dtype=dt)
                    y = torch.zeros_like(x)
                    b64 = torch.rand(D, generator=gen, device="cuda", dtype=torch.float64)
                    z64 = torch.empty_like(b64)
                    ta = timeit(lambda: g.apply(x, 0, out=y))
                    ts = timeit(lambda: g.vanka_sweep(x, y, 0))
                    tv = timeit(lambda: g.vcycle(b64, prec, out=z64))
                    sb = sweep_alg_bytes(lv, prec)
                    rows.append({"dim": dim, "n": n, "r": r, "k": k, "prec": prec, "D": D, "B": lv["patch_size"],
                                 "apply_Gdofs": round(D / ta / 1e6, 3), "apply_us": round(ta * 1e3, 1),
                                 "apply_hbm_frac": round(2 * D * sz / (ta / 1e3) / 1e9 / peak, 4),
                                 "sweep_Gdofs": round(D / ts / 1e6, 3), "sweep_us": round(ts * 1e3, 1),
                                 "sweep_GBs": round(sb / (ts / 1e3) / 1e9, 1),
                                 "sweep_hbm_frac": round(sb / (ts / 1e3) / 1e9 / peak, 4),
                                 "vcycle_Gdofs": round(D / tv / 1e6, 3), "vcycle_us": round(tv * 1e3, 1),
                                 "vectors_fit_l2": 3 * D * sz < 129e6, "setup_s": round(setup_s, 1)})
                g.close()
                del g
                torch.cuda.empty_cache()
    return {"peak_GBs": peak, "peak_kind": peak_kind, "seconds": round(time.perf_counter() - t_all, 1),
            "note": "back-to-back calls; where vectors_fit_l2 the apply's vectors are L2-resident",
            "rows": rows}


# ----------------------------------------------------------------------------- oracle
_ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle.stokes import MGConfig, Multigrid, default_hierarchy, fgmres
from workloads import fourier_forcing_2d, lid_driven_3d, taylor_green_3d
w = {w!r}
kind = {kind!r}
pb = (fourier_forcing_2d(nu=w["nu"]) if kind == "fourier" else
      lid_driven_3d(nu=w["nu"], T=w["T"]) if kind == "lid" else taylor_green_3d(nu=w["nu"]))
tau = w["T"] / w["n_slabs"]
t0 = time.time()
mg = Multigrid(w["dim"], default_hierarchy(w["n_cells"], w["r"], w["k"], {coarse_n}, {k_min}), w["nu"], tau,
               MGConfig())
t_setup = time.time() - t0
slab = mg.slabs[0]
b = slab.rhs_forcing(pb.forcing, 0.0)
if pb.boundary is not None:
    b = slab.lift(slab.boundary_vector(pb.boundary, 0.0), b)
bar, nproc, me = {barrier!r}, {nproc!r}, {me!r}
if bar:                                   # start the timed solves of all processes together
    open(os.path.join(bar, "ready.%d" % me), "w").close()
    t_wait = time.time()
    while sum(f.startswith("ready.") for f in os.listdir(bar)) < nproc and time.time() - t_wait < 900:
        time.sleep(0.05)
times = []
for rep in range({reps}):
    t0 = time.time()
    x, info = fgmres(lambda z: slab.S @ z, mg.vcycle, b, tol=1e-8)
    times.append(time.time() - t0)
if {save!r}:                              # reference solution for the parity report (untimed)
    x12, info12 = fgmres(lambda z: slab.S @ z, mg.vcycle, b, tol=1e-12)
    np.save({save!r}, x12)
print(json.dumps({{"setup_s": t_setup, "solve_s": times, "iterations": info.iterations, "D": slab.size}}))
"""


def oracle_workload():
    """The oracle's bounded sample: the workload itself in 2D; in 3D the same discretisation
    on an 8^3 mesh (the assembled 32^3 system does not fit the oracle)."""
    w = dict(WORKLOAD)
    if w["dim"] == 3:
        w["n_cells"] = min(w["n_cells"], 8)
    return w


def host_cpu():
    """CPU model and the cores this process may use."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    return model or "unknown", cores


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except Exception:
        pass
    return 16.0


def _oracle_code(reps, coarse_n, k_min, save=None, barrier=None, nproc=1, me=0):
    w = oracle_workload()
    kind = WORKLOADS_KIND.get(WORKLOAD_NAME, "fourier")
    return _ORACLE_SNIPPET.format(root=ROOT, w=w, kind=kind, reps=reps, coarse_n=min(coarse_n, w["n_cells"]),
                                  k_min=k_min, save=save, barrier=barrier, nproc=nproc, me=me)


_ENV1 = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def oracle_sample(reps, coarse_n=8, k_min=2, save=None):
    """One oracle process on one core: setup, then `reps` timed slab-1 solves to 1e-8."""
    p = subprocess.run([sys.executable, "-c", _oracle_code(reps, coarse_n, k_min, save)], capture_output=True,
                       text=True, env=_ENV1, timeout=1800)
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def oracle_sample_parallel(nproc, reps, coarse_n=8, k_min=2):
    """`nproc` single-threaded oracle processes, one per core, each solving slab 1 `reps`
    times; their timed solves start together (file barrier after the untimed setup)."""
    import shutil
    import tempfile
    bar = tempfile.mkdtemp(prefix="stmg_oracle_")
    try:
        procs = [subprocess.Popen([sys.executable, "-c", _oracle_code(reps, coarse_n, k_min, None, bar, nproc, i)],
                                  stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=_ENV1)
                 for i in range(nproc)]
        res = []
        for p in procs:
            out, err = p.communicate(timeout=1800)
            if p.returncode != 0:
                raise RuntimeError(err[-2000:])
            res.append(json.loads(out.strip().splitlines()[-1]))
        return res
    finally:
        shutil.rmtree(bar, ignore_errors=True)


def oracle_procs():
    """Processes for the all-cores oracle: one per usable core, at most one per 2.5 GB of
    available host memory (the config-2 oracle holds about 2 GB)."""
    _, cores = host_cpu()
    n = max(1, min(cores, int(_mem_available_gb() / 2.5)))
    cap = os.environ.get("STMG_ORACLE_PROCS")            # an upper limit, e.g. for a quick CPU test
    return min(n, max(1, int(cap))) if cap else n


def cpu_baseline(coarse_n=8, k_min=2):
    """The FP64 oracle on the host cores: one process per core solving slab 1 concurrently
    (value), and one process alone (single_core).  Also returns the oracle's slab-1 solution
    to 1e-12 when the sample is the benched workload itself (2D), else None."""
    import tempfile

    import numpy as np
    model, _ = host_cpu()
    ow = oracle_workload()
    same = ow["n_cells"] == WORKLOAD["n_cells"]
    save = os.path.join(tempfile.gettempdir(), f"stmg_oracle_x1_{os.getpid()}.npy") if same else None
    x_ref = None
    out = {"value": None, "unit": "space-time DoFs/s", "cores": None, "kind": "oracle", "cpu": model}
    try:
        r1 = oracle_sample(1, coarse_n, k_min, save)
        t1 = min(r1["solve_s"])
        out["single_core"] = {"value": r1["D"] / t1, "cores": 1, "solve_s": round(t1, 2),
                              "setup_s": round(r1["setup_s"], 1), "iterations": r1["iterations"]}
        if save:
            x_ref = np.load(save)
            os.remove(save)
    except Exception as e:  # the baseline is reported, not required
        out["single_core"] = {"error": str(e)[:300]}
    try:
        P = oracle_procs()
        rs = oracle_sample_parallel(P, 1, coarse_n, k_min)
        tmax = max(min(r["solve_s"]) for r in rs)
        out["value"] = P * rs[0]["D"] / tmax
        out["cores"] = P
        out["solve_s_slowest"] = round(tmax, 2)
    except Exception as e:
        out["error"] = str(e)[:300]
        if "value" in out.get("single_core", {}):
            out["value"], out["cores"] = out["single_core"]["value"], 1
    out["sample"] = (f"slab 1 of {WORKLOAD['n_slabs']} ({ow['n_cells']}^{WORKLOAD['dim']} cells) solved by the FP64 "
                     f"oracle (FGMRES + V-cycle to 1e-8, setup not timed): value = {out['cores']} single-threaded "
                     f"processes solving it concurrently, one per core ({model}); single_core = one process alone")
    return out, x_ref


def run_reference(args):
    global WORKLOAD, WORKLOAD_NAME
    rank, world, _ = dist_env()
    if rank != 0:
        return
    WORKLOAD, WORKLOAD_NAME, _ = WORKLOADS[args.workload]
    if args.coarse_n == 0:
        args.coarse_n = 8 if WORKLOAD["dim"] == 2 else 1
    if args.k_min == 0:
        args.k_min = WORKLOAD["k"] if WORKLOAD["dim"] == 2 else 1
    model, _ = host_cpu()
    P = oracle_procs()
    rs = oracle_sample_parallel(P, args.warmup + args.steps, args.coarse_n, args.k_min)
    # per step: the slowest process's solve time of that step (all processes solve concurrently)
    per_step = [max(r["solve_s"][i] for r in rs) for i in range(args.warmup, args.warmup + args.steps)]
    t = sum(per_step) / len(per_step)
    D = rs[0]["D"]
    value = P * D / t
    ow = oracle_workload()
    sample = (f"per step: slab 1 of {WORKLOAD['n_slabs']} of the same workload on {ow['n_cells']}^{ow['dim']} cells "
              f"solved by the FP64 oracle (FGMRES + V-cycle to 1e-8, {rs[0]['iterations']} iterations) in each of "
              f"{P} single-threaded processes at once, one per core ({model}); setup not timed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "space-time DoFs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "dofs_per_slab": D, "oracle_processes": P},
            "cpu_baseline": {"value": value, "unit": "space-time DoFs/s", "cores": P, "kind": "oracle",
                             "cpu": model, "sample": sample},
            "e2e": {"value": value, "unit": "space-time DoFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
