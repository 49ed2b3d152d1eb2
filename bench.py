"""Benchmark: space-time DoF/s of the heat-equation space-time multigrid solve
to a 1e-8 relative residual on one GB300 (or N independent problems on N GPUs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl stmg|reference]

A step is one full solve (st_solve) of the 2D workload heat2d_255: Q1 on the
unit square with 255^2 interior nodes, DG degree p_t = 1, N = 1024 time steps,
T = 1 (133,171,200 unknowns, 1.07 GB per FP64 vector, far above the 129 MB
L2, so no flush is needed between steps); f ~ U[-1,1] (seed 0 + rank),
u0 = sin(pi x) sin(pi y).  The headline value is the plain FP64 solve; the
mixed-precision form (FP32 V-cycles inside FP64 refinement) of the same solve
is reported under "mixed".  Device time comes from CUDA events on the
solver's stream; "e2e" repeats the solve through st_solve_host with f and u0
in pinned host memory and u written back to pinned host memory inside the
timed region (the transform kernels read and write the host buffers over the
CPU-GPU link).  Kernel time per class comes from the library's event timing
(st_profile_start/stop) over the timed region; "roofline" evaluates the
dominant class on the finest level against the measured peaks, with the DRAM
traffic of its ncu capture (profiles/).  Further legs: the paper's inexact
block inverse ("inexact_smoother"), the Example 2 protocol at p_t = 45
("high_order"), the CPU oracle on a bounded sample ("cpu_baseline"), the SM
clocks sampled during the timed region ("clocks"), and the time of one cycle
("vcycle").

Under torchrun every rank solves its own problem (no data-path collective,
"scaling": "weak"); rank 0 prints one JSON line.

--impl reference times the CPU oracle (oracle/, SciPy sparse LU) on a bounded
sample of the same workload: the first 8 of the 1024 time steps (same tau and
mesh) solved to the same tolerance; DoF/s = sampled DoF / solve time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "heat2d_255"
METRIC = "space-time DoF/s to 1e-8 rel. residual (FP64 vs mixed); V-cycle HBM GB/s"
CPU_SAMPLE_STEPS = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="stmg", choices=["stmg", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-fft-leg", action="store_true",
                    help="skip the FP64 solve with FFT sine transforms (comparison with the tensor-core transforms)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-inexact", action="store_true",
                    help="skip the solve with the inexact block inverse (one spatial V-cycle per step)")
    ap.add_argument("--no-high-order", action="store_true",
                    help="skip the Example 2 solve at p_t = 45 (generic-q kernels)")
    ap.add_argument("--inner-cycles", type=int, default=4)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the mixed-against-FP64 legs on heat3d_63 and heat2d_511")
    ap.add_argument("--no-mesh", action="store_true",
                    help="skip Example 2 on the paper's refined triangle mesh (P1 mesh solver)")
    ap.add_argument("--two-grid", action="store_true",
                    help="report mode: the two-grid convergence factors of Section 3.2 measured on the GPU over "
                         "mu = 1e-6 ... 1e6 (4 points per decade), p_t in {0, 1}, nu in {1, 2, 5}, semi and full "
                         "coarsening; prints one JSON line with every point")
    ap.add_argument("--only", choices=["fp64", "mixed", "mesh", "configs"], default=None,
                    help="profiling: one precision of the main workload only (the line's value is that "
                         "precision's), or only the mesh leg / the heat3d_63 and heat2d_511 legs (the line "
                         "carries that leg)")
    ap.add_argument("--mesh-level", type=int, default=7, help="refinements of the 4-triangle square (mesh leg)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return {"hbm_gbs": p.get("hbm_gbs", 6800.0), "src": "measured",
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", 1700.0)}
    return {"hbm_gbs": 6800.0, "src": "fallback", "bf16_tflops_sustained": 1700.0}


# FP64 vector-ALU peak of a GB300: 1.25 TFLOP/s (the published per-GPU FP64
# figure); an FMA-chain probe on this part reached 1.196 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
# FP32 vector-ALU peak: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def inputs(w, rank):
    from paper_1411_0519_gb300 import workloads
    f = workloads.uniform_load(w["d"], w["n"], w["p_t"], w["N"], seed=rank)
    u0 = workloads.sine_ic(w["d"], w["n"])
    return f, u0


def time_solves(torch, solver, f, u0, u, steps, warmup, barrier):
    """Warm-up, then `steps` solves timed with CUDA events on the solver's stream."""
    u = solver.empty() if u is None else u
    for _ in range(warmup):
        solver.solve(f, u0, u=u, initial_guess=False)
    stream = solver.stream
    iters = []
    barrier()
    torch.cuda.synchronize()
    solver.profile_start(400000)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    relres = None
    for _ in range(steps):
        _, it, relres = solver.solve(f, u0, u=u, initial_guess=False)
        iters.append(it)
    e1.record(stream)
    e1.synchronize()
    prof = solver.profile_stop()
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1), iters, relres, prof


def traffic_table():
    """Measured DRAM bytes per unknown of finest-level kernels, from the ncu
    captures summarised in profiles/ (taken on a smaller case of the same
    kernel and scaled by unknowns; each entry names the kernel, the case and
    the summary it comes from)."""
    path = os.path.join(ROOT, "profiles", "traffic_per_dof.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


TRANSFORM_CLASSES = ("dst", "dst_tc")
KERNEL_OF_CLASS = {"smooth": "k_fsmooth", "residual": "k_fresidual", "dst": "k_dst_rows_reg / k_dst_cols_reg",
                   "dst_tc": "k_dst_tc",
                   "restrict": "k_frestrict", "prolong": "k_fprolong", "space_mg": "k_fspace_pre / k_fspace_post"}


def roofline(solver, prof, fp32, pk, w, exclude=()):
    """Dominant kernel class of the timed region (classes in `exclude` left out),
    evaluated on the finest level (one launch = one pass over the finest level)."""
    classes = {k: v for k, v in prof.items() if not k.startswith("_") and v["ms"] > 0}
    dom = max((k for k in classes if k not in exclude), key=lambda k: classes[k]["ms"])
    total_ms = sum(c["ms"] for c in classes.values())
    L = solver.num_levels - 1
    v = solver.profile_level(dom, L)
    if v["launches"] == 0 or v["ms"] <= 0:
        v = classes[dom]
    sec = v["ms"] / 1e3
    gbs = v["bytes"] / sec / 1e9
    tfl = v["flops"] / sec / 1e12
    alu_peak = FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS
    f_hbm = gbs / pk["hbm_gbs"]
    f_alu = tfl / alu_peak
    if f_alu >= f_hbm:
        rf = {"bound": "alu", "achieved": round(tfl, 4), "peak": alu_peak, "unit": "TFLOP/s",
              "frac": round(f_alu, 4), "peak_src": "FP32 lanes x clock" if fp32 else
              "published FP64 rate 1.25 TFLOP/s (FMA probe on this part: 1.196)"}
    else:
        rf = {"bound": "hbm", "achieved": round(gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
              "frac": round(f_hbm, 4), "peak_src": pk["src"] + " (MEASURED_PEAKS.json hbm_gbs)"}
    launches = max(1, v["launches"])
    ndof = w["N"] * (w["p_t"] + 1) * w["n"] ** w["d"]
    key = "%s/%s/d%d_n%d_q%d" % (dom, "fp32" if fp32 else "fp64", w["d"], w["n"], w["p_t"] + 1)
    t = traffic_table().get(key)
    name = t["kernel"] if t else KERNEL_OF_CLASS.get(dom, dom) + ("_dyn" if w["p_t"] > 3 and dom in
                                                                   ("smooth", "residual") else "")
    traffic = t["bytes_per_dof"] * ndof if t else None
    rf.update({"kernel": name or dom, "level": "finest", "launches": v["launches"],
               "avg_launch_ms": round(v["ms"] / launches, 4), "share_of_class_total": round(
                   classes[dom]["ms"] / total_ms, 3),
               "alg_bytes_per_launch": v["bytes"] / launches, "alg_flops_per_launch": v["flops"] / launches,
               "traffic": traffic,
               # DRAM bytes per launch measured by ncu over this run's average launch time
               "traffic_gbs": round(traffic / (v["ms"] / launches / 1e3) / 1e9, 1) if traffic else None})
    return rf


def transform_note(prof, w, pk=None):
    """The boundary sine transforms of the solve: on the tensor cores (a digit-splitting
    pass, class dst, and the exact FP16 digit-product pass, class dst_tc, whose tensor
    rate is reported against the measured sustained BF16 GEMM rate; FP16 and BF16 run
    at the same rate), or double-float register FFTs on the FP32 pipe (class dst)."""
    classes = {k: v for k, v in prof.items() if not k.startswith("_") and v["ms"] > 0}
    total = sum(c["ms"] for c in classes.values())
    if "dst_tc" in classes:
        tc, sp = classes["dst_tc"], classes.get("dst", {"ms": 0.0, "launches": 0, "bytes": 0.0})
        peak = (pk or {}).get("bf16_tflops_sustained", 1700.0)
        tfl = tc["flops"] / (tc["ms"] / 1e3) / 1e12
        return {"kernel": "k_split_rows / k_split_cols + k_dst_tc", "arithmetic": "exact FP16 digit products, FP32 "
                "tensor-memory accumulators, integer assembly to FP64",
                "share_of_kernel_time": round((tc["ms"] + sp["ms"]) / total, 3),
                "launches": tc["launches"] + sp["launches"],
                "ms": round(tc["ms"] + sp["ms"], 3), "split_ms": round(sp["ms"], 3), "tensor_ms": round(tc["ms"], 3),
                "tensor_tflops": round(tfl, 1), "tensor_peak_tflops": peak,
                "tensor_frac": round(tfl / peak, 4), "peak_src": "MEASURED_PEAKS.json bf16_tflops_sustained",
                "split_gbs": round(sp["bytes"] / (sp["ms"] / 1e3) / 1e9, 1) if sp["ms"] > 0 else None}
    if "dst" not in classes:
        return None
    v = classes["dst"]
    return {"kernel": "k_dst_rows_reg / k_dst_cols_reg <dfloat>", "arithmetic": "double-float on the FP32 pipe",
            "share_of_kernel_time": round(v["ms"] / total, 3), "launches": v["launches"],
            "fp64_equivalent_tflops": round(v["flops"] / (v["ms"] / 1e3) / 1e12, 4),
            "bound": "latency (issue 48-52 %, 15.7 warps per SM; ncu)"}


def vcycle_times(solver, prof, steps, iters, per_step_ms, pk):
    """Time of one cycle: the solve time without the boundary transforms, per
    cycle, and the kernel time of the finest level per cycle (CUDA events of
    the library, transforms excluded); the cycle's achieved HBM rate is its
    algorithmic bytes (every kernel of the cycles and stopping tests, each
    input read once and each output written once, summed over all levels by
    the library) over that time, as a fraction of the measured copy rate."""
    L = solver.num_levels - 1
    cls = [c for c in prof if not c.startswith("_") and c not in TRANSFORM_CLASSES]
    fin = sum(solver.profile_level(c, L)["ms"] for c in cls)
    dst = sum(prof.get(c, {}).get("ms", 0.0) for c in TRANSFORM_CLASSES) / steps
    n = max(1, iters)
    ms = (per_step_ms - dst) / n
    by = sum(prof[c]["bytes"] for c in cls) / steps / n
    gbs = by / (ms / 1e3) / 1e9
    return {"ms_per_cycle_without_transforms": ms,
            "finest_level_kernel_ms_per_cycle": fin / steps / n,
            "alg_bytes_per_cycle": by, "achieved_gbs": round(gbs, 1), "peak_gbs": pk["hbm_gbs"],
            "frac": round(gbs / pk["hbm_gbs"], 4)}


def breakdown(prof):
    return {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                "GBs": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                "TFLOPs": round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 4)}
            for k, v in prof.items() if not k.startswith("_") and v["launches"] > 0}


def _oracle_worker(job):
    """One host core: the oracle (as it stands, one BLAS thread) solves the
    sampled window `job["window"]` of the workload's time steps, after all
    workers have finished their setup (barrier); returns wall-clock start/end
    of each timed solve."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass
    sys.path.insert(0, ROOT)
    from oracle import multigrid, spacetime
    from paper_1411_0519_gb300 import workloads
    w, Ns, i = job["w"], job["steps"], job["window"]
    tau = w["T"] / w["N"]
    H = multigrid.Hierarchy(w["d"], w["n"], w["p_t"], Ns, tau * Ns)
    disc = H.finest.disc
    f = workloads.uniform_load_steps(w["d"], w["n"], w["p_t"], w["N"], i * Ns, (i + 1) * Ns, seed=job["seed"])
    f = f.reshape(disc.shape())
    g = spacetime.add_ic(disc, f, workloads.sine_ic(w["d"], w["n"]))
    job["barrier"].wait()
    spans = []
    for _ in range(job["repeats"]):
        t0 = time.time()
        _, it, _ = multigrid.solve(H, g, rtol=w["rtol"], maxit=60)
        spans.append((t0, time.time(), it))
    return {"spans": spans, "dof": disc.ndof}


def cpu_baseline(w, rank, repeats=1, cores=None):
    """The oracle, as it stands, on every host core: each core (a spawned
    process with one BLAS thread) solves its own window of CPU_SAMPLE_STEPS
    consecutive time steps of the workload (same mesh and tau, its own rows of
    f) to the same tolerance, all at once after a common barrier.  Returns one
    entry per round of solves: DoF/s = DoF of all windows / wall time from the
    first start to the last end (setup excluded)."""
    import multiprocessing as mp
    if not cores:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    cores = max(1, min(cores, w["N"] // CPU_SAMPLE_STEPS))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        bar = mgr.Barrier(cores)
        jobs = [{"w": w, "steps": CPU_SAMPLE_STEPS, "window": i, "seed": rank, "repeats": repeats, "barrier": bar}
                for i in range(cores)]
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
    dof = sum(r["dof"] for r in res)
    out = []
    for k in range(repeats):
        t0 = min(r["spans"][k][0] for r in res)
        t1 = max(r["spans"][k][1] for r in res)
        its = sorted({r["spans"][k][2] for r in res})
        dt = t1 - t0
        out.append({"value": dof / dt, "unit": "DoF/s", "cores": cores, "kind": "oracle",
                    "sample": f"{cores} processes at once (one per host core, one BLAS thread each), each an oracle "
                              f"solve of its own {CPU_SAMPLE_STEPS} consecutive time steps of the {w['N']} (same mesh "
                              f"and tau, {res[0]['dof']} DoF each, {dof} in all) to {w['rtol']:g}: "
                              f"{'/'.join(map(str, its))} V-cycles, {dt:.1f} s wall; setup excluded",
                    "seconds": dt, "iters": its[-1], "dof": dof})
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    from paper_1411_0519_gb300 import workloads
    w = workloads.WORKLOADS[args.workload]
    if rank != 0:
        return 0
    # each step: one round of oracle solves of the bounded samples on every core; warm-up rounds untimed
    samples = cpu_baseline(w, 0, repeats=args.warmup + args.steps)[args.warmup:]
    sec = sum(s["seconds"] for s in samples)
    value = samples[0]["dof"] * len(samples) / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "d": w["d"], "n": w["n"], "p_t": w["p_t"], "N": w["N"],
                       "T": w["T"], "rtol": w["rtol"], "sampled_time_steps": CPU_SAMPLE_STEPS},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": samples[0]["cores"], "kind": "oracle",
                             "sample": samples[0]["sample"]},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_mixed_only(args, torch, stmg, w, f, u0, pk, world, rank, barrier, max_over_ranks, local):
    """Mixed-precision solve alone (used for profiling its kernels)."""
    d, n, p, N, T, rtol = w["d"], w["n"], w["p_t"], w["N"], w["T"], w["rtol"]
    smx = stmg.Solver(d, n, p, N, T, rtol=rtol, maxit=60, precision="mixed", inner_cycles=args.inner_cycles)
    clocks = ClockSampler(local)
    clocks.start()
    msm, itm, rrm, profm = time_solves(torch, smx, f, u0, None, args.steps, args.warmup, barrier)
    ck = clocks.stop()
    msm = max_over_ranks(msm)
    if rank == 0:
        line = {"metric": METRIC, "value": world * smx.ndof / (msm / args.steps / 1e3), "unit": "DoF/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": msm / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 V-cycle in f64 refinement", "data": "synthetic",
                "config": {"workload": args.workload, "d": d, "n": n, "p_t": p, "N": N, "T": T, "rtol": rtol,
                           "precision": "mixed", "inner_cycles": args.inner_cycles},
                "iters": itm[-1], "relres": rrm, "roofline": roofline(smx, profm, True, pk, w, exclude=TRANSFORM_CLASSES), "transform": transform_note(profm, w),
                "kernels": breakdown(profm),
                "gpu_launches": sum(v["launches"] for k, v in profm.items() if not k.startswith("_")),
                "clocks": ck}
        print(json.dumps(line), flush=True)
    smx.close()
    return 0


def timed_solve(torch, solver, run, steps, warmup, barrier, max_over_ranks):
    """`run()` (one solve returning (iterations, relres)) `warmup` times untimed,
    then `steps` times between CUDA events on the solver's stream with the
    library's per-kernel timing on."""
    for _ in range(warmup):
        run()
    barrier()
    torch.cuda.synchronize()
    solver.profile_start(400000)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(solver.stream)
    res = [run() for _ in range(steps)]
    e1.record(solver.stream)
    e1.synchronize()
    prof = solver.profile_stop()
    ms = max_over_ranks(e0.elapsed_time(e1)) / steps
    return ms, res[-1][0], res[-1][1], prof


# The paper's initial triangulation of the unit square for Example 2 (Section 4):
# 4 triangles around the centre.
SQUARE_VERTS = [[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [0.5, 0.5]]
SQUARE_CELLS = [[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]]


def mesh_leg(args, torch, stmg, barrier, max_over_ranks, world, rank, level=7):
    """Example 2's protocol (Section 4) on the paper's own mesh family: the
    4-triangle square refined `level` times (P1, node basis), tau = 1,
    N = T = 1024, f = 0, iterate ~ U[0, 1] (seed = rank), the inexact block
    inverse (one spatial V-cycle per step), to 1e-8; p_t = 1 and 3, in FP64 and
    in the mixed form (FP32 cycles inside FP64 refinement).  Each timed solve
    starts from a copy of the same iterate (the copy is inside the timed region,
    one vector)."""
    out = {"workload": f"example2_mesh: 4 triangles refined {level} times, P1, N = 1024, tau = 1, f = 0, "
                       "iterate ~ U[0, 1], inexact block inverse (nu_x = 2, omega_x = 2/3)"}
    gen = torch.Generator(device="cuda")
    for p, prec in ((1, "fp64"), (3, "fp64"), (1, "mixed"), (3, "mixed")):
        s = stmg.MeshSolver(SQUARE_VERTS, SQUARE_CELLS, level, p, 1024, 1024.0, rtol=1e-8, maxit=40,
                            precision=prec, inner_cycles=args.inner_cycles)
        gen.manual_seed(rank)
        it0 = torch.rand(s.shape, dtype=torch.float64, device="cuda", generator=gen)
        u = torch.empty_like(it0)
        fz = torch.zeros_like(it0)
        for _ in range(1):
            u.copy_(it0)
            s.solve(fz, u=u, initial_guess=True)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nst = 2
        e0.record(s.stream)
        for _ in range(nst):
            with torch.cuda.stream(s.stream):
                u.copy_(it0)
            _, it, rr = s.solve(fz, u=u, initial_guess=True)
        e1.record(s.stream)
        e1.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1)) / nst
        out["p_t=%d %s" % (p, prec)] = {"value": world * s.ndof / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms,
                                        "iters": it, "relres": rr, "dof": s.ndof, "nodes": s.Nx,
                                        "ms_per_iteration": ms / max(1, it), "levels": s.num_levels,
                                        "inner_cycles": args.inner_cycles if prec == "mixed" else None}
        s.close()
        del it0, u, fz
        torch.cuda.empty_cache()
    return out


def config_legs(args, torch, stmg, workloads, pk, barrier, max_over_ranks, world, rank):
    """The mixed-against-FP64 comparison on its two stated workloads: heat3d_63
    (63^3 Q1, p_t = 2, N = 512, 384M unknowns, Gaussian load) and heat2d_511
    (511^2 Q1, p_t = 1, N = 2048, 1.07B unknowns) across the semi / full
    coarsening threshold (T = mu / 128 for mu in 1/16, 1/4, 1, 16), each solve to
    1e-8: DoF/s, cycles, final relative residual and the dominant kernel's
    roofline; heat2d_511 adds the adjoint solve (L^T lambda = f) in both forms.
    Entries are drawn on the device (torch's CUDA generator, seed = rank) for
    heat2d_511; heat3d_63 uses the seeded Gaussian load of the tests."""
    out = {}
    # ---- heat3d_63
    w = dict(workloads.WORKLOADS["heat3d_63"])
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    f = torch.from_numpy(workloads.gaussian_load(d, n, p, N, T, seed=rank)).cuda()
    leg = {"workload": "heat3d_63: 3D 63^3 Q1, p_t = 2, N = 512, T = 1, 16 Gaussians, u0 = 0",
           "dof": N * (p + 1) * n ** d}
    for prec in ("fp64", "mixed"):
        s = stmg.Solver(d, n, p, N, T, rtol=w["rtol"], maxit=60, precision=prec, inner_cycles=args.inner_cycles)
        u = s.empty()

        def run():
            _, it, rr = s.solve(f, u=u, initial_guess=False)
            return it, rr
        ms, it, rr, prof = timed_solve(torch, s, run, 2, 1, barrier, max_over_ranks)
        leg[prec] = {"value": world * s.ndof / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms, "iters": it,
                     "relres": rr, "roofline": roofline(s, prof, prec == "mixed", pk, w,
                                                        exclude=TRANSFORM_CLASSES if prec == "mixed" else ()),
                     "cycle": vcycle_times(s, prof, 2, it, ms, pk)}
        s.close()
        del u
        torch.cuda.empty_cache()
    leg["mixed_over_fp64"] = round(leg["mixed"]["value"] / leg["fp64"]["value"], 3)
    out["heat3d_63"] = leg
    del f
    torch.cuda.empty_cache()
    # ---- heat2d_511 across mu*
    w0 = dict(workloads.WORKLOADS["heat2d_511"])
    d, n, p, N = w0["d"], w0["n"], w0["p_t"], w0["N"]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(rank)
    f = torch.rand((N, p + 1, n, n), dtype=torch.float64, device="cuda", generator=gen).mul_(2.0).sub_(1.0)
    legs = {"workload": "heat2d_511: 2D 511^2 Q1, p_t = 1, N = 2048, T = mu / 128, f ~ U[-1, 1]",
            "dof": N * (p + 1) * n ** d}
    for mu in (1.0 / 16, 0.25, 1.0, 16.0):
        w = dict(w0)
        w["T"] = mu / 128.0
        entry = {}
        for prec in ("fp64", "mixed"):
            s = stmg.Solver(d, n, p, N, w["T"], rtol=w["rtol"], maxit=80, precision=prec,
                            inner_cycles=args.inner_cycles)
            if prec == "fp64":
                entry["levels_full"] = [s.level_info(L)["full"] for L in range(s.num_levels - 1)][::-1]
            u = s.empty()

            def run():
                _, it, rr = s.solve(f, u=u, initial_guess=False)
                return it, rr

            def run_adj():
                _, _, it, rr = s.adjoint_solve(f, lam=u)
                return it, rr
            ms, it, rr, prof = timed_solve(torch, s, run, 1, 1, barrier, max_over_ranks)
            msa, ita, rra, profa = timed_solve(torch, s, run_adj, 1, 1, barrier, max_over_ranks)
            entry[prec] = {"value": world * s.ndof / (ms / 1e3), "unit": "DoF/s", "ms_per_step": ms, "iters": it,
                           "relres": rr, "roofline": roofline(s, prof, prec == "mixed", pk, w,
                                                              exclude=TRANSFORM_CLASSES if prec == "mixed" else ()),
                           "cycle": vcycle_times(s, prof, 1, it, ms, pk),
                           "adjoint": {"value": world * s.ndof / (msa / 1e3), "unit": "DoF/s", "ms_per_step": msa,
                                       "iters": ita, "relres": rra}}
            s.close()
            del u
            torch.cuda.empty_cache()
        entry["mixed_over_fp64"] = round(entry["mixed"]["value"] / entry["fp64"]["value"], 3)
        legs["mu=%g" % mu] = entry
    out["heat2d_511"] = legs
    del f
    torch.cuda.empty_cache()
    return out


TWO_GRID_NX, TWO_GRID_NT = 1023, 256


def two_grid_factor(torch, stmg, workloads, p, mu, nu, full, eps=1e-140, max_iter=250):
    """Section 3.2's measured two-grid factor: max_k ||r_{k+1}|| / ||r_k|| over the
    cycles until ||r_k|| <= eps ||r_0|| or max_iter cycles, for L u = 0 from a
    random iterate in [0, 1] (1D, 1023 interior nodes, 256 steps, tau = mu h^2).
    A two-grid cycle is the library's cycle on a two-level hierarchy whose coarse
    level (128 steps) is solved exactly by forward substitution."""
    nx, nt = TWO_GRID_NX, TWO_GRID_NT
    h = 1.0 / (nx + 1)
    s = stmg.Solver(1, nx, p, nt, mu * h * h * nt, nu1=nu, nu2=nu, coarsening="full" if full else "semi",
                    coarsest_steps=nt // 2, rtol=0.0, maxit=1)
    u = torch.from_numpy(workloads.uniform_iterate(1, nx, p, nt, seed=0)).cuda()
    f = torch.zeros_like(u)
    r = s.residual(f, u)
    r0 = s.norm2(r)
    prev, worst, it = r0, 0.0, 0
    while it < max_iter:
        s.vcycle(u, f)
        s.residual(f, u, out=r)
        rn = s.norm2(r)
        it += 1
        worst = max(worst, rn / prev)
        prev = rn
        if rn <= eps * r0 or rn == 0.0:
            break
    s.close()
    return worst, it


def run_two_grid(args):
    import torch
    from paper_1411_0519_gb300 import stmg, workloads
    mus = [10.0 ** (e / 4.0) for e in range(-24, 25)]
    points = []
    t0 = time.perf_counter()
    for full in (False, True):
        for p in (0, 1):
            for nu in (1, 2, 5):
                for mu in mus:
                    fac, it = two_grid_factor(torch, stmg, workloads, p, mu, nu, full)
                    points.append({"coarsening": "full" if full else "semi", "p_t": p, "nu": nu, "mu": mu,
                                   "factor": fac, "cycles": it})
    dt = time.perf_counter() - t0
    line = {"metric": "two-grid convergence factor max_k ||r_{k+1}|| / ||r_k|| (Section 3.2)", "unit": "1",
            "value": max(q["factor"] for q in points if q["coarsening"] == "semi"), "n_gpus": 1,
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1D heat, 1023 interior nodes, 256 time steps, f = 0, u0 ~ U[0, 1] (seed 0), "
                                   "omega = 1/2, nu1 = nu2 = nu, until 1e-140 or 250 cycles",
                       "mu": "10^(k/4), k = -24 ... 24"},
            "seconds": dt, "points": points}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.two_grid:
        return run_two_grid(args)
    import torch
    from paper_1411_0519_gb300 import dist as pd
    from paper_1411_0519_gb300 import stmg, workloads

    rank, world, local = pd.env()
    torch.cuda.set_device(local)
    pd.init("nccl", torch.device("cuda", local))
    barrier = pd.barrier

    def max_over_ranks(x):
        return pd.max_over_ranks(x, device="cuda")

    w = workloads.WORKLOADS[args.workload]
    d, n, p, N, T, rtol = w["d"], w["n"], w["p_t"], w["N"], w["T"], w["rtol"]
    f_np, u0_np = inputs(w, rank)
    f = torch.from_numpy(f_np).cuda()
    u0 = torch.from_numpy(u0_np).cuda()
    pk = peaks()

    if args.only == "mixed":
        return run_mixed_only(args, torch, stmg, w, f, u0, pk, world, rank, barrier, max_over_ranks, local)
    if args.only in ("mesh", "configs"):
        del f, u0
        torch.cuda.empty_cache()
        if args.only == "mesh":
            leg = mesh_leg(args, torch, stmg, barrier, max_over_ranks, world, rank, level=args.mesh_level)
        else:
            leg = config_legs(args, torch, stmg, workloads, pk, barrier, max_over_ranks, world, rank)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "only": args.only, "n_gpus": world, "leg": leg}), flush=True)
        pd.finalize()
        return 0

    # ---------------------------------------------------------------- FP64 (headline)
    s64 = stmg.Solver(d, n, p, N, T, rtol=rtol, maxit=60, precision="fp64")
    clocks = ClockSampler(local)
    clocks.start()
    ms64, it64, rr64, prof64 = time_solves(torch, s64, f, u0, None, args.steps, args.warmup, barrier)
    ck = clocks.stop()
    ms64 = max_over_ranks(ms64)
    per_step = ms64 / args.steps
    value = pd.job_throughput(world, s64.ndof, per_step / 1e3)
    launches = sum(v["launches"] for k, v in prof64.items() if not k.startswith("_"))

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        # st_solve_host: pinned host f, u0 in, u out; the first transform pass reads f
        # from host memory and the last inverse pass writes u to it
        fh = torch.from_numpy(f_np).pin_memory()
        u0h = torch.from_numpy(u0_np).pin_memory()
        uh = torch.empty(s64.shape, dtype=torch.float64).pin_memory()
        s64.solve_host(fh, u0h, uh)                     # allocates its device buffer once
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s64.solve_host(fh, u0h, uh)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * s64.ndof * args.steps / dt, "unit": "DoF/s",
               "h2d_bytes_per_step": fh.numel() * 8 + u0h.numel() * 8, "d2h_bytes_per_step": uh.numel() * 8,
               "ms_per_step": 1e3 * dt / args.steps, "api": "st_solve_host"}
        del fh, u0h, uh
    rf64 = roofline(s64, prof64, False, pk, w)
    vc64 = vcycle_times(s64, prof64, args.steps, it64[-1], per_step, pk)
    tr64 = transform_note(prof64, w, pk)
    s64.close()
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- the same solve with the FFT transforms
    fft64 = None
    if not args.no_fft_leg:
        sf = stmg.Solver(d, n, p, N, T, rtol=rtol, maxit=60, precision="fp64", transform="fft")
        nst = min(args.steps, 3)
        msf, itf, rrf, proff = time_solves(torch, sf, f, u0, None, nst, 1, barrier)
        msf = max_over_ranks(msf)
        dsf = sum(proff.get(c, {}).get("ms", 0.0) for c in TRANSFORM_CLASSES) / nst
        dst64 = sum(prof64.get(c, {}).get("ms", 0.0) for c in TRANSFORM_CLASSES) / args.steps
        fft64 = {"value": world * sf.ndof / (msf / nst / 1e3), "unit": "DoF/s", "ms_per_step": msf / nst,
                 "iters": itf[-1], "relres": rrf, "transform_ms_per_solve": round(dsf, 3),
                 "tensor_transform_ms_per_solve": round(dst64, 3),
                 "note": "transform=fft: the boundary sine transforms as register FFTs on the FP64 pipe"}
        sf.close()
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- mixed precision
    mixed = None
    if not args.no_mixed and args.only != "fp64":
        smx = stmg.Solver(d, n, p, N, T, rtol=rtol, maxit=60, precision="mixed", inner_cycles=args.inner_cycles)
        msm, itm, rrm, profm = time_solves(torch, smx, f, u0, None, args.steps, max(1, args.warmup), barrier)
        msm = max_over_ranks(msm)
        mixed = {"value": world * smx.ndof / (msm / args.steps / 1e3), "unit": "DoF/s",
                 "ms_per_step": msm / args.steps, "iters": itm[-1], "relres": rrm,
                 "inner_cycles": args.inner_cycles, "dtype": "f32 V-cycle in f64 refinement",
                 "refinement_step": vcycle_times(smx, profm, args.steps, itm[-1], msm / args.steps, pk),
                 "roofline": roofline(smx, profm, True, pk, w, exclude=TRANSFORM_CLASSES),
                 "transform": transform_note(profm, w, pk),
                 "kernels": breakdown(profm),
                 "gpu_launches": sum(v["launches"] for k, v in profm.items() if not k.startswith("_"))}
        smx.close()

    # ---------------------------------------------------------------- inexact block inverse
    inexact = None
    if not args.no_inexact:
        inexact = {}
        for prec in ("fp64", "mixed"):
            si = stmg.Solver(d, n, p, N, T, rtol=rtol, maxit=60, precision=prec, inner_cycles=args.inner_cycles,
                             smoother="vcycle")
            msi, iti, rri, profi = time_solves(torch, si, f, u0, None, min(args.steps, 2), 1, barrier)
            msi = max_over_ranks(msi)
            nst = min(args.steps, 2)
            inexact[prec] = {"value": world * si.ndof / (msi / nst / 1e3), "unit": "DoF/s", "ms_per_step": msi / nst,
                             "iters": iti[-1], "relres": rri, "kernels": breakdown(profi)}
            si.close()
            torch.cuda.empty_cache()
        inexact["smoother"] = "one spatial V-cycle per time step, damped point-block Jacobi nu_x=2, omega_x=2/3"

    # ---------------------------------------------------------------- high time degree (Example 2)
    high = None
    if not args.no_high_order:
        wh = workloads.WORKLOADS["example2_p45"]
        sh = stmg.Solver(wh["d"], wh["n"], wh["p_t"], wh["N"], wh["T"], rtol=wh["rtol"], maxit=40)
        it0 = torch.from_numpy(workloads.uniform_iterate(wh["d"], wh["n"], wh["p_t"], wh["N"], seed=rank)).cuda()
        it0 = it0.view(sh.shape)
        fz = torch.zeros_like(it0)
        uh = sh.empty()
        nst = min(args.steps, 2)
        for _ in range(max(1, args.warmup // 3)):
            uh.copy_(it0)
            sh.solve(fz, u=uh, initial_guess=True)
        barrier()
        torch.cuda.synchronize()
        sh.profile_start(400000)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(sh.stream)
        ith = []
        for _ in range(nst):
            with torch.cuda.stream(sh.stream):
                uh.copy_(it0)
            _, itx, rrh = sh.solve(fz, u=uh, initial_guess=True)
            ith.append(itx)
        ev1.record(sh.stream)
        ev1.synchronize()
        profh = sh.profile_stop()
        msh = max_over_ranks(ev0.elapsed_time(ev1))
        high = {"workload": "example2_p45: 2D 127^2 Q1, p_t = 45 (q = 46), N = 64, tau = 1, f = 0, "
                            "iterate ~ U[0, 1] (Example 2 protocol)",
                "value": world * sh.ndof / (msh / nst / 1e3), "unit": "DoF/s", "ms_per_step": msh / nst,
                "iters": ith[-1], "relres": rrh, "dof": sh.ndof, "roofline": roofline(sh, profh, False, pk, wh),
                "kernels": breakdown(profh)}
        sh.close()
        del it0, fz, uh
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- the other stated workloads
    configs = None
    if not args.no_configs:
        configs = config_legs(args, torch, stmg, workloads, pk, barrier, max_over_ranks, world, rank)
    mesh = None
    if not args.no_mesh:
        mesh = mesh_leg(args, torch, stmg, barrier, max_over_ranks, world, rank, level=args.mesh_level)

    if rank != 0:
        pd.finalize()
        return 0

    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline(w, 0)[0]
        for k in ("seconds", "iters", "dof"):
            cpu.pop(k, None)

    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "d": d, "n": n, "p_t": p, "N": N, "T": T, "rtol": rtol,
                   "dof_per_gpu": s64.ndof, "nu1": 2, "nu2": 2, "omega": 0.5, "precision": "fp64",
                   "l2": "inputs larger than L2 (1.07 GB per vector), no flush"},
        "iters": it64[-1], "relres": rr64, "vcycle": vc64,
        "gpu_launches": launches,
        "roofline": rf64,
        "transform": tr64,
        "fp64_fft_transforms": fft64,
        "kernels": breakdown(prof64),
        "mixed": mixed,
        "inexact_smoother": inexact,
        "high_order": high,
        "configs": configs,
        "mesh": mesh,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    pd.finalize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
