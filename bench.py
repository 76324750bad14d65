#!/usr/bin/env python3
"""Benchmark of the ADMM hot path (Zhou & Bhattacharya, Section 2.1, Steps 1-4).

Workload: 3D 128^3 compressible neo-Hookean matrix (mu = 1) with periodic
spherical inclusions (mu = 10, radius 6 voxels, seeded centres, 20 % volume
fraction), nu = 0.3, Fbar = diag(0.9, 1, 1), rho = 10, solved to r_p, r_d <=
1e-8.  One step is one complete RVE solve from the fresh state (initialise,
iterate to tolerance, homogenised stress), i.e. every kernel of the path.

Prints ONE JSON line.  ``value`` is voxel-iterations/s of the default precision
mode (RVE_MIXED: float bulk, double residuals and stress, double polish) over
the timed steps; ``fp64`` repeats the measurement in plain double.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle on host cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADMM voxel-iterations/s and fraction of HBM roofline; p50/p99 RVE solve latency"
UNIT = "voxel-iterations/s"
N, DIM, SEED = 128, 3, 0
FBAR = np.diag([0.9, 1.0, 1.0])
RHO, TOL = 10.0, 1e-8
# the headline keeps rho fixed: the metric is per-iteration throughput, and the adaptive rule
# trades iterations for polish iterations (see bench_adaptive128 for its time to solution)
RHO_POLICY = "fixed"
MU = (1.0, 10.0)
NU = 0.3
L2_BYTES = 129e6

# algorithmic bytes per voxel and launch, per kernel class (s = bytes per scalar), for the
# headline's kernels (3D float neo-Hookean on a fixed grid size, RVE_MIXED)
#   local: read u~_{k+1} (d), F, Lambda (d^2 each); write F, Lambda; phase id (1 B).  The float
#     pass takes r_d from the spectral solve; the double one also reads u~_k (d)
#   xfwd: read F, Lambda; write the spectrum (d scalars);  fwd_y / inv_y / xinv: read + write d
#   scalars;  solve: the same, and in the float phase also read + write the kept spectrum for r_d
#   local_r (double-word polish): read the float u~ increment (d), R, F hi, F lo, Lambda lo, Z
#   (d^2 floats each); write F lo, Lambda lo, R (d^2 floats each); phase id
#   xfwd_incr: read R (d^2 floats), write the float spectrum;  xinv_incr: read the float spectrum
#   and the low parts of u~_k (float pairs after the direct switch), write the low parts of
#   u~_{k+1} and the float increment.  On the 128^3 float grid the inverse y and x transforms
#   run fused per z-plane: xinv and xinv_incr then time both (the same bytes: the spectrum
#   plane stays in shared memory) and inv_y has no launches
def bytes_per_voxel(cls: str, s: int, d: int = 3) -> float:
    return {"local": (d + 4 * d * d) * s + 1 + (d * s if s == 8 else 0), "local_first": (d + 3 * d * d) * s + 1,
            "xfwd": (2 * d * d + d) * s, "fwd_y": 2 * d * s, "solve": (4 if s == 4 else 2) * d * s,
            "inv_y": 2 * d * s, "xinv": 2 * d * s, "local_r": d * 4 + 8 * d * d * 4 + 1,
            "xfwd_incr": (d * d + d) * 4, "xinv_incr": 4 * d * 4}[cls]


# DRAM bytes (read + write) per launch measured with ncu on the 128^3 inclusion cell
# (profiles/), keyed by (kernel class, precision; solve: the float phase's z solve, which
# also reads and writes the kept spectrum); absent = not captured since the kernel last changed
TRAFFIC = {("local", "fp32"): 178659584 + 89560832, ("local_r", "fp64"): 415213312 + 181827840,
           ("xfwd", "fp32"): 151093248 + 9586432, ("fwd_y", "fp32"): 25188096 + 0,
           ("solve", "fp32"): 50367488 + 5888, ("xinv", "fp32"): 25196544 + 0,
           ("xfwd_incr", "fp32"): 75529216 + 134144, ("xinv_incr", "fp32"): 50368768 + 327680}
# FP32 flops per launch by kernel class, where counted with ncu for the current kernel
# (none since the float local step became the closed form: no ALU view is reported)
FLOPS = {}
# FP32 peak from unit counts and clock: 128 lanes x 2 flops x 152 SMs x 2.07 GHz
FP32_PEAK_TFLOPS = 128 * 2 * 152 * 2.07e9 / 1e12


def combine_ranks(ms, vox_it, dist=None, device="cpu"):
    """Whole-job figures over ranks that each solve their own RVE (weak scaling, no data-path
    collective): the slowest rank's time and the sum of the ranks' voxel-iterations."""
    if dist is None:
        return float(ms), float(vox_it)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    v = torch.tensor([float(vox_it)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), float(v.item())


def peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p = {"hbm_gbs": float(m["hbm_gbs"]), "source": "measured"}
    except Exception:
        pass
    return p


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def make_inputs(n=N):
    from paper_2010_06697_gb300 import synth
    ph = synth.inclusion_phase(n, DIM, SEED)
    par = synth.two_phase_params(MU[0], MU[1], NU)
    return ph, par


def _oracle_local_chunk(job):
    """Step 1 of the oracle (oracle.local_newton, as it stands) on one chunk of voxels:
    the unit of work the CPU baseline spreads over the host's cores."""
    import oracle
    from oracle import admm as oadmm
    ph, par, F, Lam, G, rho = job
    return oadmm.local_newton(oracle.make_material("neohookean", ph, par), F, Lam, G, rho)[0]


def oracle_pool_iterations(n: int, warmup: int, steps: int, procs: int) -> dict:
    """Time consecutive ADMM iterations of the FP64 oracle on the n^3 inclusion cell
    (from the fresh state; `warmup` untimed, then `steps` timed), with Step 1 -- most of
    the oracle's time -- split into chunks of voxels over `procs` spawned processes and
    Steps 2-4 (numpy FFTs and elementwise work) in this process.  Every step calls the
    oracle's own functions, in the order of oracle.admm_solve."""
    import multiprocessing as mp

    import oracle
    from oracle import admm as oadmm
    ph, par = make_inputs(n)
    mat = oracle.make_material("neohookean", ph, par)
    mu_ref = float(np.mean(mat.mu))
    st = oadmm.initial_state(mat, FBAR, ph.shape)
    F, Lam, u = st["F"], st["Lam"], st["u"]
    Fb = FBAR.reshape(3, 3, 1, 1, 1)
    G = Fb + oadmm.grad_u(u)
    phv = ph.reshape(-1)
    cuts = np.linspace(0, phv.size, 4 * procs + 1).astype(np.int64)
    times = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for it in range(warmup + steps):
            t = time.perf_counter()
            Fv, Lv, Gv = oadmm._to_voxels(F), oadmm._to_voxels(Lam), oadmm._to_voxels(G)
            jobs = [(phv[a:b], par, Fv[a:b], Lv[a:b], Gv[a:b], RHO) for a, b in zip(cuts[:-1], cuts[1:])]
            F = oadmm._to_field(np.concatenate(pool.map(_oracle_local_chunk, jobs)), ph.shape)
            uh, u = oadmm.u_step(F, Lam, RHO)
            G_new = Fb + oadmm.grad_from_spectrum(uh)
            Lam = oadmm.multiplier_update(Lam, G_new, F, RHO)
            r_p, r_d = oadmm.rms(G_new - F), RHO / mu_ref * oadmm.rms(G_new - G)
            G = G_new
            if it >= warmup:
                times.append(time.perf_counter() - t)
    return {"seconds": float(sum(times)), "iters": steps, "voxels": int(phv.size), "procs": procs,
            "r_p": r_p, "r_d": r_d}


def oracle_child(n: int, warmup: int, steps: int, procs: int) -> dict:
    """oracle_pool_iterations in a fresh child process that never touches CUDA."""
    code = ("import json,sys;sys.path.insert(0,%r);import bench;"
            "print(json.dumps(bench.oracle_pool_iterations(%d,%d,%d,%d)))") % (ROOT, n, warmup, steps, procs)
    # one BLAS/FFT thread per process: the processes are the parallelism
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=3600,
                         cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_info():
    """The host the oracle ran on: logical CPUs and the CPU model (from /proc/cpuinfo)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model, "machine": platform.machine()}


def cpu_baseline():
    procs = host_cores()
    r = oracle_child(N, 1, 3, procs)
    v = r["voxels"] * r["iters"] / r["seconds"]
    return {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"ADMM iterations 2-4 of the {N}^3 inclusion cell from the fresh state "
                      f"({r['seconds']:.1f} s; FP64 numpy oracle, Step 1 over {procs} processes, one per host "
                      f"core, Steps 2-4 in one)", "host": host_info()}


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args):
    """The oracle on the host's cores, on the GPU arm's workload (the 128^3 inclusion
    cell): each step is one ADMM iteration, continuing one solve from the fresh state."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    procs = host_cores()
    r = oracle_child(N, args.warmup, args.steps, procs)
    secs, vox = r["seconds"], r["voxels"] * r["iters"]
    v = vox / secs
    sample = (f"each step: one ADMM iteration of the {N}^3 inclusion cell (iterations {args.warmup + 1}-"
              f"{args.warmup + args.steps} of a solve from the fresh state; FP64 numpy oracle, Step 1 over "
              f"{procs} processes, one per host core)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"inclusions{N}", "n": N, "dim": 3},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
                             "host": host_info()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm

def timed_solves(s, steps, torch, phase=None, params=None, pinned_phase=None):
    """K full solves; returns (elapsed_ms by CUDA events on the caller's stream, infos, stresses)."""
    infos, stresses = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        if pinned_phase is not None:
            s.set_material(pinned_phase, params)     # host -> device copy of the inputs
        else:
            s.reset()
        infos.append(s.solve(FBAR, RHO, TOL))
        stresses.append(s.stress())                    # device -> host read of the result
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), infos, stresses


def run_ours(args):
    import torch
    from paper_2010_06697_gb300 import build, rve

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    rve.lib()
    ph, par = make_inputs()
    V = ph.size

    def barrier():
        if dist is not None:
            dist.barrier()


    results = {}
    for prec in ([args.precision] + (["fp64"] if args.precision != "fp64" and not args.quick else [])):
        s = rve.Rve(DIM, N, "neohookean", prec, max_iter=2000, rho_policy=RHO_POLICY)
        s.set_material(ph, par)
        for _ in range(args.warmup):
            s.reset()
            s.solve(FBAR, RHO, TOL)
            s.stress()
        barrier()
        clocks = ClockSampler(local_rank) if prec == args.precision else None
        if clocks:
            clocks.start()
        ms, infos, stresses = timed_solves(s, args.steps, torch)
        if clocks:
            clk = clocks.stop()
        iters = sum(i.iterations for i in infos)
        ms, vox_it = combine_ranks(ms, V * iters, dist, "cuda")
        res = {"ms": ms, "iters_per_step": iters / args.steps, "value": vox_it / (ms / 1e3),
               "converged": all(i.converged for i in infos),
               "fp64_iters_per_step": sum(i.fp64_iterations for i in infos) / args.steps,
               "launches": sum(i.launches for i in infos) + args.steps, "stress": stresses[-1].tolist()}
        if clocks:
            res["clocks"] = clk
        # e2e: the same steps through the public API from pinned host memory
        if prec == args.precision:
            pinned = torch.empty(ph.shape, dtype=torch.uint8, pin_memory=True)
            pinned.copy_(torch.from_numpy(ph))
            barrier()
            ems, einfos, _ = timed_solves(s, args.steps, torch, params=par, pinned_phase=pinned.numpy())
            eiters = sum(i.iterations for i in einfos)
            ems, evox = combine_ranks(ems, V * eiters, dist, "cuda")
            res["e2e"] = {"value": evox / (ems / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": int(V + par.size * 8 + 72), "d2h_bytes_per_step": 72}
            # per-kernel device times (events around every launch, no graphs) for the roofline
            s.set_profiling(True)
            for _ in range(2):
                s.reset()
                s.solve(FBAR, RHO, TOL)
            res["kernels"] = s.kernel_times()
            s.set_profiling(False)
        s.close()
        results[prec] = res
        barrier()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    main = results[args.precision]
    pk = peaks()
    # roofline of the dominant kernel class
    kern = []
    for pname, table in main["kernels"].items():
        sz = 8 if pname == "fp64" else 4
        for cls, (tot, cnt) in table.items():
            if cls in ("local_r", "xfwd_incr", "xinv_incr"):
                sz = 0  # fixed mixed-width byte counts
            per_launch_ms = tot / cnt
            byts = bytes_per_voxel(cls, sz) * V
            kern.append({"kernel": cls, "precision": pname, "total_ms": tot, "launches": cnt,
                         "ms_per_launch": per_launch_ms, "alg_bytes_per_launch": byts,
                         "gbs": byts / (per_launch_ms / 1e3) / 1e9})
    kern.sort(key=lambda k: -k["total_ms"])
    top = kern[0]
    share = top["total_ms"] / sum(k["total_ms"] for k in kern)
    # every kernel of the path is bounded by HBM traffic in the byte model above (the local
    # kernels also by FP32 issue: their Newton work varies per voxel and iteration)
    roof = {"bound": "hbm", "achieved": top["gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": top["gbs"] / pk["hbm_gbs"], "traffic": TRAFFIC.get((top["kernel"], top["precision"])),
            "kernel": f"{top['kernel']} ({top['precision']})", "peak_source": pk["source"],
            "share_of_profiled_time": share}
    fl = FLOPS.get((top["kernel"], top["precision"]))
    if fl:  # the same kernel against the FP32 pipe (its Newton solve is compute-heavy)
        tf = fl / (top["ms_per_launch"] / 1e3) / 1e12
        roof["alu_view"] = {"achieved_tflops": tf, "peak_tflops": FP32_PEAK_TFLOPS, "frac": tf / FP32_PEAK_TFLOPS,
                            "flops_per_launch": fl,
                            "peak_source": "derived: 128 FP32 lanes x 2 x 152 SMs x 2.07 GHz (FMA-chain probe "
                                           "74.8 TFLOP/s at 1995 MHz)"}
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else ("f64" if args.precision == "fp64" else "f32"),
        "data": "synthetic",
        "config": {"workload": "inclusions128", "n": N, "dim": DIM, "model": "neohookean", "seed": SEED,
                   "Fbar": "diag(0.9,1,1)", "rho": RHO, "rho_policy": RHO_POLICY, "tol": TOL,
                   "precision": args.precision,
                   "step": "one full RVE solve from the fresh state", "l2": "inputs larger than L2 "
                   f"(resident state {33 * 4 * V / 1e6:.0f} MB float / {33 * 8 * V / 1e6:.0f} MB double > 129 MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "iters_per_step": main["iters_per_step"], "fp64_iters_per_step": main["fp64_iters_per_step"],
        "converged": main["converged"], "stress_xx": main["stress"][0][0],
        "gpu_launches": main["launches"],
        "clocks": main.get("clocks"),
        "e2e": main["e2e"],
        "roofline": roof,
        "kernels": [{k: (round(v, 6) if isinstance(v, float) else v) for k, v in kk.items()} for kk in kern],
    }
    if "fp64" in results and args.precision != "fp64":
        f = results["fp64"]
        line["fp64"] = {"value": f["value"], "ms_per_step": f["ms"] / args.steps,
                        "iters_per_step": f["iters_per_step"], "converged": f["converged"],
                        "stress_xx": f["stress"][0][0]}
        line["mixed_over_fp64"] = main["value"] / f["value"]
    if world == 1 and not args.no_extra:
        from paper_2010_06697_gb300 import synth
        extra = {}
        for name, fn in other_workloads():
            try:
                extra[name] = fn(torch, rve, synth)
            except Exception as e:  # report, do not lose the main line
                extra[name] = {"error": repr(e)[:300]}
        line["other_workloads"] = extra
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def other_workloads():
    """The workloads reported beside the headline line, as (name, function) pairs."""
    return (("laminate32_2d", bench_laminate32), ("inclusions128_adaptive_rho", bench_adaptive128),
            ("inclusions128_inexact", bench_inexact128),
            ("inclusions128_fraction", lambda t, r, sy: bench_inexact128(t, r, sy, ratio=0.0, fraction=0.9)),
            ("lce256", bench_lce256), ("lce128_pe_path", bench_lce_path128),
            ("lce128_pe_path_inc", lambda t, r, sy: bench_lce_path128(t, r, sy, incompressible=True)),
            ("lce128_pe_path_mixed", lambda t, r, sy: bench_lce_path128(t, r, sy, precision="mixed")),
            ("bloch512_2d", bench_bloch512), ("bloch128_3d", bench_bloch128_3d), ("batch64", bench_batch64),
            ("serving", bench_serving_pair), ("cufft128", bench_cufft128))


def run_workload(args):
    """One of the other workloads alone (for profiler captures); prints its JSON object."""
    import torch
    from paper_2010_06697_gb300 import build, rve, synth
    torch.cuda.set_device(0)
    build.build()
    rve.lib()
    fns = dict(other_workloads())
    # capture-sized variants (profiler runs only)
    fns["bloch512_2d_fixed"] = lambda t, r, sy: bench_bloch512(t, r, sy, to_tolerance=False)
    if args.workload not in fns:
        print(json.dumps({"error": f"unknown workload {args.workload}", "known": sorted(fns)}))
        return 2
    print(json.dumps(fns[args.workload](torch, rve, synth)))
    return 0


def run_single(args):
    import torch
    from paper_2010_06697_gb300 import build, rve
    torch.cuda.set_device(0)
    build.build()
    ph, par = make_inputs()
    s = rve.Rve(DIM, N, "neohookean", args.precision, max_iter=2000, rho_policy=RHO_POLICY)
    s.set_material(ph, par)
    info = s.solve(FBAR, RHO, TOL)
    S = s.stress()
    s.close()
    print(json.dumps({"single": True, "precision": args.precision, "iterations": info.iterations,
                      "fp64_iterations": info.fp64_iterations, "converged": bool(info.converged),
                      "time_ms": info.time_ms, "launches": info.launches, "stress_xx": float(S[0, 0])}))
    return 0 if info.converged else 1


# ------------------------------------------------------------------ the other workloads (extra JSON objects)

def bench_laminate32(torch, rve, synth, iters=300, reps=5):
    """2D 32x32 plane-strain neo-Hookean laminate (mu = 1 | 10, nu = 0.3), Fbar = diag(1.05, 1),
    rho = 10, exactly 300 FP64 iterations: a latency-bound cell (1024 voxels); reports the device
    time per iteration of the whole solve."""
    n = 32
    ph = synth.laminate_phase(n, 2)
    par = synth.two_phase_params(MU[0], MU[1], NU)
    s = rve.Rve(2, n, "neohookean", "fp64", max_iter=iters)
    s.set_material(ph, par)
    Fb = np.diag([1.05, 1.0, 1.0])
    s.solve(Fb, RHO, -1.0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(reps):
        s.reset()
        torch.cuda.synchronize()
        ev0.record()
        info = s.solve(Fb, RHO, -1.0)
        S = s.stress()
        ev1.record()
        torch.cuda.synchronize()
        best = min(best, ev0.elapsed_time(ev1))
    s.close()
    return {"workload": "laminate32_2d", "value": ph.size * iters / (best / 1e3), "unit": UNIT,
            "us_per_iteration": 1e3 * best / iters, "ms": best, "iterations": info.iterations,
            "stress_xx": float(S[0, 0]), "precision": "fp64"}


def bench_cufft128(torch, rve, synth, reps=20):
    """A timed comparison only (cuFFT is not on the solver's path): the library's 3D
    real-to-complex and complex-to-real transforms of the d = 3 displacement fields of
    the 128^3 cell (torch.fft, which calls cuFFT), beside the solver's own Step 2
    passes per iteration from a profiled headline solve, which also compute the
    divergence of F - Lambda/rho and apply the spectral solve.  Inputs rotate over
    buffers larger than L2, as the solver's fields are."""
    n = N
    out = {"workload": "cufft128", "note": "comparison only: cuFFT forward + inverse of 3 real fields per "
                                           "iteration vs the fused Step 2 passes (divergence, FFTs, solve)"}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        nbuf = max(2, int(2 * L2_BYTES // (3 * n ** 3 * (4 if dt == torch.float32 else 8))) + 1)
        xs = [torch.randn(3, n, n, n, device="cuda", dtype=dt) for _ in range(nbuf)]
        for x in xs[:3]:
            torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=(n, n, n), dim=(1, 2, 3))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for i in range(reps):
            y = torch.fft.irfftn(torch.fft.rfftn(xs[i % nbuf], dim=(1, 2, 3)), s=(n, n, n), dim=(1, 2, 3))
        ev1.record()
        torch.cuda.synchronize()
        out[f"cufft_{name}_us_per_iteration"] = 1e3 * ev0.elapsed_time(ev1) / reps
        del xs, y
    torch.cuda.empty_cache()
    ph, par = make_inputs(n)
    for prec, key in (("fp32", "mixed"), ("fp64", "fp64")):
        s = rve.Rve(DIM, n, "neohookean", key, max_iter=2000)
        s.set_material(ph, par)
        s.set_profiling(1)
        s.solve(FBAR, RHO, TOL)
        kt = s.kernel_times()[prec]
        s.close()
        cls = ("xfwd", "fwd_y", "solve", "inv_y", "xinv")
        out[f"solver_{prec}_us_per_iteration"] = sum(1e3 * kt[c][0] / kt[c][1] for c in cls if c in kt)
        out[f"solver_{prec}_passes_us"] = {c: round(1e3 * kt[c][0] / kt[c][1], 2) for c in cls if c in kt}
    return out


def bench_inexact128(torch, rve, synth, ratio=0.3, fraction=0.0, reps=3):
    """The headline cell (128^3 inclusions, mixed precision, tol 1e-8) with inexact local
    steps: r_l <= ratio r_d (Section 4.2's adopted strategy) or, with fraction > 0, the
    fraction-converged strategy; device time per solve, iterations and the stress, for
    comparison with the exact-local line."""
    ph, par = make_inputs()
    s = rve.Rve(DIM, N, "neohookean", "mixed", max_iter=2000, local_ratio=ratio, local_fraction=fraction)
    s.set_material(ph, par)
    s.solve(FBAR, RHO, TOL)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, info, S = 1e30, None, None
    for _ in range(reps):
        s.reset()
        torch.cuda.synchronize()
        ev0.record()
        info = s.solve(FBAR, RHO, TOL)
        S = s.stress()
        ev1.record()
        torch.cuda.synchronize()
        best = min(best, ev0.elapsed_time(ev1))
    s.close()
    return {"workload": "inclusions128_inexact", "local_ratio": ratio, "local_fraction": fraction,
            "value": ph.size * info.iterations / (best / 1e3), "unit": UNIT, "ms": best,
            "iterations": info.iterations, "fp64_iterations": info.fp64_iterations,
            "converged": bool(info.converged), "stress_xx": float(S[0, 0]), "precision": "mixed"}


def bench_adaptive128(torch, rve, synth, reps=3):
    """The headline cell and tolerance with Section 2.1's adaptive penalty from rho = 10
    (mixed; the rule acts in the float bulk, rho stays fixed through the double polish):
    fewer iterations per solve; reports the time per solve beside the fixed-rho headline."""
    ph, par = make_inputs()
    s = rve.Rve(DIM, N, "neohookean", "mixed", max_iter=2000, rho_policy="adaptive")
    s.set_material(ph, par)
    s.solve(FBAR, RHO, TOL)
    best, info = None, None
    for _ in range(reps):
        s.reset()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        info = s.solve(FBAR, RHO, TOL)
        S = s.stress()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        best = ms if best is None else min(best, ms)
    s.close()
    return {"workload": "inclusions128_adaptive_rho", "value": ph.size * info.iterations / (best / 1e3), "unit": UNIT,
            "ms_per_solve": best, "iterations": info.iterations, "fp64_iterations": info.fp64_iterations,
            "final_rho": info.rho, "converged": bool(info.converged), "stress_xx": float(S[0, 0])}


def bench_lce256(torch, rve, synth, iters=40):
    """3D 256^3 LCE polydomain (Section 5.1 readings): one phase mu = 1, lam = 20, r = 7.71,
    alpha = 0.06, wall length 2h; directors from a Gaussian random field (correlation 8
    voxels); Fbar = diag(1.2, 0.91, 0.91); mixed precision; fixed iteration count (the
    relaxation plateaus instead of reaching a tolerance)."""
    n = 256
    n0 = synth.director_grf(n, 0, corr=8.0)
    ph = np.zeros((n,) * 3, np.uint8)
    par = np.array([[1.0, 20.0, 7.71, 0.06, (2.0 / n) ** 2]])
    Fb = np.diag([1.2, 0.91, 0.91])
    s = rve.Rve(3, n, "lce", "mixed", max_iter=iters)
    s.set_material(ph, par, n0)
    s.solve(Fb, RHO, -1.0)
    s.reset()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    info = s.solve(Fb, RHO, -1.0)
    S = s.stress()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    s.close()
    # the same 40 iterations in plain FP64: the mixed result's stress error (untimed)
    s64 = rve.Rve(3, n, "lce", "fp64", max_iter=iters)
    s64.set_material(ph, par, n0)
    s64.solve(Fb, RHO, -1.0)
    S64 = s64.stress()
    s64.close()
    err = float(np.max(np.abs(S - S64)) / np.max(np.abs(S64)))
    return {"workload": "lce256", "value": ph.size * info.iterations / (ms / 1e3), "unit": UNIT,
            "ms": ms, "iterations": info.iterations, "fp64_iterations": info.fp64_iterations,
            "r_p": info.r_p, "r_d": info.r_d, "stress_xx": float(S[0, 0]), "precision": "mixed",
            "stress_rel_err_vs_fp64": err}


def bench_lce_path128(torch, rve, synth, incompressible=False, steps=5, iters=30, precision="fp64"):
    """3D 128^3 LCE polydomain under a plane-strain loading path with dissipation
    (Section 5.3): <F_11> = 1.02, 1.04, ..., <F_12> = 0, <F_22> = 1, the other components
    free (mixed control); one time step per load step with nu_F/(mu dt) = 5.6,
    nu_n/(mu dt) = 0.0106; r = 7.71, alpha = 0.06, wall length 2h, directors from a
    Gaussian random field (correlation 8 voxels); FP64 (or the mixed scheme); a fixed
    iteration count per step.  incompressible: the network with det F = 1 by the local
    multiplier."""
    n = 128
    n0 = synth.director_grf(n, 0, corr=8.0)
    ph = np.zeros((n,) * 3, np.uint8)
    par = np.array([[1.0, 20.0, 7.71, 0.06, (2.0 / n) ** 2, 5.6, 0.0106, 1.0 if incompressible else 0.0]])
    free = np.ones((3, 3), bool)
    free[0, 0] = free[0, 1] = free[1, 1] = False
    Fbars = np.stack([np.diag([1.0 + 0.02 * (k + 1), 1.0, 1.0]) for k in range(steps)])
    s = rve.Rve(3, n, "lce", precision, max_iter=iters)
    s.set_material(ph, par, n0)
    s.solve_path(Fbars[:1], RHO, -1.0, free=free)  # warm-up (kernels, graphs)
    s.set_material(ph, par, n0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    S, Fo, infos = s.solve_path(Fbars, RHO, -1.0, free=free)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    its = sum(i.iterations for i in infos)
    s.close()
    return {"workload": "lce128_pe_path" + ("_inc" if incompressible else "") + ("_mixed" if precision != "fp64" else ""),
            "value": ph.size * its / (ms / 1e3),
            "unit": UNIT, "ms": ms, "load_steps": steps, "iterations": its, "precision": precision,
            "S11": [float(x[0, 0]) for x in S], "F33": [float(x[2, 2]) for x in Fo],
            "r_p_last": infos[-1].r_p, "r_d_last": infos[-1].r_d}


def bench_bloch512(torch, rve, synth, iters=400, to_tolerance=True):
    """2D 512^2 modulus of stability beta_(2,2) (Section 2.4 with Section 4.3's example):
    one centred soft disc of radius 0.4, mu_m / mu_i = 20, kappa / mu = 9.8 in both phases,
    equi-biaxial compression <F> = 0.94 I solved to 1e-9 (FP64), then the Bloch-wave ADMM
    (FP64, rho = 200) for a fixed iteration count, timed on the device."""
    n = 512
    ph = synth.disc_phase(n, 2, 0.4)
    par = np.array([[20.0, 196.0], [1.0, 9.8]])
    s = rve.Rve(2, n, "neohookean", "fp64", max_iter=20000)
    s.set_material(ph, par)
    si = s.solve(np.diag([0.94, 0.94, 1.0]), 30.0, 1e-9)
    s.bloch((2, 2), 200.0, -1.0, 20, seed=0)  # warm-up (kernels, graphs)
    bi, _, hist = s.bloch((2, 2), 200.0, -1.0, iters, seed=0)
    # time to beta: the same cell to tol 1e-8 with Section 2.1's adaptive penalty from rho = 200,
    # in FP64 and with the float bulk (RVE_MIXED)
    Fres = s.get_field(rve.RVE_FIELD_F)
    s.close()
    tt = {}
    for prec in (("fp64", "mixed") if to_tolerance else ()):
        s2 = rve.Rve(2, n, "neohookean", prec, max_iter=10, rho_policy="adaptive")
        s2.set_material(ph, par)
        s2.set_field(rve.RVE_FIELD_F, Fres)
        ci, _, _ = s2.bloch((2, 2), 200.0, 1e-8, 40000, seed=0)
        s2.close()
        tt[prec] = {"converged": bool(ci.converged), "iterations": ci.iterations,
                    "float_iterations": ci.float_iterations, "ms": ci.time_ms, "beta22": ci.beta,
                    "rayleigh": ci.rayleigh, "final_rho": ci.rho}
    return {"workload": "bloch512_2d", "value": ph.size * bi.iterations / (bi.time_ms / 1e3), "unit": UNIT,
            "ms_per_iteration": bi.time_ms / bi.iterations, "iterations": bi.iterations, "launches": bi.launches,
            "beta22": bi.beta, "rayleigh": bi.rayleigh, "r_p": bi.r_p, "r_d": bi.r_d, "precision": "fp64",
            "equilibrium_iterations": si.iterations, "equilibrium_converged": bool(si.converged),
            "to_tolerance": {"tol": 1e-8, "rho_policy": "adaptive", **tt}}


def bench_bloch128_3d(torch, rve, synth, iters=100):
    """3D 128^3 modulus of stability beta_(2,2,2): the 128^3 inclusion cell of the headline
    (matrix mu = 1, spherical inclusions mu = 10, nu = 0.3) compressed to <F> = 0.95 I and
    solved to 1e-8 (mixed), then the Bloch-wave ADMM (rho = 40) for a fixed iteration
    count, timed on the device: in FP64, and with the float bulk (RVE_MIXED, whose
    iterations here stay in the float phase)."""
    n = 128
    ph = synth.inclusion_phase(n, 3, 0, radius=6)
    par = synth.two_phase_params(1.0, 10.0)
    s = rve.Rve(3, n, "neohookean", "mixed", max_iter=4000)
    s.set_material(ph, par)
    si = s.solve(np.diag([0.95, 0.95, 0.95]), RHO, 1e-8)
    F = s.get_field(rve.RVE_FIELD_F)
    s.close()
    out = {}
    for prec in ("fp64", "mixed"):
        b = rve.Rve(3, n, "neohookean", prec, max_iter=10)
        b.set_material(ph, par)
        b.set_field(rve.RVE_FIELD_F, F)
        b.bloch((2, 2, 2), 40.0, -1.0, 10, seed=0)  # warm-up (kernels, graphs)
        bi, _, _ = b.bloch((2, 2, 2), 40.0, -1.0, iters, seed=0)
        b.close()
        out[prec] = bi
    f = out["fp64"]
    m = out["mixed"]
    return {"workload": "bloch128_3d", "value": ph.size * f.iterations / (f.time_ms / 1e3), "unit": UNIT,
            "ms_per_iteration": f.time_ms / f.iterations, "iterations": f.iterations, "launches": f.launches,
            "beta222": f.beta, "r_p": f.r_p, "r_d": f.r_d, "precision": "fp64",
            "mixed": {"value": ph.size * m.iterations / (m.time_ms / 1e3), "ms_per_iteration": m.time_ms / m.iterations,
                      "iterations": m.iterations, "float_iterations": m.float_iterations, "beta222": m.beta},
            "equilibrium_iterations": si.iterations, "equilibrium_converged": bool(si.converged)}


def bench_batch64(torch, rve, synth, count=64):
    """64 RVEs, N uniform over {32, 48, 64, 96, 128}^3, laminate / inclusion by seed parity,
    Fbar = I + sym(E) with |E_ij| <= 0.1, tol 1e-8, mixed precision, FFT geometry tuned per
    N; one batched solve (one persistent launch per pass) against the members solved alone."""
    spec = synth.batch_spec(count, 0)
    par = synth.two_phase_params(MU[0], MU[1], NU)
    tuned = {}
    for n in sorted({m["n"] for m in spec}):
        tuned[n] = rve.rve_autotune(3, n, "mixed")

    def make():
        out = []
        for m in spec:
            ph = synth.laminate_phase(m["n"], 3) if m["kind"] == "laminate" else synth.inclusion_phase(m["n"], 3, m["seed"])
            h = rve.Rve(3, m["n"], "neohookean", "mixed", max_iter=1000)
            h.set_material(ph, par)
            out.append(h)
        return out

    Fb = np.stack([m["Fbar"] for m in spec])
    rhos = np.full(count, RHO)
    hs = make()
    b = rve.Batch(hs)
    b.solve(Fb, rhos, TOL)                  # warm-up: graphs, tile tables
    for h in hs:
        h.reset()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    infos = b.solve(Fb, rhos, TOL)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    vox_it = sum(h.n ** 3 * i.iterations for h, i in zip(hs, infos))
    # the same members one after the other
    for h in hs:
        h.reset()
    torch.cuda.synchronize()
    ev0.record()
    for h, F in zip(hs, Fb):
        h.solve(F, RHO, TOL)
    ev1.record()
    torch.cuda.synchronize()
    ms_seq = ev0.elapsed_time(ev1)
    b.close()
    for h in hs:
        h.close()
    return {"workload": "batch64", "value": vox_it / (ms / 1e3), "unit": UNIT, "ms": ms,
            "sequential_ms": ms_seq, "batch_speedup": ms_seq / ms, "voxels": int(sum(m["n"] ** 3 for m in spec)),
            "converged": int(sum(i.converged for i in infos)), "count": count,
            "mean_iterations": float(np.mean([i.iterations for i in infos])), "fft_tuned_ms": tuned,
            "precision": "mixed"}


# LCE serving requests are one implicit time step (Section 5.1's dissipation, R27):
# nu_F / (mu dt) = 20, i.e. Section 5.3's network viscosity with a step of 0.0056 s (a
# quarter of its 0.02 s), and the same value for the director.  At Section 5.3's own values
# (5.6 and 0.0106) the director field of the larger polydomain cells keeps relaxing for
# more than 1000 iterations; at 20 every request reaches the tolerance in 45-75 iterations.
SERVE_LCE_VISC = 20.0


def serving_inputs(synth, stream):
    par = synth.two_phase_params(MU[0], MU[1], NU)
    inputs = []
    for r in stream:
        n = r["n"]
        if r["kind"] == "lce":
            inputs.append(dict(phase=np.zeros((n,) * 3, np.uint8), n0=synth.director_grf(n, r["seed"], corr=8.0),
                               params=np.array([[1.0, 20.0, 7.71, 0.06, (2.0 / n) ** 2, SERVE_LCE_VISC,
                                                 SERVE_LCE_VISC]]), model="lce"))
        else:
            ph = synth.laminate_phase(n, 3) if r["kind"] == "laminate" else synth.inclusion_phase(n, 3, r["seed"])
            inputs.append(dict(phase=ph, n0=None, params=par, model="neohookean"))
    return inputs


def bench_serving(torch, rve, synth, count=200, rate=200.0, inputs=None, stream=None):
    """Poisson arrivals of RVE solve requests (200 requests; mean rate `rate`): N log-uniform
    over even 2^a 3^b in [32, 256], laminate / inclusion / LCE 40/40/20 (LCE: one time step
    with dissipation), Fbar = I + sym(E) with |E_ij| <= 0.1, tol 1e-6, at most 400 iterations,
    mixed precision, admission by a 120 GB device budget.  At 200/s the arrivals outrun the
    GPU (a burst): ``value`` is then the saturation throughput and the latencies include the
    queue; serving_sustained replays the stream at a rate the GPU keeps up with."""
    if stream is None:
        stream = synth.serving_stream(count, 0, rate_hz=rate)
        inputs = serving_inputs(synth, stream)
    tol, max_iter = 1e-6, 400
    srv = rve.Server(120 << 30, "mixed", max_iter=max_iter, check_every=8)
    for i in range(2):                           # warm-up requests (graphs, modules)
        t = srv.submit(inputs[i]["phase"], inputs[i]["params"], stream[i]["Fbar"], RHO, tol, inputs[i]["model"],
                       inputs[i]["n0"])
        while srv.poll(t) is None:
            srv.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets, results, nxt = {}, {}, 0
    while len(results) < count:
        now = time.perf_counter() - t0
        while nxt < count and stream[nxt]["t"] <= now:
            inp = inputs[nxt]
            tickets[nxt] = srv.submit(inp["phase"], inp["params"], stream[nxt]["Fbar"], RHO, tol, inp["model"],
                                      inp["n0"])
            nxt += 1
        srv.step()
        for i, t in list(tickets.items()):
            if i not in results:
                out = srv.poll(t)
                if out is not None:
                    results[i] = out
    wall = time.perf_counter() - t0
    lat = np.array([results[i][3] for i in range(count)])
    vox_it = sum(stream[i]["n"] ** 3 * results[i][2].iterations for i in range(count))
    srv.close()
    kinds = [r["kind"] for r in stream]
    conv = {k: int(sum(results[i][2].converged for i in range(count) if kinds[i] == k)) for k in set(kinds)}
    return {"workload": "serving", "value": vox_it / wall, "unit": UNIT, "requests": count,
            "rate_hz": float(count / stream[-1]["t"]) if stream[-1]["t"] > 0 else rate,
            "requests_per_s_completed": count / wall, "wall_s": wall,
            "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
            "converged": int(sum(results[i][2].converged for i in range(count))), "converged_by_kind": conv,
            "kinds": {k: kinds.count(k) for k in set(kinds)}, "precision": "mixed",
            "mean_iterations": float(np.mean([results[i][2].iterations for i in range(count)])),
            "mean_voxels": float(np.mean([r["n"] ** 3 for r in stream])),
            "arrival_span_s": float(stream[-1]["t"]),
            "mean_queue_ms": float(np.mean([results[i][4] for i in range(count)])),
            "note": "latency = queue wait (admission by device memory) + solve; see mean_queue_ms"}


def bench_serving_pair(torch, rve, synth, count=200):
    """The 200/s burst (saturation throughput), then the same 200 requests replayed at 70 %
    of the request rate the GPU completed in the burst (the highest sustainable rate, with
    margin): arrival times scaled, sizes, kinds and loads unchanged."""
    stream = synth.serving_stream(count, 0, rate_hz=200.0)
    inputs = serving_inputs(synth, stream)
    burst = bench_serving(torch, rve, synth, count, 200.0, inputs, stream)
    rate = 0.7 * burst["requests_per_s_completed"]
    scale = 200.0 / rate
    slow = [dict(r, t=r["t"] * scale) for r in stream]
    sustained = bench_serving(torch, rve, synth, count, rate, inputs, slow)
    sustained["workload"] = "serving_sustained"
    burst["sustained"] = sustained
    return burst


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the fp64 comparison run")
    ap.add_argument("--no-extra", action="store_true", help="skip the LCE, batch and serving workloads")
    ap.add_argument("--single", action="store_true",
                    help="one solve of the workload (for profiler captures), prints a short summary")
    ap.add_argument("--workload", default=None,
                    help="run one of the other workloads alone (for profiler captures) and print its JSON")
    args = ap.parse_args()
    if args.single:
        return run_single(args)
    if args.workload:
        return run_workload(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
