#!/usr/bin/env python
"""Benchmark of the SWR hot path on the scaling workload (one GB300 per rank).

One step = one complete SWR solve of the scaling workload for every subdomain
count N in {16, 64, 256, 500}: 200001 P1 nodes on (-50, 50), 500 Crank-Nicolson
steps (dt = 1e-3), seeded Gaussian-well potential and Gaussian packets, Robin
transmission p = sqrt(5) exp(-i pi/4).  Each solve is swr_build_interface
(assembly, factorisation, d and the Toeplitz columns by marches) followed by
swr_solve (right-preconditioned GMRES(30) on (I - L) g = d to an absolute
residual of 1e-10, then u(T) by superposition of the impulse responses' states
recorded during the build).

Reported: point-steps/s of all marches in the step (whole job), the solve time
per step, the roofline of the march kernel (FP64-ALU bound), the CPU oracle's
march throughput on the host CPU, and an end-to-end figure with host buffers.
Multi-GPU runs (torchrun) are replicas: every rank solves its own copy.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NSUBS = (16, 64, 256, 500)
FLOPS_PER_POINT_STEP = 36          # Thomas with stored factors, per node and time step
FLOPS_PER_POINT_STEP_TDEP = 56     # plus the per-step factorisation (one complex reciprocal)
# nonlinear march, per node and inner fixed-point iteration: the linear solve with stored
# factors (36) plus the generalised-mass term b_f(zeta) (30) and the convergence test (10)
FLOPS_PER_POINT_ITER_NL = 76
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07   # SMs x FP64 FMA/clk x 2 flop x GHz (max SM clock)

# DRAM bytes (read + write) per march launch, each scaled by the steps from 100-step
# single-launch ncu captures (profiles/k_march_static_N500_build.md, launch_list_scaling.md,
# launch_list_timedep.md).  Scaling step: the mean over its four build marches, the N = 500
# build (lean k_march_static<12>: 19.1 MB read, 593.5 MB written per 100 steps, the recorded
# states) standing for N = 256 and the N = 16 build (k_march_tl<12>: 19.2 / 547.0 MB) for
# N = 64.  V(t,x) march: the streamed per-step factors, 677.2 MB read and 0.3 MB written per
# 100 steps (captured on k_march_static's general instantiation in the modelled cluster
# shape, whose code the later k_march_tl changes did not touch; the lean one of the tuned
# shape streams the same factors, 7.1 MB per step in its 38-step probes).  Valid only for
# the march sources they were taken from (sha256 prefix of swr_march.cu +
# swr_internal.cuh), null otherwise.
MARCH_TRAFFIC = {"sources": "647131b39d98daf0",
                 "scaling": 2947000000.0, "timedep": 6775000000.0}


def march_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("swr_march.cu", "swr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1503_02564_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="swr", choices=["swr", "reference"])
    ap.add_argument("--nsub", default=",".join(str(n) for n in NSUBS))
    ap.add_argument("--precond", default="causal", choices=["causal", "none"])
    ap.add_argument("--workload", default="scaling",
                    choices=["scaling", "timedep", "adjoint", "batch", "nonlinear", "tcs",
                             "fp64peak"],
                    help="scaling: the N in {16,64,256,500} static-potential step (default); "
                         "timedep: the time-dependent potential case (60001 nodes, 1000 steps, "
                         "N = 64, GMRES preconditioned by the mean-potential operator); "
                         "adjoint: the scaling step plus the misfit gradient dJ/dV by "
                         "swr_adjoint (every step recorded when it fits, else checkpoints "
                         "every 50); batch: 128 independent "
                         "instances (uneven partitions, 100-400 steps) in one batched plan, "
                         "reported beside one plan per instance; nonlinear: |u|^2 + V0 "
                         "(20001 nodes, 1000 steps, N = 32), preconditioned fixed point, then "
                         "the misfit gradient dJ/dV0 by swr_adjoint (the library's checkpoint "
                         "interval); "
                         "tcs: the comparison of transmission conditions and interface solvers "
                         "in the setting of the paper's Section 6 (V=-x^2 on (-21,21), dx=1e-5, "
                         "N in {2,500}, random g0); fp64peak: the FP64 throughput probes "
                         "(DFMA and DMMA m8n8k4), each timed for >= 1 s with clocks sampled")
    ap.add_argument("--tc", default="robin", choices=["robin", "s02"],
                    help="transmission condition of the scaling workload: Robin "
                         "p = sqrt(5) e^{-i pi/4} (default) or the order-2 potential "
                         "strategy S_0^2")
    ap.add_argument("--pc-sweeps", type=int, default=-1,
                    help="block-Jacobi sweeps of the causal preconditioner's same-step "
                         "coupling (-1: the library's choice)")
    ap.add_argument("--nt", type=int, default=0,
                    help="override the workload's number of time steps (smaller cases for "
                         "profiling; 0: the workload's own)")
    ap.add_argument("--tcs-nx", type=int, default=84001,
                    help="nodes of the tcs workload on (-21, 21): 84001 is dx = 5e-4; the "
                         "paper's dx = 1e-5 (4200001 nodes) needs 2.1M-node subdomains at N = 2, "
                         "beyond the 69632-node subdomain limit of the march")
    ap.add_argument("--tune", default="",
                    help="execution choices of the plans (swr_tuning fields), e.g. "
                         "'autotune=-1,chunk_L=12' (profiling with a fixed launch shape)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="scaling workload: skip the sub-records of the other workloads "
                         "(plain, batch, time-dependent, nonlinear + gradient)")
    ap.add_argument("--sub-steps", type=int, default=2)
    ap.add_argument("--sub-warmup", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def tuning_of(args):
    """The --tune option as a dict for swr.Plan(tuning=...) (None: library defaults)."""
    if not getattr(args, "tune", ""):
        return None
    out = {}
    for kv in args.tune.split(","):
        k, v = kv.split("=")
        out[k.strip()] = int(v)
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replicas_max_ms(t_ms, dev=None):
    """Replicas (torchrun, one rank per GPU, each solving its own copy): the
    job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_ms
    t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, t_ms):
    """Units all ranks processed per second of the slowest rank's time."""
    return units_per_rank_step * steps * world / (t_ms * 1e-3)


def workload_name(nsubs, tc="robin", nt=500):
    tcs = ("S_0^2 c2=e^{-i pi/4}sqrt(2/dt)" if tc == "s02" else "Robin p=sqrt(5)e^{-i pi/4}")
    return ("swr_scaling: x in (-50,50), 200001 P1 nodes, T=%g dt=1e-3 (%d steps), "
            "N in {%s}, V=-5*sum of 8 seeded Gaussians, u0=4 seeded packets, "
            "%s, build interface + GMRES(30) to 1e-10 + u(T) by superposition"
            % (nt * 1e-3, nt, ",".join(str(n) for n in nsubs), tcs))


def workload_name_timedep(nt=1000):
    return ("swr_timedep: x in (-30,30), 60001 P1 nodes, T=%g dt=1e-3 (%d steps), N=64, " % (nt * 1e-3, nt) +
            "V=-x^2/4(1+0.5 sin 4t)-10exp(-(x-5 sin t)^2), seeded packet, Robin "
            "p=sqrt(5)e^{-i pi/4}, d = R0 + GMRES(60) on g - Rg + d preconditioned by the "
            "mean-potential interface operator to 1e-10 + final march")


def workload_name_nonlinear(nt=1000):
    return ("swr_nonlinear: x in (-20,20), 20001 P1 nodes, T=%g dt=5e-4 (%d steps), N=32, "
            "V=|u|^2+V0, V0=-sum of 6 seeded Gaussian wells (depth 2-10), u0=sech(x)e^{2ix}, "
            "Robin p=sqrt(5)e^{-i pi/4}, inner fixed point to 1e-13 per step, outer fixed point "
            "preconditioned by the V0 interface operator to 1e-10 + final march (recording "
            "v_n of every step when it fits); then J = ||u(T) - u_target||_M^2 and dJ/dV0 by "
            "swr_adjoint (monodomain discrete adjoint about the recorded v_n, one segment)"
            % (nt * 5e-4, nt))


def march_point_steps(wl):
    """Point-steps of the marches of one solve with a final march: per subdomain
    the d march, the impulse marches (one per existing neighbour) and the final
    march.  The reported value uses the library's own count of the marches that
    ran (no final march when u(T) is superposed)."""
    off = wl.off
    N = wl.nsub
    tot = 0
    for j in range(N):
        n = int(off[j + 1] - off[j] + 1)
        marches = 1 + (1 if j > 0 else 0) + (1 if j < N - 1 else 0) + 1
        tot += marches * n * wl.nt
    return tot


def host_info(threads_used=1):
    """The host the CPU oracle is timed on: logical CPUs and the CPU model."""
    import platform
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model, "threads_used": threads_used}


def march_point_steps_d(wl):
    """Point-steps of one d march of every subdomain."""
    return sum(int(wl.off[j + 1] - wl.off[j] + 1) * wl.nt for j in range(wl.nsub))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"swr_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
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
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(wl_full, nsub_sample, min_seconds=0.0, max_passes=20):
    """Time the CPU oracle's subdomain marches (interface operator R applied to
    zero fluxes, i.e. the d march of every subdomain) on the first nsub_sample
    subdomains of the workload, in passes repeated until min_seconds have
    elapsed (at most max_passes).  Returns (point-steps/s, seconds, point-steps)."""
    import numpy as np
    import oracle as O
    P = O.Problem(wl_full.a0, wl_full.b0, wl_full.nx, wl_full.dt, wl_full.nt,
                  wl_full.off.astype(np.int64), wl_full.u0, wl_full.V, vkind=wl_full.vkind,
                  tc=wl_full.tc, sigma=wl_full.sigma)
    t0 = time.perf_counter()
    ps = 0
    N = P.nsub
    for _ in range(max_passes):
        for j in range(nsub_sample):
            a, b = int(P.off[j]), int(P.off[j + 1])
            l = np.zeros(P.nt, np.complex128) if j > 0 else None
            r = np.zeros(P.nt, np.complex128) if j < N - 1 else None
            O.sub_march(P, j, P.u0[a:b + 1], l, r)
            ps += (b - a + 1) * P.nt
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    return ps / dt, dt, ps


def cpu_oracle_marches(wl_full, threads, min_seconds=0.0, max_passes=50):
    """The oracle's subdomain d-marches (R applied to zero fluxes) of every subdomain of
    the workload, one march per task on `threads` host threads (the oracle's C march
    releases the interpreter lock), passes repeated until min_seconds have elapsed.
    Returns (point-steps/s, seconds, point-steps)."""
    import concurrent.futures
    import numpy as np
    import oracle as O
    P = O.Problem(wl_full.a0, wl_full.b0, wl_full.nx, wl_full.dt, wl_full.nt,
                  wl_full.off.astype(np.int64), wl_full.u0, wl_full.V, vkind=wl_full.vkind,
                  tc=wl_full.tc, sigma=wl_full.sigma)
    N = P.nsub

    def one(j):
        a, b = int(P.off[j]), int(P.off[j + 1])
        l = np.zeros(P.nt, np.complex128) if j > 0 else None
        r = np.zeros(P.nt, np.complex128) if j < N - 1 else None
        O.sub_march(P, j, P.u0[a:b + 1], l, r)
        return (b - a + 1) * P.nt

    ps = 0
    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        for _ in range(max_passes):
            ps += sum(ex.map(one, range(N)))
            if time.perf_counter() - t0 >= min_seconds:
                break
        dt = time.perf_counter() - t0
    return ps / dt, dt, ps


def cpu_oracle_adjoint_sample(wl_full, nt_sample):
    """Time the oracle's discrete adjoint (monodomain forward march keeping every
    v_n, then the adjoint solves) on the workload's grid for nt_sample steps.
    Returns (point-steps/s, seconds, point-steps) with 2 x nodes x steps."""
    import numpy as np
    import oracle as O
    from paper_1503_02564_gb300 import workloads as W
    P = O.Problem(wl_full.a0, wl_full.b0, wl_full.nx, wl_full.dt, nt_sample,
                  wl_full.off.astype(np.int64), wl_full.u0, wl_full.V, vkind=wl_full.vkind,
                  tc=wl_full.tc, sigma=wl_full.sigma)
    t0 = time.perf_counter()
    O.adjoint_gradient(P, W.misfit_target(wl_full))
    dt = time.perf_counter() - t0
    ps = 2 * P.nx * nt_sample
    return ps / dt, dt, ps


def cpu_oracle_adjoint_nl_sample(wl_full, nt_sample):
    """Time the oracle's discrete adjoint of the nonlinear monodomain scheme
    (forward march with the inner fixed points, then the exact linearised
    adjoint solves) on the workload's grid for nt_sample steps.  Returns
    (point-steps/s, seconds, point-steps) with 2 x nodes x steps."""
    import numpy as np
    import oracle as O
    from paper_1503_02564_gb300 import workloads as W
    P = O.Problem(wl_full.a0, wl_full.b0, wl_full.nx, wl_full.dt, nt_sample,
                  wl_full.off.astype(np.int64), wl_full.u0, wl_full.V, vkind=wl_full.vkind,
                  tc=wl_full.tc, sigma=wl_full.sigma, nl_coef=wl_full.nl_coef, nl_tol=1e-13,
                  nl_maxit=50)
    t0 = time.perf_counter()
    O.adjoint_gradient_nl(P, W.misfit_target(wl_full))
    dt = time.perf_counter() - t0
    ps = 2 * P.nx * nt_sample
    return ps / dt, dt, ps


def fp64_probe(kind, seconds, dev, sampler=None):
    """Run the library's FP64 throughput probe (kind 0: DFMA, 1: DMMA m8n8k4) for about
    `seconds` of device time after a calibration launch; returns (GFLOP/s, ms, clocks)."""
    import torch
    from paper_1503_02564_gb300 import swr
    blocks, threads = 152 * 4, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    iters = 2000
    swr.swr_fp64_peak(kind, iters, blocks, threads, sink)            # warm-up
    flops, ms = swr.swr_fp64_peak(kind, iters, blocks, threads, sink)
    iters = max(iters, int(iters * seconds * 1e3 / max(ms, 1e-3)))
    if sampler is not None:
        sampler.start()
    flops, ms = swr.swr_fp64_peak(kind, iters, blocks, threads, sink)
    clocks = sampler.stop() if sampler is not None else None
    if not torch.isfinite(sink).all():
        raise RuntimeError("FP64 probe produced non-finite values")
    return flops / (ms * 1e-3) / 1e9, ms, clocks


def run_fp64peak(args):
    """FP64 DFMA and DMMA throughput on this GPU, each timed for >= 1 s with the SM
    clock sampled during the launch (time x median MHz reported beside each)."""
    import torch
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    out = {}
    for kind, name in ((0, "dfma"), (1, "dmma_m8n8k4"), (2, "dfma_and_dmma_together")):
        gf, ms, clocks = fp64_probe(kind, 1.5, dev, ClockSampler(local))
        out[name] = {"gflops": gf, "ms": ms, "clocks": clocks,
                     "ms_x_median_mhz": ms * clocks["sm_mhz"] if clocks else None,
                     "gflops_per_ghz": gf / (clocks["sm_mhz"] * 1e-3) if clocks else None}
    line = {"metric": "FP64 throughput (DFMA vector pipe and DMMA m8n8k4 tensor path)",
            "value": out["dfma"]["gflops"], "unit": "GFLOP/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fp64peak: 608 CTAs x 256 threads, >= 1 s per probe",
                       "dfma": "8 independent fma chains per thread",
                       "dmma": "4 independent m8n8k4 accumulator tiles per warp"},
            "probes": out,
            "nominal_dfma_gflops_at_max_clock": FP64_PEAK_GFLOPS}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_1503_02564_gb300 import workloads as W
    wl = W.config2(nsub=500)
    if args.tc == "s02":
        wl.tc = 1
    # each step: 25 of the 500 subdomain marches (about 5e6 point-steps)
    for _ in range(args.warmup):
        cpu_oracle_sample(wl, 25)
    tot_ps, tot_s = 0, 0.0
    for _ in range(args.steps):
        _, s, ps = cpu_oracle_sample(wl, 25)
        tot_ps += ps
        tot_s += s
    value = tot_ps / tot_s
    line = {
        "impl": "reference", "metric": "SWR subdomain CN point-steps/s (solve time to 1e-10 "
        "interface residual reported as ms_per_step)", "value": value, "unit": "point-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(NSUBS, args.tc),
                   "sample": "oracle d-marches of subdomains 0..24 of N=500 per step"},
        "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": 1, "kind": "oracle", "host": host_info(),
                         "sample": "25 of 500 subdomain marches (401 nodes x 500 steps each)"},
        "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, peak=None):
    """128 independent instances of the batch workload: one batched plan (every
    launch covers all instances) against one plan per instance, same solver.
    Returns the JSON record."""
    import numpy as np
    import torch
    from paper_1503_02564_gb300 import swr
    from paper_1503_02564_gb300 import workloads as W
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if peak is None:
        pg, pms, pclk = fp64_probe(0, 1.5, dev, ClockSampler(local))
        peak = (pg, "measured FP64 DFMA rate of this GPU (swr_fp64_peak, %.0f ms, median SM "
                    "%s MHz)" % (pms, pclk["sm_mhz"] if pclk else "?"))
    wls = W.config3()
    shared = dict(p=wls[0].sigma, restart=30, maxit=2000, tol_abs=1e-10,
                  precond=swr.SWR_PC_CAUSAL)
    insts = [dict(nx=w.nx, a0=w.a0, b0=w.b0, nt=w.nt, nsub=w.nsub, node_off=w.off) for w in wls]
    plan = swr.BatchPlan(insts, dt=wls[0].dt, **shared)
    V = torch.tensor(np.concatenate([w.V for w in wls]), dtype=torch.float64, device=dev)
    u0 = torch.tensor(np.concatenate([w.u0 for w in wls]), dtype=torch.complex128, device=dev)
    uT = torch.zeros(plan.nx, dtype=torch.complex128, device=dev)
    singles = []
    for w in wls:
        p1 = swr.Plan(nx=w.nx, a0=w.a0, b0=w.b0, nt=w.nt, dt=w.dt, nsub=w.nsub, node_off=w.off,
                      **shared)
        singles.append(dict(plan=p1, V=torch.tensor(w.V, dtype=torch.float64, device=dev),
                            u0=torch.tensor(w.u0, dtype=torch.complex128, device=dev),
                            uT=torch.zeros(w.nx, dtype=torch.complex128, device=dev)))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def batched():
        plan.build_interface(V, u0)
        return plan.solve(None, False, uT)

    def one_by_one():
        its = []
        for c in singles:
            c["plan"].build_interface(c["V"], c["u0"])
            its.append(c["plan"].solve(None, False, c["uT"])["iterations"])
        return its

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms, out = [], None
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            out = fn()
            ev1.record()
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return sum(ms), out

    plan.get_stats(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = swr.swr_kernel_launch_count()
    t_b, info = timed(batched)
    launches = swr.swr_kernel_launch_count() - launches0
    clocks = sampler.stop()
    st = plan.get_stats(reset=True)
    t_s, its = timed(one_by_one)
    u_b = uT.cpu().numpy()
    k, dev_max = 0, 0.0
    for w, c in zip(wls, singles):
        u1 = c["uT"].cpu().numpy()
        dev_max = max(dev_max, float(np.linalg.norm(u_b[k:k + w.nx] - u1) / np.linalg.norm(u1)))
        k += w.nx
    ps = st["march_point_steps"] / args.steps
    value = ps / (t_b / args.steps * 1e-3)
    achieved = FLOPS_PER_POINT_STEP * st["march_point_steps"] / (st["march_ms"] * 1e-3) / 1e9
    # end to end: concatenated inputs from pinned host memory, u(T) back
    hV, hu0 = V.cpu().pin_memory(), u0.cpu().pin_memory()
    huT = torch.empty(plan.nx, dtype=torch.complex128).pin_memory()

    def e2e_step():
        V.copy_(hV, non_blocking=True)
        u0.copy_(hu0, non_blocking=True)
        r = batched()
        huT.copy_(uT, non_blocking=True)
        return r
    t_e, _ = timed(e2e_step)
    cpu = None
    if not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        runs = {}
        for thr in (ncores, 1):
            secs, pss = 0.0, 0
            for w in wls[:8]:
                _, s1, p1 = cpu_oracle_marches(w, thr)
                secs += s1
                pss += p1
            runs[thr] = (pss / secs, secs, pss)
        v, secs, pss = runs[ncores]
        cpu = {"value": v, "unit": "point-steps/s", "cores": ncores, "kind": "oracle",
               "host": host_info(ncores),
               "sample": f"oracle d-marches of every subdomain of the first 8 instances, one "
                         f"march per task on {ncores} threads ({pss:.3g} point-steps, "
                         f"{secs:.1f} s)",
               "one_core": {"value": runs[1][0], "cores": 1,
                            "sample": f"the same on one thread ({runs[1][2]:.3g} point-steps, "
                                      f"{runs[1][1]:.1f} s)"}}
    line = {
        "metric": "SWR subdomain CN point-steps/s (solve time to 1e-10 interface residual "
                  "reported as ms_per_step)",
        "value": value, "unit": "point-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_b / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "swr_batch: 128 independent instances, 2k-40k P1 nodes each "
                               "(h=1e-3), N=4-64 uneven subdomains of 200-2000 nodes, 100-400 "
                               "steps (dt=1e-3), 4 seeded Gaussian bumps, one packet, Robin "
                               "p=sqrt(5)e^{-i pi/4}; build interface + GMRES(30) with the "
                               "causal preconditioner to 1e-10 on the concatenated system + "
                               "final march, one batched plan",
                   "instances": len(wls), "nodes": int(sum(w.nx for w in wls)),
                   "subdomains": int(sum(w.nsub for w in wls)),
                   "point_steps_per_step": ps, "l2": "flushed by a 256 MB write before each step",
                   "parallelism": "single GPU"},
        "roofline": {"kernel": "k_march_static", "bound": "alu", "achieved": achieved,
                     "peak": peak[0], "unit": "GFLOP/s",
                     "frac": achieved / peak[0], "traffic": None,
                     "launches": st["march_launches"],
                     "avg_launch_ms": st["march_ms"] / max(st["march_launches"], 1),
                     "flops_per_point_step": FLOPS_PER_POINT_STEP,
                     "peak_basis": peak[1], "frac_of_nominal": achieved / FP64_PEAK_GFLOPS},
        "per_instance_plans": {"ms_per_step": t_s / args.steps,
                               "speedup_of_batched": t_s / t_b,
                               "iterations_min_max": [min(its), max(its)],
                               "max_rel_diff_uT": dev_max},
        "batched_iterations": info["iterations"], "batched_residual": info["residual"],
        "batched_phases_ms": {"build": info["t_build_ms"], "solve": info["t_solve_ms"],
                              "final": info["t_final_ms"]},
        "cpu_baseline": cpu,
        "e2e": {"value": ps / (t_e / args.steps * 1e-3), "unit": "point-steps/s",
                "h2d_bytes_per_step": V.numel() * 8 + u0.numel() * 16,
                "d2h_bytes_per_step": uT.numel() * 16, "ms_per_step": t_e / args.steps},
        "gpu_launches": launches, "clocks": clocks,
    }
    plan.destroy()
    for c in singles:
        c["plan"].destroy()
    return line


def oracle_solve_split(P, threads, solver="gmres", restart=30, maxit=2000):
    """The oracle's whole new-algorithm solve (Algorithm 3) split into its parts, the
    marches of each part run one per task on `threads` host threads: build (d and the
    first columns), Krylov (GMRES(restart) on (I - L) g = d to 1e-10, or the fixed point
    g <- L g + d), final march.  Returns a dict of seconds, iterations, point-steps."""
    import concurrent.futures
    import numpy as np
    import oracle as O
    N, nt = P.nsub, P.nt
    e1 = np.zeros(nt, np.complex128)
    e1[0] = 1.0
    zero = np.zeros(nt, np.complex128)

    def flux(j, m, lj, rj, out, which):
        if j > 0:
            out[("a", j, which)] = (-lj if lj is not None else 0) + O.s_flux(P, m.va, j, 0)
        if j < N - 1:
            out[("b", j, which)] = (-rj if rj is not None else 0) + O.s_flux(P, m.vb, j, 1)

    def build_task(job):
        j, which = job
        a, b = int(P.off[j]), int(P.off[j + 1])
        u0 = P.u0[a:b + 1] if which == "d" else np.zeros(b - a + 1, np.complex128)
        lj = ((e1 if which == "l" else zero) if j > 0 else None)
        rj = ((e1 if which == "r" else zero) if j < N - 1 else None)
        m = O.sub_march(P, j, u0, lj, rj)
        out = {}
        flux(j, m, lj, rj, out, which)
        return out, (b - a + 1) * nt

    jobs = [(j, w) for j in range(N) for w in ("d", "l", "r")
            if not ((w == "l" and j == 0) or (w == "r" and j == N - 1))]
    ps = 0
    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        t0 = time.perf_counter()
        res = {}
        for out, n in ex.map(build_task, jobs):
            res.update(out)
            ps += n
        d = np.zeros((P.nblk, nt), np.complex128)
        cols = np.zeros((N, 4, nt), np.complex128)
        for j in range(N):
            if j > 0:
                d[O.blk_r(j - 1)] = res[("a", j, "d")]
                cols[j, 0] = res[("a", j, "l")]
                if j < N - 1:
                    cols[j, 1] = res[("a", j, "r")]
            if j < N - 1:
                d[O.blk_l(j + 1)] = res[("b", j, "d")]
                cols[j, 3] = res[("b", j, "r")]
                if j > 0:
                    cols[j, 2] = res[("b", j, "l")]
        t1 = time.perf_counter()
        if solver == "gmres":
            r = O.gmres(lambda v: O.apply_I_minus_L(P, cols, v), d, None, m=restart,
                        tol=1e-10, maxit=maxit)
        else:
            r = O.fixed_point(lambda v: O.apply_L(P, cols, v) + d, np.zeros_like(d), tol=1e-10,
                              maxit=maxit)
        g = np.asarray(r.x).reshape(d.shape)
        t2 = time.perf_counter()

        def final_task(j):
            a, b = int(P.off[j]), int(P.off[j + 1])
            O.sub_march(P, j, P.u0[a:b + 1], g[O.blk_l(j)] if j > 0 else None,
                        g[O.blk_r(j)] if j < N - 1 else None)
            return (b - a + 1) * nt
        ps += sum(ex.map(final_task, range(N)))
        t3 = time.perf_counter()
    return {"build_s": t1 - t0, "krylov_s": t2 - t1, "final_s": t3 - t2, "total_s": t3 - t0,
            "iterations": int(r.iterations), "converged": bool(r.converged),
            "point_steps": ps, "threads": threads}


def run_plain(args, dev, local, peak):
    """The plain workload (1001 nodes on (-12, 12), 200 steps, N = 4, V = -x^2/4): the
    new algorithm (Algorithm 3: d and L built by marches, GMRES(30) on (I - L) g = d to
    1e-10, u(T)) against the classical algorithm (Algorithm 1: g <- R g with full
    marches until ||g^{k+1} - g^k|| < 1e-10), for the configuration's Robin condition
    S-bar v = sqrt(5) e^{-i pi/4} v and for the paper's S_0^2.  Timed per solve on the
    plan's stream; the record's value is the new algorithm's (Robin, GMRES with the
    causal preconditioner) point-steps/s."""
    import numpy as np
    import torch
    import oracle as O
    from paper_1503_02564_gb300 import swr
    from paper_1503_02564_gb300 import workloads as W
    wl = W.config1()
    V = torch.tensor(wl.V, dtype=torch.float64, device=dev)
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    CLASSICAL_CAP = 100

    def plan_for(tc, solver, precond, maxit=2000):
        return swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                        node_off=wl.off, p=wl.sigma, tc=tc, solver=solver, precond=precond,
                        restart=30, maxit=maxit, tol_abs=1e-10)

    def timed(plan, host=None):
        g = torch.zeros(plan.n_interface, dtype=torch.complex128, device=dev)
        uT = torch.zeros(wl.nx, dtype=torch.complex128, device=dev)
        ms, info = [], None
        for k in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            if host is not None:
                V.copy_(host[0], non_blocking=True)
                u0.copy_(host[1], non_blocking=True)
            plan.build_interface(V, u0)
            info = plan.solve(g, False, uT, allow_not_converged=True)
            if host is not None:
                host[2].copy_(uT, non_blocking=True)
            ev1.record()
            ev1.synchronize()
            if k >= args.warmup:
                ms.append(ev0.elapsed_time(ev1))
        return sum(ms) / len(ms), info, uT.cpu().numpy()

    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  sigma=wl.sigma)
    _, u_mono = O.mono_interface(P)
    rows = []
    head = None
    for tcname, tc in (("Robin p=sqrt(5)e^{-i pi/4}", swr.SWR_TC_ROBIN),
                       ("S_0^2", swr.SWR_TC_S02)):
        for alg, solver, precond, cap in (
                ("new (Alg. 3), GMRES(30) + causal preconditioner", swr.SWR_SOLVER_GMRES,
                 swr.SWR_PC_CAUSAL, 2000),
                ("new (Alg. 3), GMRES(30)", swr.SWR_SOLVER_GMRES, swr.SWR_PC_NONE, 2000),
                ("classical (Alg. 1)", swr.SWR_SOLVER_CLASSICAL, swr.SWR_PC_NONE,
                 CLASSICAL_CAP)):
            plan = plan_for(tc, solver, precond, cap)
            plan.get_stats(reset=True)
            ms, info, uT = timed(plan)
            st = plan.get_stats(reset=True)
            row = {"tc": tcname, "algorithm": alg, "ms": ms, "iterations": info["iterations"],
                   "converged": info["status"] == swr.SWR_OK,
                   "residual0": info["residual0"], "residual": info["residual"],
                   "rel_err_uT_vs_monodomain": float(np.linalg.norm(uT - u_mono) /
                                                     np.linalg.norm(u_mono)),
                   "march_point_steps": st["march_point_steps"] / (args.warmup + args.steps),
                   "march_ms": st["march_ms"] / (args.warmup + args.steps)}
            if solver == swr.SWR_SOLVER_CLASSICAL and not row["converged"]:
                row["note"] = ("diverges: ||g^{k+1} - g^k|| went from %.3g to %.3g in %d "
                               "iterations (cap)" % (info["residual0"], info["residual"],
                                                     info["iterations"]))
            rows.append(row)
            if head is None:
                head = (plan, ms, st)
            else:
                plan.destroy()
    plan, ms, st = head
    ps = st["march_point_steps"] / (args.warmup + args.steps)
    achieved = FLOPS_PER_POINT_STEP * st["march_point_steps"] / (st["march_ms"] * 1e-3) / 1e9
    hV, hu0 = V.cpu().pin_memory(), u0.cpu().pin_memory()
    huT = torch.empty(wl.nx, dtype=torch.complex128).pin_memory()
    e_ms, _, _ = timed(plan, (hV, hu0, huT))
    plan.destroy()
    cpu = None
    if not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        Ps = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                       sigma=wl.sigma, tc=O.TC_S02)
        sp_all = oracle_solve_split(Ps, ncores)
        sp_one = oracle_solve_split(Ps, 1)
        cpu = {"value": sp_all["point_steps"] / sp_all["total_s"], "unit": "point-steps/s",
               "cores": ncores, "kind": "oracle", "host": host_info(ncores),
               "sample": "the oracle's whole new-algorithm solve of this workload with S_0^2 "
                         "(build marches, GMRES(30) to 1e-10, final march), marches one per "
                         "task on %d threads: %d GMRES iterations, %.2f s" % (
                             ncores, sp_all["iterations"], sp_all["total_s"]),
               "split_all_cores": sp_all, "split_one_core": sp_one}
    return {
        "metric": "SWR subdomain CN point-steps/s (solve time to 1e-10 interface residual "
                  "reported as ms_per_step)",
        "value": ps / (ms * 1e-3), "unit": "point-steps/s", "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
        "config": {"workload": "swr_plain: x in (-12,12), 1001 P1 nodes, T=0.2 dt=1e-3 (200 "
                               "steps), N=4 equal, V=-x^2/4, u0=exp(-x^2/2+5ix) with +-1e-3 "
                               "seeded phase noise, Robin p=sqrt(5)e^{-i pi/4}; new algorithm "
                               "(GMRES(30), causal preconditioner) vs classical, to 1e-10",
                   "l2": "flushed by a 256 MB write before each solve"},
        "algorithms": rows,
        "roofline": {"kernel": "k_march_static", "bound": "alu", "achieved": achieved,
                     "peak": peak[0], "unit": "GFLOP/s", "frac": achieved / peak[0],
                     "traffic": None, "peak_basis": peak[1],
                     "flops_per_point_step": FLOPS_PER_POINT_STEP,
                     "note": "4 systems of 251 nodes: latency-bound, one CTA per system"},
        "e2e": {"value": ps / (e_ms * 1e-3), "unit": "point-steps/s",
                "h2d_bytes_per_step": wl.nx * 8 + wl.nx * 16,
                "d2h_bytes_per_step": wl.nx * 16, "ms_per_step": e_ms},
        "cpu_baseline": cpu,
    }


def run_tcs(args):
    """Transmission conditions x interface solvers in the setting of the paper's
    comparison (Section 6): V = -x^2 on (-21, 21), dx = 5e-4 by default (the paper's
    1e-5 needs subdomains beyond the march's size limit at N = 2), dt = 1e-3,
    T = 0.5, N in {2, 500}, random initial interface vector, no preconditioner (the
    new algorithm); per entry the build, the solve to ||residual||_2 < 1e-10 (the fixed
    point: ||g^{k+1} - g^k||_2 < 1e-10) and its iterations.  Robin takes the paper's
    parameters per N and solver (S-bar v = -i p v).  One step is the whole table."""
    import numpy as np
    import torch
    from paper_1503_02564_gb300 import swr
    from paper_1503_02564_gb300 import workloads as W
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    conds = [("S_0^2", swr.SWR_TC_S02), ("S_0^3", swr.SWR_TC_S03), ("S_0^4", swr.SWR_TC_S04),
             ("S_1^2", swr.SWR_TC_S12), ("S_1^4", swr.SWR_TC_S14), ("Robin", swr.SWR_TC_ROBIN)]
    solvers = [("fixed point", swr.SWR_SOLVER_FIXED_POINT), ("gmres", swr.SWR_SOLVER_GMRES),
               ("bicgstab", swr.SWR_SOLVER_BICGSTAB)]
    robin_p = {(2, "fixed point"): 44.0, (2, "gmres"): 5.0, (2, "bicgstab"): 5.0,
               (500, "fixed point"): 45.0, (500, "gmres"): 19.0, (500, "bicgstab"): 6.0}
    nt = args.nt if args.nt > 0 else 500
    table, ps_total, t_total = [], 0, 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for N in (2, 500):
        wl = W.tc_comparison(nsub=N, nx=args.tcs_nx, nt=nt)
        V = torch.tensor(wl.V, dtype=torch.float64, device=dev)
        u0 = torch.tensor(wl.u0, dtype=torch.complex128, device=dev)
        g0 = torch.tensor(W.random_interface(wl.nblk, wl.nt, 1).ravel(), dtype=torch.complex128,
                          device=dev)
        for cname, tc in conds:
            for sname, solver in solvers:
                p = -1j * robin_p[(N, sname)] if tc == swr.SWR_TC_ROBIN else 0j
                # 4.2M nodes: keep u(T) from the final march
                plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=N,
                                node_off=wl.off, tc=tc, p=p, solver=solver, restart=200,
                                maxit=2000, tol_abs=1e-10, tuning={"superpose": -1})
                g = g0.clone()
                torch.cuda.synchronize()
                ev0.record()
                plan.build_interface(V, u0)
                info = plan.solve(g, True, None, allow_not_converged=True)
                ev1.record()
                ev1.synchronize()
                ms = ev0.elapsed_time(ev1)
                st = plan.get_stats(reset=True)
                plan.destroy()
                ps_total += st["march_point_steps"]
                t_total += ms
                table.append({"N": N, "tc": cname, "solver": sname,
                              "robin_p": robin_p[(N, sname)] if tc == swr.SWR_TC_ROBIN else None,
                              "iterations": info["iterations"],
                              "converged": info["status"] == swr.SWR_OK,
                              "residual": info["residual"], "solve_ms": info["t_solve_ms"],
                              "build_ms": info["t_build_ms"], "total_ms": ms})
    line = {
        "metric": "SWR subdomain CN point-steps/s (solve time to 1e-10 interface residual "
                  "reported as ms_per_step)",
        "value": ps_total / (t_total * 1e-3), "unit": "point-steps/s", "n_gpus": world,
        "steps": 1, "warmup": 0, "ms_per_step": t_total, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "swr_tc_comparison: x in (-21,21), dx=%g (%d P1 nodes), "
                               "T=%g dt=1e-3, V=-x^2, u0=exp(-(x+10)^2+20i(x+10)), N in {2,500}, "
                               "random g0; S_0^2..S_1^4 and Robin x fixed point / GMRES(200) / "
                               "BiCGStab, no preconditioner, to 1e-10"
                               % (42.0 / (args.tcs_nx - 1), args.tcs_nx, nt * 1e-3),
                   "parallelism": "single GPU"},
        "table": table,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        line = run_batch(args)
        if dist_env()[0] == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload == "tcs":
        return run_tcs(args)
    if args.workload == "fp64peak":
        return run_fp64peak(args)
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # the roofline's denominator: this GPU's FP64 DFMA rate, measured now (about 1.5 s)
    peak_gf, peak_ms, peak_clk = fp64_probe(0, 1.5, dev, ClockSampler(local))
    peak = (peak_gf, "measured FP64 DFMA rate of this GPU (swr_fp64_peak, %.0f ms, median SM "
                     "%s MHz)" % (peak_ms, peak_clk["sm_mhz"] if peak_clk else "?"))
    line = run_workload(args, args.workload, rank, world, local, dev, peak)
    if (rank == 0 and world == 1 and args.workload == "scaling" and not args.no_sub
            and args.nt == 0):
        # the other workloads of the method, fewer steps each, beside the headline
        import copy
        subs = {}
        for name in ("plain", "batch", "timedep", "nonlinear"):
            t0 = time.perf_counter()
            try:
                sa = copy.copy(args)
                sa.steps, sa.warmup = args.sub_steps, args.sub_warmup
                if name == "plain":
                    subs[name] = run_plain(sa, dev, local, peak)
                elif name == "batch":
                    subs[name] = run_batch(sa, peak)
                else:
                    sa.workload, sa.nsub, sa.precond = name, "", "causal"
                    subs[name] = run_workload(sa, name, rank, world, local, dev, peak)
            except Exception as e:   # a failed sub-record must not hide the headline
                subs[name] = {"error": "%s: %s" % (type(e).__name__, e)}
            subs[name]["wall_s"] = time.perf_counter() - t0
        line["sub"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_workload(args, workload, rank, world, local, dev, peak):
    """One timed workload (scaling / timedep / adjoint / nonlinear): W warm-up steps,
    K timed steps with the L2 flushed before each, CUDA events on the plans' stream,
    max over ranks; the march roofline from the library's per-launch events, an
    end-to-end figure from pinned host buffers, and the CPU oracle's rate.  Returns the
    JSON record (rank 0) or None."""
    import numpy as np
    import torch
    from paper_1503_02564_gb300 import swr
    from paper_1503_02564_gb300 import workloads as W

    peak_gf, peak_basis = peak
    nsubs = tuple(int(x) for x in args.nsub.split(",")) if args.nsub else NSUBS
    precond = swr.SWR_PC_CAUSAL if args.precond == "causal" else swr.SWR_PC_NONE
    timedep = workload == "timedep"
    nonlin = workload == "nonlinear"
    adjoint = workload in ("adjoint", "nonlinear")
    if timedep:
        nsubs = (64,)
    if nonlin:
        nsubs = (32,)

    cases = []
    for N in nsubs:
        if nonlin:
            wl = W.config5(nsub=N, nt=args.nt) if args.nt > 0 else W.config5(nsub=N)
            plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=N,
                            node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_NONLINEAR,
                            solver=swr.SWR_SOLVER_FIXED_POINT, maxit=200, tol_abs=1e-10,
                            precond=swr.SWR_PC_MEAN_POTENTIAL, nl_tol=1e-13, nl_maxit=50,
                            tuning=tuning_of(args))
        elif timedep:
            wl = W.config4(nsub=N, nt=args.nt) if args.nt > 0 else W.config4(nsub=N)
            plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=N,
                            node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_TIME, restart=60,
                            maxit=400, tol_abs=1e-10, precond=swr.SWR_PC_MEAN_POTENTIAL,
                            tuning=tuning_of(args))
        else:
            wl = W.config2(nsub=N, nt=args.nt) if args.nt > 0 else W.config2(nsub=N)
            if args.tc == "s02":
                wl.tc = swr.SWR_TC_S02
            plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=N,
                            node_off=wl.off, p=wl.sigma, tc=wl.tc, restart=30, maxit=2000,
                            tol_abs=1e-10, precond=precond, pc_sweeps=args.pc_sweeps,
                            tuning=tuning_of(args))
        V = torch.tensor(np.ascontiguousarray(wl.V).ravel(), dtype=torch.float64, device=dev)
        u0 = torch.tensor(wl.u0, dtype=torch.complex128, device=dev)
        g = torch.zeros(plan.n_interface, dtype=torch.complex128, device=dev)
        uT = torch.zeros(wl.nx, dtype=torch.complex128, device=dev)
        cases.append(dict(N=N, wl=wl, plan=plan, V=V, u0=u0, g=g, uT=uT,
                          ps=march_point_steps(wl)))
        if adjoint:
            if nonlin:
                # the misfit target: u(T) for the seeded perturbed potential (untimed)
                plan.build_interface(torch.tensor(W.config5_target_potential(wl),
                                                  dtype=torch.float64, device=dev), u0)
                tgt_t = torch.zeros(wl.nx, dtype=torch.complex128, device=dev)
                plan.solve(None, False, tgt_t)
                tgt_np = tgt_t.cpu().numpy()
            else:
                tgt_np = W.misfit_target(wl)
            cases[-1].update(
                tgt=torch.tensor(tgt_np, dtype=torch.complex128, device=dev),
                ubar=torch.empty_like(uT),
                grad=torch.empty(wl.nx, dtype=torch.float64, device=dev),
                ev=(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)))
    ps_step = sum(c["ps"] for c in cases)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step():
        infos = []
        for c in cases:
            c["plan"].build_interface(c["V"], c["u0"])
            infos.append(c["plan"].solve(c["g"], False, c["uT"]))
            if adjoint:
                c["ev"][0].record()
                c["J"] = c["plan"].misfit(c["uT"], c["tgt"], c["ubar"])
                c["plan"].adjoint(c["ubar"], c["grad"], 0)
                c["ev"][1].record()
        return infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for c in cases:
        c["plan"].get_stats(reset=True)

    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = swr.swr_kernel_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    per_step_ms, infos_last = [], None
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                        # L2 flush between timed steps (untimed)
        torch.cuda.synchronize()
        ev0.record()
        infos_last = step()
        ev1.record()
        ev1.synchronize()
        per_step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = swr.swr_kernel_launch_count() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    t_ms = replicas_max_ms(sum(per_step_ms), dev)

    # march kernel statistics inside the timed region (events around each launch)
    st = [c["plan"].get_stats(reset=True) for c in cases]
    m_launch = sum(s["march_launches"] for s in st)
    m_ms = sum(s["march_ms"] for s in st)
    m_ps = sum(s["march_point_steps"] for s in st)
    # V(t,x): variant 3 streams every step's factors (computed once per build)
    # through the constant-matrix march kernel; variant 1 refactorises per step
    variant = st[0]["march_variant"]
    traffic = None
    if (march_sources_hash() == MARCH_TRAFFIC["sources"] and args.nt == 0 and args.tc == "robin"
            and (timedep or tuple(nsubs) == NSUBS)):
        traffic = MARCH_TRAFFIC["timedep" if timedep else "scaling"]
    streamed = variant == swr.MARCH_TDEP_STREAMED
    fpp = FLOPS_PER_POINT_STEP_TDEP if variant == swr.MARCH_TDEP_REFACTOR else FLOPS_PER_POINT_STEP
    m_kernel = "k_march_tdep" if variant == swr.MARCH_TDEP_REFACTOR else "k_march_static"
    nl_pit = sum(s["march_point_iterations"] for s in st)
    nl_ms = sum(s["nl_march_ms"] for s in st)
    nl_launch = sum(s["nl_march_launches"] for s in st)
    # algorithmic bytes per point-step: u read + written (32 B) plus, streamed,
    # the factors of that node and step
    bpp = 32.0
    if streamed:
        bpp += st[0]["march_factor_bytes_per_step"] / float(cases[0]["wl"].nx)
    achieved = fpp * m_ps / (m_ms * 1e-3) / 1e9 if m_ms > 0 else 0.0
    if nonlin:
        # the nonlinear marches (forward SWR sweeps and the adjoint's monodomain marches)
        # dominate: their flops per node and inner iteration over their own device time
        m_kernel = "k_march_nl_tl (forward sweeps and the gradient's monodomain marches)"
        achieved = FLOPS_PER_POINT_ITER_NL * nl_pit / (nl_ms * 1e-3) / 1e9 if nl_ms > 0 else 0.0
    # whole-step throughput from the library's own count of marched point-steps
    # (equal to the analytic count for the scaling step; GMRES-dependent otherwise)
    ps_step = m_ps / args.steps
    value = whole_job_rate(ps_step, args.steps, world, t_ms)
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    march_pss = m_ps / (m_ms * 1e-3) if m_ms > 0 else 0.0

    # end-to-end: host (pinned) buffers through the public API, copies inside the region
    e2e = None
    if not args.no_e2e:
        hosts = []
        for c in cases:
            hosts.append(dict(V=c["V"].cpu().pin_memory(), u0=c["u0"].cpu().pin_memory(),
                              uT=torch.empty_like(c["uT"], device="cpu").pin_memory()))
            if adjoint:
                hosts[-1].update(tgt=c["tgt"].cpu().pin_memory(),
                                 grad=torch.empty_like(c["grad"], device="cpu").pin_memory())
        h2d = sum(h["V"].numel() * 8 + h["u0"].numel() * 16 for h in hosts)
        d2h = sum(h["uT"].numel() * 16 for h in hosts)
        if adjoint:
            h2d += sum(h["tgt"].numel() * 16 for h in hosts)
            d2h += sum(h["grad"].numel() * 8 + 8 for h in hosts)
        torch.cuda.synchronize()
        e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            for c, h in zip(cases, hosts):
                c["V"].copy_(h["V"], non_blocking=True)
                c["u0"].copy_(h["u0"], non_blocking=True)
                c["plan"].build_interface(c["V"], c["u0"])
                c["plan"].solve(c["g"], False, c["uT"])
                h["uT"].copy_(c["uT"], non_blocking=True)
                if adjoint:
                    c["tgt"].copy_(h["tgt"], non_blocking=True)
                    c["plan"].misfit(c["uT"], c["tgt"], c["ubar"])
                    c["plan"].adjoint(c["ubar"], c["grad"], 0)
                    h["grad"].copy_(c["grad"], non_blocking=True)
            ev1.record()
            ev1.synchronize()
            e_ms += ev0.elapsed_time(ev1)
        e_ms = replicas_max_ms(e_ms, dev)
        e2e = {"value": whole_job_rate(ps_step, args.steps, world, e_ms), "unit": "point-steps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e_ms / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nonlin:
        v, s, ps = cpu_oracle_adjoint_nl_sample(cases[0]["wl"], 40)
        cpu = {"value": v, "unit": "point-steps/s", "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": f"oracle discrete adjoint of the nonlinear monodomain scheme on the "
                         f"{cases[0]['wl'].nx}-node grid, first 40 steps (forward march with "
                         f"inner fixed points, exact linearised adjoint solves; {ps:.3g} "
                         f"point-steps, {s:.1f} s)"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline and adjoint:
        v, s, ps = cpu_oracle_adjoint_sample(cases[0]["wl"], 100)
        cpu = {"value": v, "unit": "point-steps/s", "cores": 1, "kind": "oracle", "host": host_info(),
               "sample": f"oracle discrete adjoint of the monodomain scheme on the "
                         f"{cases[0]['wl'].nx}-node grid, first 100 steps (forward and adjoint "
                         f"marches, {ps:.3g} point-steps, {s:.1f} s)"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        if timedep:
            wl_cpu = cases[0]["wl"]
        else:
            wl_cpu = cases[-1]["wl"] if cases[-1]["N"] == 500 else W.config2(nsub=500)
        ncores = os.cpu_count() or 1
        v, s, ps = cpu_oracle_marches(wl_cpu, ncores, min_seconds=8.0)
        v1, s1, ps1 = cpu_oracle_marches(wl_cpu, 1, min_seconds=6.0)
        what = "time-dependent" if timedep else "N=500 scaling"
        cpu = {"value": v, "unit": "point-steps/s", "cores": ncores, "kind": "oracle",
               "host": host_info(ncores),
               "sample": f"oracle d-marches of the {what} workload's {wl_cpu.nsub} subdomains, "
                         f"one march per task on {ncores} threads ({ps:.3g} point-steps, "
                         f"{s:.1f} s)",
               "one_core": {"value": v1, "cores": 1,
                            "sample": f"the same marches on one thread ({ps1:.3g} "
                                      f"point-steps, {s1:.1f} s)"}}

    line = None
    if rank == 0:
        per_n = []
        for c, info in zip(cases, infos_last):
            per_n.append({"N": c["N"], "iterations": info["iterations"],
                          "causal_sweeps": st[len(per_n)]["causal_sweeps"],
                          "causal_window": st[len(per_n)]["causal_window"],
                          "superposed": st[len(per_n)]["superposed"],
                          "toeplitz_fft_length": st[len(per_n)]["toeplitz_fft_length"],
                          "residual": info["residual"], "build_ms": info["t_build_ms"],
                          "solve_ms": info["t_solve_ms"], "final_ms": info["t_final_ms"],
                          "interface_jump": info["interface_jump"]})
            if adjoint:
                per_n[-1].update(J=c["J"], adjoint_ms=c["ev"][0].elapsed_time(c["ev"][1]),
                                 grad_norm=float(c["grad"].norm()))
        line = {
            "metric": "SWR subdomain CN point-steps/s (solve time to 1e-10 interface residual "
                      "reported as ms_per_step)",
            "value": value, "unit": "point-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name_timedep(cases[0]["wl"].nt) if timedep else
                       workload_name_nonlinear(cases[0]["wl"].nt) if nonlin else
                       (workload_name(nsubs, args.tc, cases[0]["wl"].nt)
                        + ("; then J = ||u(T) - u_target||_M^2 and dJ/dV(x) by swr_adjoint, "
                           "the library's checkpoint interval" if adjoint else "")),
                       "point_steps_per_step": ps_step,
                       "precond": "mean_potential" if (timedep or nonlin) else args.precond,
                       "l2": "flushed by a 256 MB write before each step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"kernel": m_kernel, "bound": "alu",
                         "achieved": achieved,
                         "peak": peak_gf, "unit": "GFLOP/s",
                         "frac": achieved / peak_gf, "traffic": traffic,
                         "launches": m_launch, "avg_launch_ms": m_ms / max(m_launch, 1),
                         "flops_per_point_step": fpp,
                         **({"flops_per_point_iteration": FLOPS_PER_POINT_ITER_NL,
                             "point_iterations": nl_pit, "nl_launches": nl_launch,
                             "nl_ms": nl_ms} if nonlin else {}),
                         "peak_basis": peak_basis,
                         "frac_of_nominal": achieved / FP64_PEAK_GFLOPS,
                         "march_share_of_step": m_ms / t_ms if t_ms > 0 else None},
            "hbm_roof": {"point_steps_per_s": hbm * 1e9 / bpp,
                         "march_point_steps_per_s": march_pss,
                         "frac": march_pss / (hbm * 1e9 / bpp),
                         "bytes_per_point_step": bpp,
                         "basis": "32 B/point-step (read+write complex128 u)"
                                  + (" + streamed per-step factors" if streamed else "")
                                  + " at measured HBM GB/s"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "wall_s": wall, "per_n": per_n,
            "stats": {"toeplitz_ms": sum(s["toeplitz_ms"] for s in st),
                      "precond_ms": sum(s["precond_ms"] for s in st),
                      "march_ms": m_ms},
        }
    for c in cases:
        c["plan"].destroy()
    return line if rank == 0 else None


if __name__ == "__main__":
    main()
