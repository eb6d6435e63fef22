#!/usr/bin/env python
"""Throughput of the parallel-in-time solve: space-time DOF/s at relative
residual 1e-8 on one GB300 (N GPUs: independent replicas, weak scaling).

One step = one pint_solve of the workload from the initial iterate (zero by default) to
||b - K(U)|| / ||b|| <= tol: residual, alpha-scaled time FFT, spatial shifted
solves, inverse FFT + update, repeated until the tolerance is met.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|mixed_ff|fp64]
                  [--alpha A] [--init 0|2] [--workload NAME] [--impl ours|reference]

The headline is the mixed form: complex64 time transforms and shifted spatial
solves, with the residual, the alpha-scaling and unscaling and the update in
FP64 (the residual and its scaling exactly in block fixed point on the integer
pipes).  The plain FP64 form and the float-float form are timed beside it, and
every timed solve's result is compared with the oracle's sequential solution,
computed once in a separate process outside the timed region.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle
(sequential backward Euler with banded LU) on a bounded sample of the same
workload, single-threaded.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Workloads (synthetic inputs shaped like the paper's experiments).
WORKLOADS = {
    # 2-D linearized Cahn-Hilliard, homogeneous Neumann, cell-centred 256x256,
    # beta = 0.5, eps = 0.05, N_t = 128, T = 0.1, u0 iid uniform[-0.05, 0.05].
    "linear_ch_2d_256x256_nt128": dict(equation="linear_ch", dim=2, nx=256, ny=256, bc="neumann", eps=0.05,
                                       beta=0.5, T=0.1, nt=128, n_windows=1, u0="uniform0.05"),
    # The same equation on a 512x512 grid (inputs larger than L2; used for kernel profiles).
    "linear_ch_2d_512x512_nt128": dict(equation="linear_ch", dim=2, nx=512, ny=512, bc="neumann", eps=0.05,
                                       beta=0.5, T=0.1, nt=128, n_windows=1, u0="uniform0.05"),
    # 2-D Cahn-Hilliard, Neumann, cell-centred 512x512, eps = 0.02, dt = 1e-4, 8 windows of 256 steps,
    # u0 = 0.1 uniform[-1,1] minus its mean (adaptive window policy on).
    "cahn_hilliard_2d_512x512_8x256": dict(equation="cahn_hilliard", dim=2, nx=512, ny=512, bc="neumann", eps=0.02,
                                           beta=0.0, T=2048 * 1e-4, nt=256, n_windows=8, u0="ch"),
    # The same at 128x128 (a size the CPU oracle finishes).
    "cahn_hilliard_2d_128x128_8x256": dict(equation="cahn_hilliard", dim=2, nx=128, ny=128, bc="neumann", eps=0.02,
                                           beta=0.0, T=2048 * 1e-4, nt=256, n_windows=8, u0="ch"),
    # 2-D Cahn-Hilliard with Eyre's splitting (PinT-II): Neumann 64x64, eps = 0.01, dt = 1e-5, 39 windows of
    # 256 steps (T = 0.09984), alpha = 0.05, u0 = 0.1 uniform[-1,1] minus its mean (the paper's 2-D PinT-II demo)
    "cahn_hilliard_eyre_2d_64x64_39x256": dict(equation="cahn_hilliard_eyre", dim=2, nx=64, ny=64, bc="neumann",
                                               eps=0.01, beta=0.0, T=39 * 256 * 1e-5, nt=256, n_windows=39,
                                               u0="ch", alpha=0.05),
    # 1-D linearized CH over a long time axis (four-step time FFT): Neumann 128 cells, N_t = 65536,
    # T = 0.3 (dt = 4.6e-6; the growing modes then keep alpha G <= 0.1), beta = 0.5, eps = 0.05,
    # u0 iid uniform[-0.05, 0.05]
    "linear_ch_1d_128_nt65536": dict(equation="linear_ch", dim=1, nx=128, ny=1, bc="neumann", eps=0.05, beta=0.5,
                                     T=0.3, nt=65536, n_windows=1, u0="uniform0.05"),
    # 1-D biharmonic over about a million steps (the paper's dt = 1e-6 case): Neumann 64 cells (h = 1/64),
    # N_t = 2^20 (three-pass time FFT), T = 1.048576, alpha = 1e-3, u0 iid uniform[-0.05, 0.05]
    "biharmonic_1d_64_nt1048576": dict(equation="biharmonic", dim=1, nx=64, ny=1, bc="neumann", eps=1.0, beta=0.0,
                                       T=(1 << 20) * 1e-6, nt=1 << 20, n_windows=1, u0="uniform0.05", alpha=1e-3),
    # 1-D biharmonic, simply supported, 64 vertices, N_t = 32, T = 0.01, u0 = sin(pi x) + 0.5 sin(3 pi x)
    "biharmonic_1d_64_nt32": dict(equation="biharmonic", dim=1, nx=64, ny=1, bc="ss", eps=1.0, beta=0.0,
                                  T=0.01, nt=32, n_windows=1, u0="sines"),
}
DEFAULT_WORKLOAD = "linear_ch_2d_256x256_nt128"
L2_FLUSH_BYTES = 512 * 2**20   # > 129 MB L2


def make_u0(wl: dict, seed: int):
    from paper_2304_14021_gb300 import synth
    ns = wl["nx"] * (wl["ny"] if wl["dim"] == 2 else 1)
    if wl["u0"] == "uniform0.05":
        return synth.u0_uniform(ns, -0.05, 0.05, seed)
    if wl["u0"] == "sines":
        return synth.u0_sine_modes(wl["nx"])
    return synth.u0_ch(ns, seed)


def solver_kw(wl: dict, args, precision=None) -> dict:
    kw = {k: v for k, v in wl.items() if k not in ("u0", "alpha")}
    kw.update(alpha=wl.get("alpha", args.alpha), tol=args.tol, max_iter=250, precision=precision or args.precision,
              init_guess=args.init)
    return kw


# DRAM bytes per launch of a kernel, from one ncu capture of the named workload,
# valid only for the source file's contents it was taken on (sha256 prefix).
KERNEL_TRAFFIC = {
    ("residual", "mixed_ff"): {"src": "k_residual_ff.cu", "src_sha256_16": "f2beb509f59f81f0",
                               "workload": "linear_ch_2d_256x256_nt128", "dram_bytes": 68294656 + 5862912},
    ("residual", "mixed"): {"src": "k_residual_fx.cu", "src_sha256_16": "073bf41d6c8c168b",
                            "workload": "linear_ch_2d_256x256_nt128", "dram_bytes": 71845376 + 10023424},
}


def _kernel_traffic(phase: str, precision: str, workload: str):
    import hashlib
    t = KERNEL_TRAFFIC.get((phase, precision))
    if t is None or t["workload"] != workload:
        return None
    path = os.path.join(ROOT, "paper_2304_14021_gb300", "csrc", t["src"])
    try:
        sha = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return t["dram_bytes"] if sha == t["src_sha256_16"] else None


def host_cpu() -> dict:
    """Core count and CPU model of the host the CPU baseline runs on."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def ff_residual_ops_per_dof(equation: str, dim: int, accurate: bool = False) -> float:
    """FP32 lane operations (add, multiply or FMA: one each) per space-time DOF
    of the float-float residual kernel on square cells, counted from its code:
    TwoSum 6, fast TwoSum 3, exact product 2 (FMUL + FMA), double-word multiply
    8, accurate double-word add 20, one step of the error-free sum 8 and its
    final renormalization 6.  An unscaled Laplacian point sums 3 (1-D) or 5
    (2-D) terms plus a power-of-two scaling (2 ops): 24 / 40 ops with the
    error-free sum, 42 / 82 with chained accurate adds.  The first Laplacian (and
    u^3 for Cahn-Hilliard) covers the tile plus a one-point halo: 514/512 (1-D),
    34*18/(32*16) (2-D).  The residual dt*r = u_{n-1} - u_n - sum of the operator
    terms is one error-free sum (accurate: two subtractions and an add per extra
    term); 4 more ops scale s and accumulate the norms."""
    halo = 514.0 / 512.0 if dim == 1 else (34.0 * 18.0) / (32.0 * 16.0)
    if equation == "cahn_hilliard_eyre" and not accurate:
        # Eyre's splitting: c2 Lap^2 u_n and cN Lap(u_n^3) (multiply, multiply, accurate add), the
        # explicit c1 Lap u_{n-1} (one multiply), one error-free sum of four terms
        lap = 24.0 if dim == 1 else 40.0
        return lap * halo + lap + 16.0 * halo + lap + 8.0 + 8.0 + 20.0 + 8.0 + 30.0 + 4.0
    nterm = 1 + (equation in ("linear_ch", "cahn_hilliard")) + (equation == "cahn_hilliard")
    if accurate:
        lap = 42.0 if dim == 1 else 82.0
        f = lap * halo + lap + 8.0 * nterm + 20.0 * (nterm - 1) + 40.0
    else:
        lap = 24.0 if dim == 1 else 40.0
        f = lap * halo + lap + 8.0 * nterm + 8.0 * (nterm + 1) + 6.0
    if equation == "cahn_hilliard":
        f += 16.0 * halo + lap          # u^3 on tile + halo, Lap(u^3)
    return f + 4.0


STEP_PHASES = ("time_fwd", "spatial0", "spatial1", "spatial2", "time_inv")


def phase_bytes_per_dof(precision: str, nt: int) -> dict:
    """Algorithmic HBM bytes per space-time DOF of each phase (one launch)."""
    t = 4 if precision in ("mixed", "mixed_ff") else 8   # real transform word (the iterate is 8 B in all modes)
    spec = 2 * t * (nt // 2 + 1) / nt                    # half spectrum, complex, per DOF
    return {
        "residual": 8 + t,            # read U (f64), write s = gamma r
        "check": 0.0,
        "time_fwd": t + spec,         # read s, write S
        "spatial0": 2 * spec, "spatial1": 2 * spec, "spatial2": 2 * spec,   # read + write S
        "time_inv": spec + 16,        # read S, read + write U (f64)
        "setup": 8.0,
    }


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples (the JSON line carries their summary)
        self.path = os.path.join(tempfile.gettempdir(), f"pint_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "10"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): run single-threaded in a child
# ----------------------------------------------------------------------------
def cpu_worker(workload: str, alpha: float, budget_s: float, seed: int, samples: int = 1) -> dict:
    """Time the oracle's sequential solve on a bounded sample of the workload:
    the banded LU factorization plus as many time steps as fit in budget_s,
    extrapolated to the full N_t-step solve (DOF/s).  With samples > 1 the
    whole measurement is repeated that many times in this process and every
    sample's extrapolated solve time is returned (`seconds_samples`)."""
    if samples > 1:
        runs = [cpu_worker(workload, alpha, budget_s, seed) for _ in range(samples)]
        out = dict(runs[-1])
        out["seconds_samples"] = [r["seconds_full_solve"] for r in runs]
        return out
    import numpy as np
    import scipy.sparse as sp

    from oracle import pint_oracle as O
    wl = WORKLOADS[workload]
    p = O.Problem(**{k: wl[k] for k in ("equation", "dim", "nx", "ny", "bc", "eps", "beta", "T", "nt",
                                         "n_windows")}, alpha=alpha)
    u0 = make_u0(wl, seed)
    if p.equation == O.CAHN_HILLIARD:
        t0 = time.perf_counter()
        n = 0
        u = u0.copy()
        while n < p.nt and (n == 0 or time.perf_counter() - t0 < budget_s):
            u, _ = O.ch_step_newton(p, u)
            n += 1
        t = time.perf_counter() - t0
        total = t / n * p.nt
        sample = f"{n} of {p.nt} Newton BE steps"
    else:
        A = O.operator_A(p)
        I = sp.identity(A.shape[0], format="csr")
        bw = 2 if p.dim == 1 else 2 * p.nx
        t0 = time.perf_counter()
        lu = O.BandedLU(I / p.dt + A, bw, bw)
        tf = time.perf_counter() - t0
        rhs = (I / p.dt).tocsr()
        u = u0.copy()
        n = 0
        t1 = time.perf_counter()
        while n < p.nt and (n == 0 or time.perf_counter() - t1 < budget_s):
            u = lu.solve(rhs @ u)
            n += 1
        ts = (time.perf_counter() - t1) / n
        total = tf + ts * p.nt
        sample = (f"banded LU factorization ({tf:.2f} s) + {n} of {p.nt} backward-Euler steps "
                  f"({ts * 1e3:.1f} ms each), extrapolated to the full {p.nt}-step solve")
    dof = p.nspace * p.nt
    _ = np
    return {"value": dof / total, "seconds_full_solve": total, "sample": sample, "cores": 1}


def run_cpu_worker(workload: str, alpha: float, budget_s: float, seed: int = 0, samples: int = 1) -> dict:
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", workload,
           "--alpha", str(alpha), "--cpu-budget", str(budget_s), "--seed", str(seed), "--cpu-samples", str(samples)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(f"cpu worker failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------
# Replicas (N > 1): host-side pieces, also exercised by the CPU gloo tests
# ----------------------------------------------------------------------------
def replica_seed(seed: int, rank: int) -> int:
    """Input seed of a replica: every rank solves its own instance of the workload."""
    return seed + rank


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest of the ranks' values (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, dof_per_rank: int, seconds: float) -> float:
    """Space-time DOF/s of the whole job: all ranks' DOF over the slowest rank's time."""
    return world * dof_per_rank / seconds


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
ORACLE_MAX_BAND_WORK = 3e10   # nspace * bandwidth^2 above which the sequential oracle is not run here


def oracle_solution_worker(workload: str, seed: int, out_path: str) -> dict:
    """The oracle's sequential solution of the workload's input (linear equations:
    backward Euler with banded LU), saved to out_path (.npy), for the error of
    every timed GPU solve against it.  Runs in its own process."""
    import numpy as np

    from oracle import pint_oracle as O
    wl = WORKLOADS[workload]
    p = O.Problem(**{k: wl[k] for k in ("equation", "dim", "nx", "ny", "bc", "eps", "beta", "T", "nt",
                                         "n_windows")})
    u0 = make_u0(wl, seed)
    t0 = time.perf_counter()
    U = O.sequential(p, u0)[-p.nt:]
    np.save(out_path, U)
    return {"seconds": time.perf_counter() - t0}


def oracle_feasible(wl: dict) -> bool:
    if wl["equation"] not in ("linear_ch", "biharmonic") or wl.get("n_windows", 1) != 1:
        return False
    ns = wl["nx"] * (wl["ny"] if wl["dim"] == 2 else 1)
    bw = 2 if wl["dim"] == 1 else 2 * wl["nx"]
    return ns * bw * bw <= ORACLE_MAX_BAND_WORK and ns * wl["nt"] <= 2**24


def start_oracle_worker(workload: str, seed: int):
    path = os.path.join(tempfile.gettempdir(), f"pint_oracle_{workload}_{seed}_{os.getpid()}.npy")
    # it runs beside the timed GPU passes: few threads at low priority, so that
    # the host thread that launches the solves and reads their status is not
    # kept waiting for a core (the timed region ends with an event recorded
    # after the solve's final synchronization)
    nthr = "2"
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS=nthr, OPENBLAS_NUM_THREADS=nthr,
               MKL_NUM_THREADS=nthr)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", "--workload", workload, "--seed", str(seed),
           "--oracle-out", path]
    proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)
    return proc, path


def finish_oracle_worker(handle):
    """The oracle solution (numpy array) or the reason it is missing."""
    import numpy as np
    proc, path = handle
    out, err = proc.communicate()
    if proc.returncode != 0:
        return None, f"oracle worker failed: {err[-500:]}"
    try:
        ref = np.load(path)
        info = json.loads(out.strip().splitlines()[-1])
    finally:
        try:
            os.remove(path)
        except OSError:
            pass
    return ref, info


def short_serving_sample(args, stream) -> dict:
    """p50/p99 latency and DOF/s of a served Poisson stream at two rates (about a
    second each), requests drawn from the batched-instance distribution."""
    import numpy as np

    from paper_2304_14021_gb300 import serve, synth
    pool = synth.batched_instances(64, args.seed + 1, alpha=args.alpha, max_dof=2**22)
    rng = np.random.default_rng(args.seed)
    srv = serve.Server(hbm_budget_bytes=150e9, max_slots=32, precision=args.precision, tol=args.tol,
                       tol_update=args.tol_update)

    def stream_at(rate, n):
        t_next = time.perf_counter()
        futs = []
        for _ in range(n):
            x = pool[int(rng.integers(0, len(pool)))]
            t_next += rng.exponential(1.0 / rate)
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            f = srv.submit(x["u0"], **x["problem"])
            f.add_done_callback(lambda fu: fu.result().release() if fu.exception() is None else None)
            futs.append(f)
        res = [f.result() for f in futs]
        rep = srv.report(res)
        return {"rate_req_s": rate, "n": rep["n"], "p50_ms": rep["p50_s"] * 1e3, "p99_ms": rep["p99_s"] * 1e3,
                "dof_per_s": rep["dof_per_s"], "failed": rep["failed"]}

    stream_at(200, 64)                                   # warm-up: solver entries and graphs per shape
    rows = [stream_at(100, 100), stream_at(1000, 300)]
    srv.close()
    return {"precision": args.precision, "slots": 32, "hbm_budget_bytes": 150e9, "rates": rows,
            "requests": "batched-instance distribution (dof <= 2^22), seeded"}


def main_gpu(args) -> None:
    import numpy as np
    import torch

    from paper_2304_14021_gb300 import build_lib, pint

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    seed = replica_seed(args.seed, rank)       # each replica solves its own instance
    # the oracle's sequential solution, computed in its own process while the GPU is timed
    oracle = start_oracle_worker(args.workload, seed) if (oracle_feasible(wl) and not args.no_oracle) else None
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build_lib.build()
    if dist:
        dist.barrier()

    kw = solver_kw(wl, args)
    u0_np = make_u0(wl, seed)
    stream = torch.cuda.current_stream()

    def make_solver(kwargs):
        sv = pint.Solver(stream=stream, **kwargs)
        if wl["equation"] in ("cahn_hilliard", "cahn_hilliard_eyre"):
            sv.set_adaptive_windows(True)
            if args.varying_jacobian:
                sv.set_varying_jacobian(args.varying_jacobian)
        if args.no_graphs:
            sv.set_graphs(False)
        if args.time_gemm != -1:
            sv.set_time_gemm(args.time_gemm)
        return sv

    s = make_solver(kw)
    nt, ns = s.nt, s.nspace
    nwin = wl.get("n_windows", 1)
    dof = nt * ns * nwin                 # space-time DOF of the whole solve (all windows)
    u0 = torch.from_numpy(u0_np).cuda()
    U = torch.zeros(nt, ns, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    stats = None
    for _ in range(args.warmup):
        stats = s.solve(u0, U)

    def timed_steps(sv, k):
        ts, st_ = [], None
        for _ in range(k):
            flush.zero_()                                # L2 flush outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st_ = sv.solve(u0, U)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, st_

    # Clocks are sampled over every timed pass below (headline, profiled pass,
    # precision forms, the second alpha).
    clocks = ClockSampler(local)
    clocks.start()
    # Pass A (the reported value): the production path, each window's iteration
    # loop as one CUDA graph.
    s.profile_read(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, stats = timed_steps(s, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches_a = s.profile_read(reset=True)
    U_head = U.cpu().numpy()
    # Pass B (per-kernel durations for the roofline): the same steps with CUDA
    # events recorded on the solver's stream around every kernel phase (this
    # uses the host-launched loop, whose kernels are the same).
    s.profile_enable(True)
    s.profile_read(reset=True)
    torch.cuda.synchronize()
    times_b, _ = timed_steps(s, args.steps)
    torch.cuda.synchronize()
    prof = s.profile_read(reset=True)
    # Pass C: two events per iteration only, around the residual with its check
    # and around the whole diagonalized step, so that the step's time is not
    # inflated by event records between its kernels.
    s.profile_enable(2)
    s.profile_read(reset=True)
    torch.cuda.synchronize()
    timed_steps(s, args.steps)
    torch.cuda.synchronize()
    prof_c = s.profile_read(reset=True)
    s.profile_enable(False)
    ms = statistics.mean(times)
    ms_b = statistics.mean(times_b)
    ms = max_over_ranks(ms, dist, "cuda")

    # The other precision forms and the second alpha on the same input, each
    # with its own warm-up and timed repeats; results kept for the error check.
    variants, results = {}, {"headline": U_head}
    if not args.no_variants:
        alpha0 = wl.get("alpha", args.alpha)
        runs = [(prec, alpha0) for prec in ("fp64", "mixed", "mixed_ff") if prec != args.precision]
        if "alpha" not in wl:
            runs += [(prec, a) for prec in (args.precision,) for a in (1e-3,) if a != alpha0]
        for prec, a in runs:
            name = prec if a == alpha0 else f"{prec}_alpha{a:g}"
            kwv = dict(solver_kw(wl, args, prec), alpha=a)
            sv = make_solver(kwv)
            try:
                for _ in range(2):
                    sv.solve(u0, U)
                tv, st_v = timed_steps(sv, args.variant_steps)
            finally:
                sv.close()
            results[name] = U.cpu().numpy()
            mv = statistics.mean(tv)
            variants[name] = {"precision": prec, "alpha": a, "ms_per_step": mv, "value": dof / (mv * 1e-3),
                              "timed_steps": len(tv), "iterations": st_v["iters"],
                              "final_rel_residual": st_v["rel_residual"]}
    clk = clocks.stop()

    # The oracle's process ends before the end-to-end timing, whose host-side
    # work (the call, the copy into host memory) it would otherwise compete with.
    oracle_res = finish_oracle_worker(oracle) if oracle is not None else None

    # End to end through the host-buffer entry point: H2D of u0 and D2H of U inside.
    e2e_s = None
    if not args.no_e2e:
        U_host = torch.zeros(nt, ns, dtype=torch.float64).pin_memory().numpy()
        u0_host = torch.from_numpy(u0_np.copy()).pin_memory().numpy()
        s.solve_host(u0_host, U_host)
        e2e_times = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.solve_host(u0_host, U_host)
            e2e_times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.mean(e2e_times), dist, "cuda")

    # Solve latency of the headline workload over the timed steps, and a short
    # serving sample: Poisson arrivals at two rates drawn from the batched
    # distribution, continuous batching with admission by HBM footprint.
    lat_sorted = sorted(times)

    def pct(v, q):
        return v[min(len(v) - 1, int(q * len(v)))]

    latency = {"p50_ms": pct(lat_sorted, 0.5), "p99_ms": pct(lat_sorted, 0.99), "max_ms": lat_sorted[-1],
               "solves": len(lat_sorted)}
    serving = None
    if not args.no_serving and world == 1:
        serving = short_serving_sample(args, stream)

    # Per-phase times and the rooflines.  Per-launch time = phase time / launches
    # that did work (launches that found the solve already converged are excluded).
    bpd = phase_bytes_per_dof(args.precision, nt)
    # DOF one launch processes: a window, or under the adaptive window policy a
    # segment (approximated by the mean segment size of the solve)
    dof_l = dof / max(1, stats.get("segments", 1)) if nwin > 1 or stats.get("segments", 1) > 1 else dof
    iters_per_step = stats["iters"]
    zero_start = args.init == 2 and not wl["equation"].startswith("cahn_hilliard")   # CH starts from u0
    res_evals = iters_per_step + (0 if zero_start else 1)   # the zero start skips the first residual
    active = {k: (args.steps * (res_evals if k == "residual" else iters_per_step)
                  if k not in ("setup", "check") else prof[k]["launches"]) for k in prof}
    dom = max((k for k in prof if prof[k]["launches"] > 0 and k != "check"), key=lambda k: prof[k]["ms"])
    per_launch_ms = prof[dom]["ms"] / max(1, active[dom])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_src = "MEASURED_PEAKS.json hbm_gbs (measured)"
    except Exception:
        peak_src = "fallback 6800 GB/s (MEASURED_PEAKS.json absent)"
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    ach = bpd[dom] * dof_l / (per_launch_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": _kernel_traffic(dom, args.precision, args.workload), "bytes_per_dof": bpd[dom],
            "per_launch_us": per_launch_ms * 1e3, "peak_note": peak_src}
    if dom == "residual" and args.precision == "mixed_ff":
        # secondary: FP32 lane-operation occupancy of the float-float residual (nominal peak)
        fp32_ops_peak = 152 * 128 * 2.070e9 / 1e12
        ops = ff_residual_ops_per_dof(wl["equation"], wl["dim"]) * dof_l
        roof["fp32_issue"] = {"achieved": ops / (per_launch_ms * 1e-3) / 1e12, "peak": fp32_ops_peak,
                              "unit": "T FP32 lane ops/s", "ops_per_dof": ops / dof_l,
                              "note": "nominal 152 SMs x 128 lanes x 2.07 GHz"}
    # The diagonalized step (Steps 1-3 of Eq. 2.8: time FFT, spatial solves,
    # inverse FFT with the unscaling and update) against the strict minimum of
    # one read of the residual and one write of the correction: 8 B/DOF in the
    # mixed forms, 16 in FP64.
    step_ms_iter = prof_c["time_fwd"]["ms"] / max(1, args.steps * iters_per_step)
    roof["diag_step_us_per_iteration_phase_events"] = (sum(prof[k]["ms"] for k in STEP_PHASES)
                                                       / max(1, args.steps * iters_per_step) * 1e3)
    roof["residual_check_us_per_evaluation"] = prof_c["residual"]["ms"] / max(1, args.steps * res_evals) * 1e3
    step_bytes = (8 if args.precision in ("mixed", "mixed_ff") else 16) * dof_l
    roof["diag_step_us_per_iteration"] = step_ms_iter * 1e3
    roof["diag_step_bytes_per_dof"] = step_bytes / dof_l
    roof["diag_step_frac"] = step_bytes / (step_ms_iter * 1e-3) / 1e9 / hbm_peak
    roof["diag_step_kernel_bytes_frac"] = (sum(bpd[k] for k in STEP_PHASES if prof[k]["launches"] > 0) * dof_l
                                           / (step_ms_iter * 1e-3) / 1e9 / hbm_peak)
    phases = {}
    for k, v in prof.items():
        if v["launches"] == 0:
            continue
        t_l = v["ms"] / max(1, active[k])
        phases[k] = {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                     "us_per_active_launch": t_l * 1e3,
                     "hbm_frac": (bpd[k] * dof_l / (t_l * 1e-3) / 1e9 / hbm_peak) if bpd.get(k) else None}
    launches_total = sum(v["launches"] for v in launches_a.values())

    if rank == 0:
        errs, oracle_info = None, None
        if oracle_res is not None:
            ref, oracle_info = oracle_res
            if ref is not None:
                errs = {name: float(np.max(np.abs(Ux - ref)) / np.max(np.abs(ref))) for name, Ux in results.items()}
                for name, v in variants.items():
                    v["err_vs_oracle"] = errs.get(name)
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            hc = host_cpu()
            try:
                cpu = run_cpu_worker(args.workload, args.alpha, args.cpu_budget, args.seed)
                cpu = {"value": cpu["value"], "unit": "space-time DOF/s", "cores": cpu["cores"], "kind": "oracle",
                       "sample": cpu["sample"], **hc}
            except Exception as ex:  # report, do not hide
                cpu = {"value": None, "unit": "space-time DOF/s", "cores": 1, "kind": "oracle",
                       "sample": f"failed: {ex}", **hc}
        dtype = {"mixed_ff": "f32 (float-float iterate)", "mixed": "f64 residual/scaling/update + c64 transforms",
                 "fp64": "f64"}[args.precision]
        out = {
            "metric": "space-time DOF/s at rel. residual 1e-8",
            "value": whole_job_value(world, dof, ms * 1e-3),
            "unit": "space-time DOF/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": dtype,
            "data": "synthetic",
            "config": {"workload": args.workload, "precision": args.precision, "alpha": wl.get("alpha", args.alpha),
                       "tol": args.tol, "init": "zero" if zero_start else "u0", "dof_per_gpu": dof,
                       "iterations": stats["iters"], "segments": stats.get("segments"),
                       "varying_jacobian": args.varying_jacobian or None,
                       "final_rel_residual": stats["rel_residual"], "l2": "flushed between steps",
                       "time_transforms": {0: "fft", 1: "tensor-core DFT (step 1), fft (step 3)",
                                           2: "fft (step 1), tensor-core DFT (step 3)",
                                           3: "tensor-core DFT (steps 1, 3)"}[stats.get("time_gemm", 0)],
                       "spatial": "fused 2-D slice kernel" if stats.get("fused_spatial") else "separate passes",
                       "autotuner": "choices from the table" if stats.get("tune_cached") else "measured for this handle",
                       "parallelism": f"replicas x{world}"},
            "latency": latency,
            "serving": serving,
            "err_vs_oracle": (errs or {}).get("headline"),
            "oracle": oracle_info if oracle is not None else "not run (size or equation outside the CPU oracle's reach)",
            "e2e": ({"value": whole_job_value(world, dof, e2e_s), "unit": "space-time DOF/s",
                     "h2d_bytes_per_step": ns * 8,
                     "d2h_bytes_per_step": nt * ns * 8} if e2e_s else None),
            "gpu_launches": launches_total,
            "ms_per_step_profiled_pass": ms_b,
            "roofline": roof,
            "phases": phases,
            "variants": variants,
            "speedup_vs_fp64": (variants["fp64"]["ms_per_step"] / ms) if "fp64" in variants else None,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


def _sync_time(torch, fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def main_batched(args) -> None:
    """64 seeded independent instances of mixed equations and sizes solved
    concurrently (pint_solve_batch: one host thread and one stream per instance,
    each window's iteration loop one CUDA graph).  Reports aggregate DOF/s beside
    the same instances solved one at a time, and one at a time in plain FP64."""
    import torch

    from paper_2304_14021_gb300 import build_lib, pint, synth
    build_lib.build()
    torch.cuda.set_device(0)
    inst = synth.batched_instances(64, args.seed, alpha=args.alpha)
    dof = sum(x["dof"] for x in inst)
    streams = [torch.cuda.Stream() for _ in inst]

    def kw(x, prec):
        return dict(x["problem"], precision=prec, tol=args.tol, max_iter=250, init_guess=2,
                    tol_update=args.tol_update)

    u0s = [torch.from_numpy(x["u0"]).cuda() for x in inst]
    Us = [torch.zeros(x["problem"]["nt"], x["u0"].size, dtype=torch.float64, device="cuda") for x in inst]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    solvers = [pint.Solver(stream=st, **kw(x, args.precision)) for st, x in zip(streams, inst)]
    for _ in range(args.warmup):
        pint.solve_batch(solvers, u0s, Us)
    times, stats = [], None
    for _ in range(args.steps):
        flush.zero_()
        t, stats = _sync_time(torch, lambda: pint.solve_batch(solvers, u0s, Us))
        times.append(t)
    t_batch = statistics.mean(times)
    t_seq, _ = _sync_time(torch, lambda: [s.solve(u, U, check=False) for s, u, U in zip(solvers, u0s, Us)])
    iters = [st["iters"] for st in stats]
    for s in solvers:
        s.close()
    fp = [pint.Solver(stream=st, **kw(x, "fp64")) for st, x in zip(streams, inst)]
    for s, u, U in zip(fp, u0s, Us):
        s.solve(u, U, check=False)                      # graph capture outside the timing
    t_fp64, _ = _sync_time(torch, lambda: [s.solve(u, U, check=False) for s, u, U in zip(fp, u0s, Us)])
    for s in fp:
        s.close()
    bytes_alg = sum(64.5 * x["dof"] * it for x, it in zip(inst, iters))
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    out = {"metric": "space-time DOF/s at rel. residual 1e-8 (64 independent instances)", "value": dof / t_batch,
           "unit": "space-time DOF/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t_batch * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": args.precision, "data": "synthetic",
           "config": {"workload": "batched_64", "instances": len(inst), "total_dof": dof, "precision": args.precision,
                      "alpha": args.alpha, "tol": args.tol, "tol_update": args.tol_update,
                      "failed": sum(1 for st in stats if st["rc"] != 0),
                      "stopped_on_residual": sum(1 for st in stats if st["rc"] == 0 and st["rel_residual"] <= args.tol),
                      "iterations_total": sum(iters), "timing": "host wall clock between device synchronizations"},
           "one_at_a_time": {"ms": t_seq * 1e3, "value": dof / t_seq, "speedup_of_batch": t_seq / t_batch},
           "one_at_a_time_fp64": {"ms": t_fp64 * 1e3, "value": dof / t_fp64, "speedup_of_batch": t_fp64 / t_batch},
           "aggregate_algorithmic_hbm_frac": bytes_alg / t_batch / 1e9 / hbm}
    print(json.dumps(out), flush=True)


def main_serving(args) -> None:
    """Poisson request streams (rates swept) drawn from the batched-instance
    distribution, served with continuous batching and admission by HBM
    footprint; p50/p99 latency and DOF/s per rate, beside a one-at-a-time
    plain-FP64 server."""
    import numpy as np
    import torch

    from paper_2304_14021_gb300 import build_lib, serve, synth
    build_lib.build()
    torch.cuda.set_device(0)
    pool = synth.batched_instances(256, args.seed + 1, alpha=args.alpha)
    rng = np.random.default_rng(args.seed)

    def run(rate, n, slots, precision, budget):
        srv = serve.Server(hbm_budget_bytes=budget, max_slots=slots, precision=precision, tol=args.tol,
                           tol_update=args.tol_update)
        t_next = time.perf_counter()
        futs = []
        for i in range(n):
            x = pool[int(rng.integers(0, len(pool)))]
            t_next += rng.exponential(1.0 / rate)
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            f = srv.submit(x["u0"], **x["problem"])
            # the solution's bytes go back to the admission budget as soon as it is done
            f.add_done_callback(lambda fu: fu.result().release() if fu.exception() is None else None)
            futs.append(f)
        res = [f.result() for f in futs]
        rep = srv.report(res)
        srv.close()
        rep["rate_req_s"] = rate
        return rep

    run(50, 16, 8, args.precision, 150e9)            # warm-up (module load, graph capture paths)
    rows = []
    for rate in (10, 30, 100, 300, 1000, 2000):
        n = int(min(args.serve_max_requests, max(8, rate * args.serve_seconds)))
        rows.append(run(rate, n, 32, args.precision, 150e9))
    base = run(10, int(min(args.serve_max_requests, max(8, 10 * args.serve_seconds))), 1, "fp64", 150e9)
    best = max(rows, key=lambda r: r["dof_per_s"])
    out = {"metric": "p50/p99 solve latency and DOF/s under Poisson arrivals", "value": best["dof_per_s"],
           "unit": "space-time DOF/s", "n_gpus": 1, "higher_is_better": True, "dtype": args.precision,
           "data": "synthetic", "config": {"workload": "serving", "slots": 32, "hbm_budget_bytes": 150e9,
                                           "seconds_per_rate": args.serve_seconds,
                                           "max_requests_per_rate": args.serve_max_requests},
           "rates": rows, "baseline_fp64_one_at_a_time": base}
    print(json.dumps(out), flush=True)


REFERENCE_TOTAL_S = 150.0   # wall-time target of the whole reference-arm run


def main_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # All warm-up and timed samples run in one single-threaded worker process; each
    # sample's time-step budget shrinks with their number so that the whole run
    # stays within about three minutes (each sample also pays the LU factorization).
    n = args.warmup + args.steps
    budget = max(0.3, min(args.cpu_budget, REFERENCE_TOTAL_S / n - 2.0))
    res = run_cpu_worker(args.workload, args.alpha, budget, args.seed, samples=n)
    times = res["seconds_samples"][args.warmup:] if n > 1 else [res["seconds_full_solve"]]
    wl = WORKLOADS[args.workload]
    dof = wl["nx"] * (wl["ny"] if wl["dim"] == 2 else 1) * wl["nt"]
    secs = statistics.mean(times)
    v = dof / secs
    out = {"impl": "reference", "metric": "space-time DOF/s at rel. residual 1e-8", "value": v,
           "unit": "space-time DOF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "precision": "fp64 (oracle)", "alpha": args.alpha},
           "cpu_baseline": {"value": v, "unit": "space-time DOF/s", "cores": 1, "kind": "oracle",
                            "sample": res["sample"], **host_cpu()},
           "e2e": {"value": v, "unit": "space-time DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_ff", "fp64"])
    ap.add_argument("--variant-steps", type=int, default=10,
                    help="timed repeats of each other precision form and of the second alpha")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle's sequential solution (error check)")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving sample of the headline line")
    ap.add_argument("--time-gemm", type=int, default=-1, choices=[-1, 0, 1],
                    help="time transforms: -1 chosen by measurement per handle, 0 FFT, 1 tensor-core DFT products")
    ap.add_argument("--oracle-worker", action="store_true")
    ap.add_argument("--oracle-out", default="")
    ap.add_argument("--init", type=int, default=2, choices=[0, 2],
                    help="initial iterate: 0 = u0 at every level, 2 = zero")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-launched iteration loop (profilers then see every kernel)")
    ap.add_argument("--alpha", type=float, default=1e-2)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["batched_64", "serving"])
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--tol-update", type=float, default=1e-10,
                    help="batched/serving: also stop when ||delta||/||U|| <= this (stiff instances)")
    ap.add_argument("--serve-max-requests", type=int, default=300)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=8.0)
    ap.add_argument("--varying-jacobian", type=int, default=0,
                    help="Cahn-Hilliard: inner GMRES length of the space-varying Jacobian in Step 2 (0 = scalar mean)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-worker", action="store_true")
    ap.add_argument("--cpu-samples", type=int, default=1)
    args = ap.parse_args()
    if args.cpu_worker:
        print(json.dumps(cpu_worker(args.workload, args.alpha, args.cpu_budget, args.seed, args.cpu_samples)))
        return
    if args.oracle_worker:
        try:
            os.nice(15)
        except OSError:
            pass
        print(json.dumps(oracle_solution_worker(args.workload, args.seed, args.oracle_out)))
        return
    if args.impl == "reference":
        main_reference(args)
        return
    if args.workload == "batched_64":
        main_batched(args)
        return
    if args.workload == "serving":
        main_serving(args)
        return
    main_gpu(args)


if __name__ == "__main__":
    main()
