#!/usr/bin/env python3
"""Factor + solve throughput of the IFMM on GB300 (unknowns/s), one JSON line on rank 0.

Workload: N = 2^20 points i.i.d. uniform in [0,1]^2 (seeded), uniform quadtree of depth 7
(16,384 leaves x 64 points), K(x,y) = 1/|x-y| off the diagonal, A_ii = sqrt(N), Chebyshev 4x4
(initial rank 16), fill compression eps = 1e-6 (matrix-scale threshold), 32 right-hand sides,
GMRES-based FP64 refinement (preconditioner = the IFMM solve) until the estimated relative error
is <= 1e-7; the error to the manufactured solution is measured and reported.

Precisions (--precision): mixed_solve (default) = FP64 elimination, solve phase on the FP32 pipe in
double-float arithmetic (replay of double-float copies of the factors and double-float FMM matvec
inside GMRES, FP64 residual at every restart, FP64 update); fp64 = every step in FP64; mixed = FP32
elimination (FP32 Schur updates, panels and compression, FP64 pivot blocks, residuals and
refinement). The precisions not chosen are timed alongside (one step each) and reported with their
errors.

One step = ifmm_factor (every level, Algorithm 1, plus the level-1 system) + ifmm_solve of the
32 right-hand sides with refinement (Algorithm 2 replay + FP64 matvec per refinement step).
value = N / step time (whole job: N x ranks / max step time over ranks for --gpus > 1, where
every rank solves its own independent system: replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "factor+solve unknowns/s at N=2^20, err<=1e-6, mixed vs FP64 GPU; % of roofline"
WORKLOAD = dict(N=1 << 20, depth=7, cheb_p=4, eps=1e-6, nrhs=32, seed=1411, tau_ref=1, refine_tol=1e-7,
                refine_maxit=120, refine_restart=60, refine_inner=1e-4)
# bounded CPU sample of the same workload family for the oracle (same points per leaf, settings)
CPU_SAMPLE = dict(N=1 << 16, depth=5, cheb_p=4, eps=1e-6, nrhs=32, seed=1411, tau_ref=1, refine_tol=1e-7,
                  refine_maxit=120, refine_restart=60)
# the same on one thread, smaller (about 10 s)
CPU_SAMPLE_1T = dict(CPU_SAMPLE, N=1 << 14, depth=4)


PRECISION_DESC = {
    "fp64": "FP64",
    "mixed_solve": ("FP64 elimination, double-float (FP32-pair) solve phase on the FP32 pipe (replay + matvec in "
                    "GMRES), FP64 final residual and update"),
    "mixed": "FP32 elimination (FP64 pivots) + FP64 refinement",
}


def precision_code(ifmm, prec):
    return {"fp64": ifmm.IFMM_FP64, "mixed": ifmm.IFMM_MIXED, "mixed_solve": ifmm.IFMM_MIXED_SOLVE}[prec]


def workload_desc(w, precision):
    return (f"N={w['N']} uniform [0,1]^2, quadtree depth {w['depth']} ({4 ** w['depth']} leaves), "
            f"1/r + sqrt(N) I, Chebyshev {w['cheb_p']}x{w['cheb_p']} (rank {w['cheb_p'] ** 2}), "
            f"eps {w['eps']:g} (matrix-scale threshold), {w['nrhs']} RHS, {precision}")


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline of the GPU arm)
# ------------------------------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def oracle_gmres(o, b, tol, restart, maxit):
    """Left-preconditioned GMRES(restart) on A~ x = b with the oracle's FMM matvec as A~ and its
    IFMM solve as M^{-1}: the refinement the library runs (same recurrence: classical Gram-Schmidt
    twice, Givens rotations, one independent Krylov space per right-hand side sharing every operator
    application), stopped when max_j ||M^{-1}(b_j - A~ x_j)|| / ||x_j|| <= tol. Returns (x, inner
    iterations, preconditioner applications)."""
    import numpy as np

    N, nrhs = b.shape
    x = np.zeros_like(b)
    it = applications = 0
    xn = None
    while True:
        r = b if it == 0 and xn is None else b - o.matvec(x)
        z = o.solve(r)
        applications += 1
        beta = np.linalg.norm(z, axis=0)
        if xn is None:
            xn = beta.copy()
        est = float(np.max(np.where(xn > 0, beta / np.maximum(xn, 1e-300), 0.0)))
        if est <= tol or it >= maxit:
            break
        V = [z / np.where(beta > 0, beta, 1.0)]
        H = np.zeros((restart + 1, restart, nrhs))
        cs, sn = np.zeros((restart, nrhs)), np.zeros((restart, nrhs))
        g = np.zeros((restart + 1, nrhs))
        g[0] = beta
        k = 0
        for j in range(restart):
            w = o.solve(o.matvec(V[j]))
            applications += 1
            for _ in range(2):
                for i in range(j + 1):
                    hij = np.sum(V[i] * w, axis=0)
                    H[i, j] += hij
                    w = w - V[i] * hij
            hn = np.linalg.norm(w, axis=0)
            for i in range(j):
                a, bb = H[i, j].copy(), H[i + 1, j].copy()
                H[i, j] = cs[i] * a + sn[i] * bb
                H[i + 1, j] = -sn[i] * a + cs[i] * bb
            den = np.hypot(H[j, j], hn)
            cs[j] = np.where(den > 0, H[j, j] / np.where(den > 0, den, 1.0), 1.0)
            sn[j] = np.where(den > 0, hn / np.where(den > 0, den, 1.0), 0.0)
            H[j, j] = den
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            V.append(w / np.where(hn > 0, hn, 1.0))
            it += 1
            k = j + 1
            est = float(np.max(np.abs(g[j + 1]) / np.maximum(xn, 1e-300)))
            if est <= tol or it >= maxit:
                break
        y = np.zeros((k, nrhs))
        for i in range(k - 1, -1, -1):
            acc = g[i] - np.sum(H[i, i + 1:k] * y[i + 1:k], axis=0)
            y[i] = np.where(H[i, i] != 0, acc / np.where(H[i, i] != 0, H[i, i], 1.0), 0.0)
        for i in range(k):
            x = x + V[i] * y[i]
        xn = np.linalg.norm(x, axis=0)
        if it >= maxit:
            break
    return x, it, applications


def oracle_step(w, threads=0, parts=None):
    """One oracle factor + refined solve (GMRES, as the library refines) on the bounded sample;
    returns (seconds, error). `parts` (a dict), if given, receives the build, factor and solve
    seconds and the GMRES iteration count."""
    import numpy as np

    from oracle import oracle as O
    from paper_1407_1572_gb300 import inputs
    N = w["N"]
    pts = inputs.uniform_points(w["seed"], N)
    prm = O.make_params(w["depth"], w["cheb_p"], O.K_INV_R, eps=w["eps"], diag=math.sqrt(N), tau_ref=w["tau_ref"],
                        threads=threads)
    tb = time.perf_counter()
    o = O.Oracle(pts, prm)
    tb = time.perf_counter() - tb
    xs = inputs.rhs(w["seed"] + 1, N, w["nrhs"])
    b = o.matvec(xs)
    t0 = time.perf_counter()
    o.factor()
    tf = time.perf_counter() - t0
    x, its, _ = oracle_gmres(o, b, w["refine_tol"], w["refine_restart"], w["refine_maxit"])
    dt = time.perf_counter() - t0
    err = float(np.max(np.linalg.norm(x - xs, axis=0) / np.linalg.norm(xs, axis=0)))
    if parts is not None:
        parts.update(t_build_s=tb, t_factor_s=tf, t_solve_s=dt - tf, gmres_iters=its)
    return dt, err


def oracle_headline_sample(w, gpu_iters):
    """The oracle on the headline workload itself (same N, points and settings): its factorisation
    timed in full, one 32-column IFMM solve and one FMM matvec timed once, and the solve phase taken
    as the GPU step's number of preconditioned matvecs times (solve + matvec) plus one solve. Returns
    a dict of seconds."""
    from oracle import oracle as O
    from paper_1407_1572_gb300 import inputs
    N = w["N"]
    pts = inputs.uniform_points(w["seed"], N)
    o = O.Oracle(pts, O.make_params(w["depth"], w["cheb_p"], O.K_INV_R, eps=w["eps"], diag=math.sqrt(N),
                                    tau_ref=w["tau_ref"]))
    b = inputs.rhs(w["seed"] + 1, N, w["nrhs"])
    t0 = time.perf_counter()
    o.factor()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    x = o.solve(b)
    ts1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.matvec(x)
    tm1 = time.perf_counter() - t0
    return {"t_factor_s": tf, "t_solve_once_s": ts1, "t_matvec_once_s": tm1,
            "t_solve_modelled_s": (gpu_iters + 1) * ts1 + gpu_iters * tm1}


def cpu_baseline_entry(gpu_iters=None, full=False):
    """The oracle timed on this host. At the headline size (gpu_iters given): the oracle's factor timed
    in full and its refined solve sampled (one solve and one FMM matvec, scaled by the GPU step's GMRES
    iteration count), so the ratio compares the same factorisation and the same number of operator
    applications per unknown; on a bounded sample of the headline workload (65,536 of its points'
    density: same points per leaf and settings, about 10 s), or with `full` on the bench's own 2^20
    points (about 3 minutes). Otherwise the complete factor + GMRES-refined solve on the 65,536-point
    sample. All add one thread on 16,384 points."""
    w1 = CPU_SAMPLE_1T
    dt1, err1 = oracle_step(w1, threads=1)
    single = {"value": w1["N"] / dt1, "unit": "unknowns/s", "cores": 1,
              "sample": f"factor + GMRES-refined solve on N={w1['N']} (depth {w1['depth']}), one thread, {dt1:.1f} s, "
                        f"err {err1:.1e}"}
    if gpu_iters is None:
        parts = {}
        w = CPU_SAMPLE
        dt, err = oracle_step(w, parts=parts)
        return {"value": w["N"] / dt, "unit": "unknowns/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                "cpu_model": cpu_model(),
                "sample": f"oracle factor + GMRES-refined {w['nrhs']}-RHS solve on N={w['N']} (depth {w['depth']}, "
                          f"same settings per leaf), {dt:.1f} s, err {err:.1e}",
                **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in parts.items()},
                "single_thread": single}
    ws = WORKLOAD if full else dict(WORKLOAD, N=CPU_SAMPLE["N"], depth=CPU_SAMPLE["depth"])
    hs = oracle_headline_sample(ws, gpu_iters)
    n = ws["N"]
    total = hs["t_factor_s"] + hs["t_solve_modelled_s"]
    what = (f"the headline workload itself (N={n}, same points and settings)" if full else
            f"a {n}-point sample of the headline workload (depth {ws['depth']}, same points per leaf and settings)")
    return {"value": n / total, "unit": "unknowns/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"oracle on {what}: factor timed in full "
                       f"({hs['t_factor_s']:.1f} s), one {ws['nrhs']}-RHS solve ({hs['t_solve_once_s']:.1f} s) "
                       f"and one FMM matvec ({hs['t_matvec_once_s']:.1f} s) timed and scaled to the GPU step's "
                       f"{gpu_iters} preconditioned matvecs: {total:.1f} s per step"),
            "factor_only_value": n / hs["t_factor_s"], "seconds": {k: round(v, 3) for k, v in hs.items()},
            "single_thread": single}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = CPU_SAMPLE
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_step(w)
    times, errs = [], []
    for _ in range(args.steps):
        dt, err = oracle_step(w)
        times.append(dt)
        errs.append(err)
    ms = 1000.0 * sum(times) / len(times)
    value = w["N"] / (ms / 1000.0)
    sample = (f"oracle (plain FP64 C++, OpenMP over same-colour boxes) on N={w['N']} (depth {w['depth']}), "
              f"same settings per leaf; factor + {w['nrhs']}-RHS solve refined by GMRES({w['refine_restart']}) "
              f"as the library refines; err {max(errs):.2e}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(w, "FP64 CPU oracle"), "N": w["N"], "depth": w["depth"],
                       "nrhs": w["nrhs"], "eps": w["eps"], "err": max(errs)},
            "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Arithmetic peaks of the CUDA cores. Measured at run time by the pipe probe (measure/pipe_peaks.cu:
# chains of independent FMAs over 8 blocks per SM, CUDA events), else the unit-count figures at
# 2.07 GHz: FP32 = 152 SMs x 128 lanes x 2 flops; FP64 = 304 DFMA per clock (1.26 TFLOP/s). The
# double-float rate is the FP32 rate at 11 FP32 instructions per multiply-add (exact product, two
# cross terms, exact sum), counted as 2 FP64-equivalent flops per multiply-add.
NOMINAL_PIPES = {"fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64_tflops": 304 * 2 * 2.07e9 / 1e12}


def measure_pipes():
    """FP64 and FP32 FMA rates of this GPU (TFLOP/s) from the pipe probe; None if it cannot run."""
    import ctypes

    try:
        from paper_1407_1572_gb300 import build as _b
        lib = ctypes.CDLL(_b.build_peaks())
        out = (ctypes.c_double * 4)()
        if lib.ifmm_pipe_peaks(out) != 0:
            return None
        return {"fp64_tflops": out[0], "fp32_tflops": out[1], "sms": int(out[2]),
                "how": "measure/pipe_peaks.cu: 8 independent FMA chains per thread, 8 blocks of 256 threads per "
                       "SM, CUDA events, one launch after a warm-up"}
    except (OSError, RuntimeError):
        return None


def pipe_peaks(measured):
    src = "measured (pipe probe)" if measured else "nominal unit counts at 2.07 GHz"
    m = measured or NOMINAL_PIPES
    return {"fp64": m["fp64_tflops"], "fp32": m["fp32_tflops"], "dfl": m["fp32_tflops"] / 11.0, "source": src}


# arithmetic of each factor kernel per precision
ARITH = {
    "fp64": {k: "FP64" for k in ("k_pivot", "k_panel", "k_schur", "k_compress", "k_redirect")},
    "mixed_solve": {"k_pivot": "FP64",
                    "k_panel": "double-float GEMM", "k_schur": "double-float GEMM",
                    "k_compress": "double-float projection GEMMs and Gram-Schmidt column work + FP64 re-orthogonalisation",
                    "k_redirect": "double-float GEMM"},
    "mixed": {k: "FP32" for k in ("k_panel", "k_schur", "k_compress", "k_redirect")} | {"k_pivot": "FP64"},
}


# DRAM traffic of a kernel (dram__bytes_read.sum + dram__bytes_write.sum) per eliminated box, from a
# bounded ncu capture of one leaf-level launch at 65,536 points (profiles/), scaled to a launch of
# the bench by the boxes it eliminates on average (the units of the launch; a leaf box of 64 points
# costs the same at any N); keyed by the SHA-256 of the kernel sources it was taken on, so that it
# reads null once a source differs. Empty: no capture of the current sources.
TRAFFIC = {
    # profiles/k_compress_n65536_mixed.md: one level-5 launch over 110 boxes, 316.60 MB
    ("mixed_solve", "k_compress"): {"bytes_per_box": 316.597248e6 / 110},
    # profiles/k_schur_n65536_mixed.md: one level-5 launch over 110 boxes, 215.90 MB
    ("mixed_solve", "k_schur"): {"bytes_per_box": 215.897088e6 / 110},
}
TRAFFIC_SRC = {
    "ifmm_factor.cu": "fe69162075983cc58219a76574eb447374b915f4ae06e8160de7bfbd55a55876",
    "ifmm_common.cuh": "d7aff101b7cda20e870e39e7916fe24394fab8c076c58869e434e0c44a0b6ecc",
    # the captured header with the refinement launchers' declarations changed (a scratch argument
    # for the fixed-order reductions); nothing the captured kernels compile from changed
    "ifmm_internal.h": "a6f4888f1d3fd7b0af29ad7e5fe75d1aac4eb915db08234f3b6e2b88c0c37d14",
}


def _traffic(precision, name, boxes_per_launch):
    import hashlib
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1407_1572_gb300", "csrc")
    if not TRAFFIC_SRC or not boxes_per_launch:
        return None
    for f, h in TRAFFIC_SRC.items():
        with open(os.path.join(csrc, f), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != h:
                return None
    rec = TRAFFIC.get((precision, name))
    if not rec:
        return None
    return rec["bytes_per_box"] * boxes_per_launch


def _kernel_roofline(stats, precision, i, pipes, boxes=0):
    from paper_1407_1572_gb300.ifmm import FACTOR_KERNELS
    ms, launches, flops = stats["kernel_ms"], stats["kernel_launches"], stats["kernel_flops"]
    name = FACTOR_KERNELS[i]
    nl = max(launches[i], 1)
    t = ms[i] / nl / 1000.0                       # seconds per launch (CUDA events, handle's stream)
    flops_pl = flops[i] / nl
    arith = ARITH[precision][name]
    parts = None
    if name == "k_compress" and precision == "mixed_solve":
        # two pipes in one kernel: the projection products and the Gram-Schmidt's column work (dot
        # products, updates, norms) in double-float on the FP32 pipe, the re-orthogonalisation of
        # each new direction in FP64; the peak is the rate at which the kernel's own mix would run
        # if each part ran at its pipe's peak (time-weighted)
        proj = stats["compress_proj_flops"] / nl
        reorth = stats.get("compress_reorth_flops", 0.0) / nl
        cols = flops_pl - proj - reorth
        t_ideal = (proj + cols) / (pipes["dfl"] * 1e12) + reorth / (pipes["fp64"] * 1e12)
        peak = flops_pl / t_ideal / 1e12 if t_ideal > 0 else pipes["fp64"]
        src = f"time-weighted blend of the double-float ({pipes['dfl']:.2f}) and FP64 ({pipes['fp64']:.2f}) peaks, {pipes['source']}"
        parts = {"projection_flops_per_launch": proj, "gram_schmidt_column_flops_per_launch": cols,
                 "reorthogonalisation_flops_per_launch": reorth,
                 "projection_share_of_flops": proj / max(flops_pl, 1.0)}
    elif name == "k_compress" and precision == "fp64":
        peak, src = pipes["fp64"], f"FP64 pipe, {pipes['source']}"
    elif arith.startswith("double-float GEMM"):
        peak, src = pipes["dfl"], f"double-float rate of the FP32 pipe (11 instructions per multiply-add), {pipes['source']}"
    elif arith == "FP32":
        peak, src = pipes["fp32"], f"FP32 pipe, {pipes['source']}"
    else:
        peak, src = pipes["fp64"], f"FP64 pipe, {pipes['source']}"
    ach = flops_pl / t / 1e12
    traffic = _traffic(precision, name, boxes / nl if boxes else 0)
    out = {"kernel": name, "arith": arith, "share_of_factor_kernels": ms[i] / max(sum(ms), 1e-30),
           "avg_launch_ms": ms[i] / nl, "launches": launches[i], "flops_per_launch": flops_pl,
           "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
           "traffic": traffic, "traffic_unit": "bytes per launch",
           "achieved_dram_gbs": traffic / t / 1e9 if traffic else None, "peak_source": src}
    if parts:
        out.update(parts)
    return out


def roofline(stats, precision, peaks, peak_kind, pipes, boxes=0):
    """Dominant factor kernel (CUDA-event time); `schur` adds the Schur-update kernel, the dense
    contraction of the elimination, against the peak of its own arithmetic. boxes: the boxes one
    factorisation eliminates (all levels), for the traffic per launch."""
    ms = stats["kernel_ms"]
    top = max(range(5), key=lambda i: ms[i])
    out = _kernel_roofline(stats, precision, top, pipes, boxes)
    out["schur"] = _kernel_roofline(stats, precision, 2, pipes, boxes)
    # every factor kernel against the peak of its own arithmetic (CUDA-event time per launch)
    from paper_1407_1572_gb300.ifmm import FACTOR_KERNELS
    out["factor_kernels"] = {}
    for i, name in enumerate(FACTOR_KERNELS):
        k = _kernel_roofline(stats, precision, i, pipes, boxes)
        out["factor_kernels"][name] = {f: k[f] for f in ("arith", "launches", "avg_launch_ms", "achieved", "peak",
                                                         "frac", "share_of_factor_kernels")}
    # the Schur step's algorithmic bytes, for the intensity against HBM
    nl = max(stats["kernel_launches"][2], 1)
    bytes_pl = stats["schur_bytes"] / nl
    sc = out["schur"]
    sc["intensity_flop_per_byte"] = (stats["kernel_flops"][2] / nl) / max(bytes_pl, 1.0)
    sc["hbm_peak_gbs"] = peaks["hbm_gbs"]
    sc["hbm_peak_source"] = f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
    # attainable = min(arithmetic peak, intensity x HBM bandwidth)
    sc["attainable"] = min(sc["peak"], sc["intensity_flop_per_byte"] * peaks["hbm_gbs"] / 1000.0)
    sc["frac_attainable"] = sc["achieved"] / sc["attainable"]
    sc["algorithmic_gbs"] = bytes_pl / (sc["avg_launch_ms"] / 1000.0) / 1e9
    out["pipes"] = pipes
    return out


# the octree workload (d = 3): points uniform in the unit cube, 64 per leaf, 1/r + sqrt(N) I (the 3D
# Laplace kernel), Chebyshev 3 x 3 x 3, eps 1e-6, refined to an estimated error of 1e-7 (2^15 points:
# the 2^18-point octree takes 44 s per step, too long for a bench leg)
OCTREE = dict(N=1 << 15, depth=3, cheb_p=3, eps=1e-6, nrhs=8, seed=1413, refine_tol=1e-7, steps=3)


def run_octree(precision: str):
    """One warm-up and OCTREE['steps'] timed factor + solve steps of the octree workload on this GPU
    (CUDA events on the solver's stream), error against the manufactured solution."""
    import torch

    from paper_1407_1572_gb300 import ifmm, inputs

    o = OCTREE
    N, nrhs = o["N"], o["nrhs"]
    stream = torch.cuda.current_stream()
    pts = inputs.uniform(o["seed"], 3 * N).reshape(N, 3)
    prm = ifmm.default_params(dim=3, depth=o["depth"], cheb_p=o["cheb_p"], eps=o["eps"], diag=math.sqrt(N),
                              precision=precision_code(ifmm, precision), tau_ref=1, refine_tol=o["refine_tol"],
                              refine_maxit=200, refine_restart=60)
    g = ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm, stream)
    xs = torch.from_numpy(inputs.rhs(o["seed"] + 1, N, nrhs).T.copy()).cuda()
    b = torch.empty_like(xs)
    ifmm.ifmm_matvec(g.h, xs.data_ptr(), b.data_ptr(), nrhs, N)
    x = torch.empty_like(xs)

    def step():
        ifmm.ifmm_factor(g.h, allow_overflow=True)
        ifmm.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), nrhs, N, allow_noconv=True)

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(o["steps"]):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / o["steps"]
    st = ifmm.ifmm_get_stats(g.h)
    err = float(((x - xs).norm(dim=1) / xs.norm(dim=1)).max().item())
    g.close()
    return {"value": N / (ms / 1000.0), "unit": "unknowns/s", "ms_per_step": ms, "steps": o["steps"], "warmup": 1,
            "err": err, "meets_err_1e-6": err <= 1e-6, "precision": PRECISION_DESC[precision],
            "t_factor_ms": st["t_factor_ms"], "t_solve_ms": st["t_solve_ms"], "refine_iters": st["refine_iters"],
            "max_rank": st["max_rank"], "device_gb": st["device_bytes"] / 1e9,
            "kernel_ms": dict(zip(ifmm.FACTOR_KERNELS, st["kernel_ms"])),
            "workload": (f"octree: {N} points uniform in the unit cube, depth {o['depth']} (64 per leaf), "
                         f"Chebyshev {o['cheb_p']}^3, 1/r + sqrt(N) I, eps {o['eps']:g}, {nrhs} RHS, "
                         f"refined to {o['refine_tol']:g}")}


BATCH = dict(count=256, seed=1409, nmin=2048, nmax=32768, rhs_min=1, rhs_max=16, cheb_p=4, eps=1e-6, leaf_max=64,
             refine_tol=1e-7, wave=64, workers=48)


def partition_work(work, world: int):
    """Independent systems over `world` ranks: largest work first, each to the rank with the least
    work so far (ties to the lower rank, then the lower index). Returns each rank's indices, sorted."""
    parts = [[] for _ in range(world)]
    load = [0.0] * world
    for i in sorted(range(len(work)), key=lambda i: (-work[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(i)
        load[r] += work[i]
    return [sorted(p) for p in parts]


def aggregate_batched(tf: float, ts: float, err: float, dmin: int, dmax: int, dist, device):
    """A rank's batched results combined over ranks: the job's time is the slowest rank's factor +
    solve time; error and depth range over all systems. Returns (t_total, tf, ts, err, dmin, dmax)."""
    t = reduce_max(tf + ts, dist, device)
    return (t, reduce_max(tf, dist, device), reduce_max(ts, dist, device), reduce_max(err, dist, device),
            -reduce_max(-dmin, dist, device), reduce_max(dmax, dist, device))


def run_batched(precision: str, rank: int = 0, world: int = 1, dist=None):
    """The batched workload (independent uneven systems): 256 systems, N log-uniform in [2048, 32768],
    half uniform clouds and half Gaussian blobs (8 centres, sigma 0.05), automatic depth (fullest
    leaf <= 64 points, empty leaves kept), 1-16 right-hand sides each, 1/r + sqrt(N) I, rank 16,
    eps 1e-6, refined to 1e-7. Systems are built, factored (ifmm_factor_batch) and solved
    (ifmm_solve_batch) in waves of 64, half uniform and half blobs per wave, each system on its own
    stream; one untimed warm-up wave of 16 first. Timed: the batched factor + solve calls, in two
    sweeps: with the fixed launch-split rule, then with the table ifmm_autotune builds (untimed) on
    the first wave's systems; `value` is the tuned sweep's, the fixed rule's is reported beside it. Over
    several ranks every rank runs its share (partition_work on N x nrhs) and the job's time is the
    slowest rank's (strong scaling: the 256 systems are fixed)."""
    import torch

    from paper_1407_1572_gb300 import ifmm, inputs

    c = BATCH
    systems = inputs.batch_systems(seed=c["seed"], count=c["count"], nmin=c["nmin"], nmax=c["nmax"],
                                   rhs_min=c["rhs_min"], rhs_max=c["rhs_max"])
    half = c["count"] // 2
    mine = partition_work([s["points"].shape[0] * s["nrhs"] for s in systems], world)[rank]
    uni = [systems[i] for i in mine if i < half]
    blob = [systems[i] for i in mine if i >= half]

    def wave(sy, tune=False):
        handles, xs_l, bs_l, xo_l = [], [], [], []
        for s in sy:
            n = s["points"].shape[0]
            prm = ifmm.default_params(depth=0, leaf_max=c["leaf_max"], cheb_p=c["cheb_p"], eps=c["eps"],
                                      diag=math.sqrt(n), tau_ref=1, precision=precision_code(ifmm, precision),
                                      refine_tol=c["refine_tol"], refine_maxit=120, refine_restart=60)
            g = ifmm.IFMM(s["points"], ifmm.IFMM_K_INV_R, prm, torch.cuda.Stream())
            xs = torch.from_numpy(inputs.rhs(s["seed"], n, s["nrhs"]).T.copy()).cuda()
            b = torch.empty_like(xs)
            ifmm.ifmm_matvec(g.h, xs.data_ptr(), b.data_ptr(), s["nrhs"], n)
            handles.append(g)
            xs_l.append(xs)
            bs_l.append(b)
            xo_l.append(torch.empty_like(xs))
        torch.cuda.synchronize()
        if tune:   # untimed: the autotuner's table for this wave's launches (ifmm_autotune)
            t0 = time.perf_counter()
            ifmm.ifmm_autotune([g.h for g in handles], workers=c["workers"])
            tune_s.append(time.perf_counter() - t0)
        t1 = time.perf_counter()
        ifmm.ifmm_factor_batch([g.h for g in handles], workers=c["workers"], allow_overflow=True)
        t2 = time.perf_counter()
        ifmm.ifmm_solve_batch([g.h for g in handles], [b.data_ptr() for b in bs_l], [x.data_ptr() for x in xo_l],
                              [s["nrhs"] for s in sy], [s["points"].shape[0] for s in sy], workers=c["workers"],
                              allow_noconv=True)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        err = max(float(((x - xs).norm(dim=1) / xs.norm(dim=1)).max()) for x, xs in zip(xo_l, xs_l))
        depths = [g.stats()["depth"] for g in handles]
        for g in handles:
            g.close()
        return t2 - t1, t3 - t2, err, depths

    tune_s = []
    ifmm.ifmm_autotune_clear()
    if uni or blob:
        wave(uni[:8] + blob[:8])
    if dist:
        dist.barrier()
    per = c["wave"] // 2
    nw = max(-(-len(uni) // per), -(-len(blob) // per))

    def sweep(tuned):
        tf = ts = err = 0.0
        depths = []
        for w in range(nw):
            f_, s_, e_, d_ = wave(uni[w * per:(w + 1) * per] + blob[w * per:(w + 1) * per], tune=tuned and w == 0)
            tf += f_
            ts += s_
            err = max(err, e_)
            depths += d_
        return tf, ts, err, depths

    # the fixed launch rule, then the table the autotuner builds on the first wave (kept for the rest)
    tf0, ts0, err0, _ = sweep(False)
    tf, ts, err, depths = sweep(True)
    table_size = ifmm.ifmm_autotune_size()
    ifmm.ifmm_autotune_clear()
    t0, tf0, ts0, err0, _, _ = aggregate_batched(tf0, ts0, err0, 0, 0, dist, "cuda")
    t, tf, ts, err, dmin, dmax = aggregate_batched(tf, ts, err, min(depths, default=99), max(depths, default=0),
                                                   dist, "cuda")
    n_tot = sum(s["points"].shape[0] for s in systems)
    unk = sum(s["points"].shape[0] * s["nrhs"] for s in systems)
    return {"value": n_tot / t, "unit": "unknowns/s", "systems": c["count"], "N_total": n_tot, "ranks": world,
            "scaling": "strong", "rhs_columns_x_N": unk, "t_factor_s": tf, "t_solve_s": ts, "err": err,
            "meets_err_1e-6": err <= 1e-6, "depth_range": [int(dmin), int(dmax)], "precision": PRECISION_DESC[precision],
            "workers": c["workers"], "timing": "host clock around the blocking batched calls (device synchronised)",
            "autotune": {"table_entries": table_size, "tuning_s": sum(tune_s),
                         "value_fixed_rule": n_tot / t0, "t_factor_s_fixed_rule": tf0, "t_solve_s_fixed_rule": ts0,
                         "err_fixed_rule": err0,
                         "note": "value uses the autotuner's launch splits, tuned (untimed) on the first wave"},
            "workload": ("256 systems, N log-uniform in [2048, 32768], half uniform / half Gaussian blobs "
                         "(8 centres, sigma 0.05), automatic depth (leaf <= 64), 1-16 RHS, 1/r + sqrt(N) I, "
                         "rank 16, eps 1e-6, refined to 1e-7")}


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s point set: every replica solves its own independent system."""
    return base + rank


def reduce_max(v: float, dist, device) -> float:
    """The maximum of v over ranks (all-reduce MAX, then a barrier so that no rank starts the next
    phase early); `dist` None for one process."""
    if dist is None:
        return v
    import torch

    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def reduce_max_ms(ms: float, dist, device) -> float:
    """The step time of the whole job: the maximum over ranks."""
    return reduce_max(ms, dist, device)


def whole_job_value(world: int, n: int, ms: float) -> float:
    """Unknowns per second over all ranks: every rank factors and solves n unknowns per step."""
    return world * n / (ms / 1000.0)


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1407_1572_gb300 import ifmm, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = dict(WORKLOAD)
    if args.n:
        w["N"] = args.n
        w["depth"] = max(2, round(math.log(args.n / 64, 4)))
    N, nrhs = w["N"], w["nrhs"]
    precision = args.precision
    stream = torch.cuda.current_stream()
    ifmm.ifmm_set_compress_cluster(args.compress_cluster)

    def make_solver(prec):
        prm = ifmm.default_params(depth=w["depth"], cheb_p=w["cheb_p"], eps=w["eps"], diag=math.sqrt(N),
                                  precision=precision_code(ifmm, prec),
                                  tau_ref=w["tau_ref"], refine_tol=w["refine_tol"],
                                  refine_maxit=w["refine_maxit"] if prec != "mixed" else 30,
                                  refine_restart=w["refine_restart"], refine_inner=w["refine_inner"],
                                  tc_products=args.tc_products)
        pts = inputs.uniform_points(replica_seed(w["seed"], rank), N)
        return ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm, stream)

    pipes_measured = measure_pipes()   # before any solver work: the probe runs alone on the GPU
    solver = make_solver(precision)
    h = solver.h
    # manufactured solution x* and b = A~ x* (FP64 FMM matvec), column-major (nrhs, N) buffers
    xs = torch.from_numpy(inputs.rhs(w["seed"] + 1, N, nrhs).T.copy()).cuda()
    b = torch.empty_like(xs)
    ifmm.ifmm_matvec(h, xs.data_ptr(), b.data_ptr(), nrhs, N)
    x = torch.empty_like(xs)

    def step(hh):
        ifmm.ifmm_factor(hh, allow_overflow=True)
        ifmm.ifmm_solve(hh, b.data_ptr(), x.data_ptr(), nrhs, N, allow_noconv=True)

    tuned = None
    if args.autotune:
        # untimed, before the warm-up: the panel / Schur launch splits of this system's levels,
        # timed candidate by candidate on its own factorisation (ifmm_autotune); the results do
        # not depend on the splits, only the launch shapes do
        ifmm.ifmm_autotune_clear()
        t_tune = time.perf_counter()
        ifmm.ifmm_autotune([h], workers=1)
        tuned = {"table_entries": ifmm.ifmm_autotune_size(), "tuning_s": time.perf_counter() - t_tune}
    for _ in range(args.warmup):
        step(h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step(h)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = reduce_max_ms(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    st = ifmm.ifmm_get_stats(h)
    err = float(((x - xs).norm(dim=1) / xs.norm(dim=1)).max().item())
    value = whole_job_value(world, N, ms)
    launches_per_step = st["launches_factor"] + st["launches_solve"]
    peaks, peak_kind = load_peaks()
    boxes = sum(4 ** k for k in range(2, w["depth"] + 1))   # uniform points: no empty box
    rf = roofline(st, precision, peaks, peak_kind, pipe_peaks(pipes_measured), boxes)

    # end to end through the C ABI with host buffers in pinned memory (copies inside the timed region)
    b_pin = torch.empty((nrhs, N), dtype=torch.float64, pin_memory=True)
    b_pin.copy_(b.cpu())
    x_pin = torch.zeros((nrhs, N), dtype=torch.float64, pin_memory=True)
    b_host, x_host = b_pin.numpy(), x_pin.numpy()       # (nrhs, N) = column-major N x nrhs
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ifmm.ifmm_factor(h, allow_overflow=True)
        ifmm.ifmm_solve_host(h, b_host, x_host, nrhs, N, allow_noconv=True)
    e2e_ms = reduce_max_ms(1000.0 * (time.perf_counter() - t0) / e2e_steps, dist, "cuda")
    e2e_err = float(np.max(np.linalg.norm(x_host - xs.cpu().numpy(), axis=1) / np.linalg.norm(xs.cpu().numpy(), axis=1)))

    extra = {}
    if args.compare and rank == 0:
        solver.close()
        for other in [q for q in ("fp64", "mixed_solve", "mixed") if q != precision]:
            so = make_solver(other)
            ifmm.ifmm_matvec(so.h, xs.data_ptr(), b.data_ptr(), nrhs, N)
            if args.autotune:
                ifmm.ifmm_autotune([so.h], workers=1)   # tuned as the headline was (untimed)
            step(so.h)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            step(so.h)
            f1.record(stream)
            torch.cuda.synchronize()
            mso = f0.elapsed_time(f1)
            sto = ifmm.ifmm_get_stats(so.h)
            erro = float(((x - xs).norm(dim=1) / xs.norm(dim=1)).max().item())
            extra[f"{other}_gpu"] = {
                "value": N / (mso / 1000.0), "unit": "unknowns/s", "ms_per_step": mso, "err": erro,
                "meets_err_1e-6": erro <= 1e-6, "steps": 1, "warmup": 1, "precision": PRECISION_DESC[other],
                "t_factor_ms": sto["t_factor_ms"], "t_solve_ms": sto["t_solve_ms"],
                "refine_iters": sto["refine_iters"], "max_rank": sto["max_rank"],
                "kernel_ms": dict(zip(ifmm.FACTOR_KERNELS, sto["kernel_ms"]))}
            if other == "mixed":
                extra[f"{other}_gpu"]["note"] = (
                    "FP32 elimination: its pivot blocks (condition numbers 1e4..5e7 after balancing) exceed "
                    "1/u_fp32, so the FP32 factorisation is not an accurate preconditioner on 1/r + sqrt(N) I "
                    "(refinement capped at 30 iterations)")
            so.close()
        solver = None

    if args.octree and rank == 0:
        if solver is not None:
            solver.close()
            solver = None
        extra["octree_gpu"] = run_octree(precision)

    if args.batch:   # every rank runs its share of the independent systems
        if solver is not None:
            solver.close()
            solver = None
        extra["batched_gpu"] = run_batched(precision, rank, world, dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(st["refine_iters"] if N == WORKLOAD["N"] else None, full=args.cpu_full)
        cpu["gpu_over_oracle"] = value / cpu["value"]
        if "factor_only_value" in cpu:
            cpu["gpu_factor_over_oracle_factor"] = (N / (st["t_factor_ms"] / 1000.0)) / cpu["factor_only_value"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32+f64", "data": "synthetic",
                "precision": precision, "meets_err_1e-6": err <= 1e-6,
                "config": {"workload": workload_desc(w, PRECISION_DESC[precision]),
                           "N": N, "depth": w["depth"], "cheb_p": w["cheb_p"], "nrhs": nrhs, "eps": w["eps"],
                           "parallelism": "replicas" if world > 1 else "1 GPU",
                           "compress_cluster": args.compress_cluster,
                           "autotune": tuned,
                           "l2": "inputs larger than L2 (factor touches tens of GB per step)",
                           "err": err, "refine_iters": st["refine_iters"], "max_rank": st["max_rank"],
                           "t_factor_ms": st["t_factor_ms"], "t_solve_ms": st["t_solve_ms"],
                           "solve_rhs_unknowns_per_s": N * nrhs / (st["t_solve_ms"] / 1000.0),
                           "kernel_ms": dict(zip(ifmm.FACTOR_KERNELS, st["kernel_ms"])),
                           "level_ms": {str(k): round(st["level_ms"][k], 2) for k in range(2, w["depth"] + 1)},
                           "factor_tflop": st["factor_flops"] / 1e12,
                           "device_gb": st["device_bytes"] / 1e9},
                "roofline": rf, "cpu_baseline": cpu,
                "e2e": {"value": whole_job_value(world, N, e2e_ms), "unit": "unknowns/s",
                        "h2d_bytes_per_step": int(b_host.nbytes), "d2h_bytes_per_step": int(x_host.nbytes),
                        "host_buffers": "pinned", "ms_per_step": e2e_ms, "err": e2e_err},
                "gpu_launches": int(launches_per_step * args.steps), "clocks": clocks}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if solver is not None:
        solver.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed_solve", choices=["fp64", "mixed_solve", "mixed"],
                    help="headline precision; the others are timed alongside (one step each)")
    ap.add_argument("--n", type=int, default=0, help="override N (depth follows 64 points per leaf)")
    ap.add_argument("--compare", dest="compare", action="store_true", default=True,
                    help="also time one step of the other precision (reported, not the headline)")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="time the oracle's factorisation on the full 2^20-point workload (about 3 minutes) "
                         "instead of its 65,536-point sample")
    ap.add_argument("--tc-products", type=int, default=0, choices=[0, 1, 2],
                    help="mixed_solve: tensor-core products in the replay (1), the replay and the Schur "
                         "update (2), or double-float on the FP32 pipe (0)")
    ap.add_argument("--compress-cluster", type=int, default=16, choices=[1, 2, 4, 8, 16],
                    help="largest thread-block cluster one fill compression may use (1: one block each)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", default=True,
                    help="headline: keep the fixed launch-split rule instead of tuning the splits first")
    ap.add_argument("--batch", dest="batch", action="store_true", default=True,
                    help="also time the batched workload of 256 uneven systems (default)")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-octree", dest="octree", action="store_false", default=True,
                    help="skip the 3D (octree) workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
