#!/usr/bin/env python
"""Throughput of the beyond-Limber FFTLog C_ell hot path on GB300.

Metric: C_ell evaluations per second, one evaluation = the 120 spectra x 103 ell of one
parameter point of the N5K-shaped workload (10 clustering + 5 lensing windows, N_FFT = 2048,
N_k = 1024, N_I = 150 k-knots), forward + VJP (the whole hot path: FFTLog, Gamma-ratio
contraction with k-interpolation, k-quadrature and their reverse mode).  Inputs are seeded,
synthetic and resident in HBM when the timed region starts; L2 is flushed (256 MB write)
before every timed step.  Under torchrun every rank evaluates its own parameter points (weak
scaling, no collective on the data path) and the slowest rank's time counts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x9|tf32x6|3xtf32|fp64]
                    [--walkers B] [--impl ours|reference] [--sweep none|nell|cpu] [--limber L]

--impl reference times the FP64 oracle (NumPy/SciPy on the host cores) on the same workload, one
tracer's forward + VJP per step (15 steps = one evaluation), so that the default step count ends in
minutes.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "C_ell evals/s (120 spectra×103 ℓ), fwd & fwd+grad, vs FP64 GPU path at 1e-4 rel"
WORKLOAD = ("N5K-shaped: 15 tracers (10 Gaussian clustering + 5 Smail lensing bins), 120 spectra, "
            "103 log-spaced ell in [2,2000], N_FFT=2048, N_k=1024 in [1e-4,10] h/Mpc, N_I=150 k-knots, "
            "D(k,z)=(1+z)^-1(1+0.01 ln(k/0.1)); one evaluation = forward + VJP")
WORKLOAD_LARGE = ("large: 30 tracers (20 Gaussian clustering bins, sigma_z=0.03 + 10 Smail lensing bins), "
                  "465 spectra, every ell in [2,3000], N_FFT=4096, N_k=4096 in [1e-5,20] h/Mpc, N_I=200 "
                  "k-knots, bias b(k,z)=b0(1+z)^0.5(1+0.1k^2) in B_i; one evaluation = forward + VJP")

# measured peaks (MEASURED_PEAKS.json written by the pool driver); FP64 derived below
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 2 DFMA/clk/SM (FMA-loop probe: 1.19 TF/s at 2070 MHz)
TF32_OVER_BF16 = 1.1 / 2.25                      # nominal dense ratio


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x9", choices=["fp64", "3xtf32", "tf32x6", "bf16x9"])
    ap.add_argument("--walkers", type=int, default=1, help="parameter points per step per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the sub-records (general profile, 256-walker batch) and the TF32/FP64 "
                         "peak measurement")
    ap.add_argument("--sweep", default="none", choices=["none", "nell", "cpu", "cpu-child", "e2e"],
                    help="nell: time per evaluation against the number of multipoles (one JSON "
                         "line per point and a linear fit), instead of the headline line; cpu: the "
                         "oracle on the host cores for each workload size, with the BLAS thread "
                         "count pinned to one and to all cores; e2e: one step's host wall time "
                         "through the device-pointer graph and through swcl_step_host")
    ap.add_argument("--limber", type=int, default=0,
                    help="Limber branch for multipoles >= this (0: off, the paper's setting)")
    ap.add_argument("--workload", default="n5k", choices=["n5k", "large"],
                    help="large: one evaluation of the 30-tracer, 2999-multipole configuration "
                         "(one GPU, one walker; no CPU baseline)")
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="the context's memory budget in GiB (0: unlimited); a budget below the "
                         "whole-Delta workspace makes the VJP recompute Delta chunk by chunk")
    return ap.parse_args()


# ------------------------------------------------------------------ inputs ----

def make_inputs(walkers: int, rank: int, world: int, workload: str = "n5k"):
    """This rank's parameter points: walkers per GPU x world in all (weak scaling), the rank's
    contiguous block from paper_2505_22718_gb300.sharding.shard.  The large workload is one
    evaluation on one GPU, with a seeded N(0,1) cotangent."""
    from workloads import make_workload
    from paper_2505_22718_gb300.sharding import shard
    if workload == "large":
        if walkers != 1 or world != 1:
            raise SystemExit("--workload large runs one evaluation on one GPU")
        w = make_workload("large")
        return w, np.random.default_rng(31).standard_normal((1, len(w.ells), w.n_tr, w.n_tr))
    if walkers <= 1 and world == 1:
        w = make_workload("n5k_vjp")
        return w, w.C_bar[None] if w.C_bar.ndim == 3 else w.C_bar
    first, count = shard(walkers * world, world, rank)
    w = make_workload("walkers", n_walkers=count, first_walker=first)
    w.ell_lists = None  # every walker evaluates the full 103-ell set for the headline metric
    rng = np.random.default_rng([99, first])
    cbar = rng.standard_normal((count, len(w.ells), w.n_tr, w.n_tr))
    return w, cbar


def n_walk(w):
    return 1 if w.W.ndim == 2 else w.W.shape[0]


# ---------------------------------------------------------------- roofline ----

def algorithmic_work(w, walkers, rank, n_ell_useful=None):
    """Algorithmic FLOPs per launch of each kernel and, for tensor-core kernels, the number of
    compensated products each useful multiply-add costs (6 in basis mode: both operands in 3 bf16
    planes, the products with plane indices summing to at most 2; 9 for the knot-stencil bf16x9
    form; 3 or 6 for the TF32 forms).  The useful work of the contraction is
    4 n_h N_tr N_k N_ell per parameter point (the real form of the complex sum over n); with
    ragged multipole lists only the listed multipoles count (n_ell_useful = sum over walkers)."""
    n_h = w.N // 2 + 1
    ntr, nk, nl, ni, N = w.n_tr, len(w.k), len(w.ells), len(w.knots), w.N
    ell_units = n_ell_useful if n_ell_useful is not None else nl * walkers
    contraction = 4.0 * n_h * ntr * nk * ell_units
    rows = rank if rank else ni                                 # FFT rows per tracer
    fft = 2.5 * N * np.log2(N) * ntr * rows * walkers           # real FFT of length N per row
    return {
        "contract fp64": ("alu", contraction, 1),
        "contract adj fp64": ("alu", contraction, 1),
        "contract tc": ("tensor", contraction, None),
        "contract adj tc": ("tensor", contraction, None),
        "basis gemm fwd": ("tensor", contraction, 6),
        "basis gemm adj": ("tensor", contraction, 6),
        "fftlog": ("alu", fft, 1),
        "fftlog adj": ("alu", fft, 1),
    }


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel at the
# benchmark workload (one walker), from the ncu capture summarised in profiles/, valid only for
# the kernel source it was taken from (sha256 of the file; otherwise reported as null).
TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture per (kernel, tile code), one
    # walker, N5K-shaped workload (profiles/basis_gemm_n5k_bf16.md); valid while basis_tc.cu is
    # the file whose sha256 is recorded
    ("basis gemm adj", 16736): {"bytes": 25439232, "walkers": 1, "workload": "n5k",
                               "src": "paper_2505_22718_gb300/csrc/basis_tc.cu",
                               "sha256": "0e9f3ff4655bc6f91d9ef2dae84baf3ebf09bfb862c184be3b5fec9aa3aae851"},
    ("basis gemm adj", 16592): {"bytes": 25639936, "walkers": 1, "workload": "n5k",
                               "src": "paper_2505_22718_gb300/csrc/basis_tc.cu",
                               "sha256": "0e9f3ff4655bc6f91d9ef2dae84baf3ebf09bfb862c184be3b5fec9aa3aae851"},
    ("basis gemm adj", 16608): {"bytes": 25048576, "walkers": 1, "workload": "n5k",
                               "src": "paper_2505_22718_gb300/csrc/basis_tc.cu",
                               "sha256": "0e9f3ff4655bc6f91d9ef2dae84baf3ebf09bfb862c184be3b5fec9aa3aae851"},
}


def traffic_for(name, walkers, workload="n5k", tiles=None):
    import hashlib
    code = None
    if tiles and name.startswith("basis gemm"):
        code = tiles.get("adj" if name.endswith("adj") else "fwd")
    t = TRAFFIC.get((name, code))
    if not t or t["walkers"] != walkers or t["workload"] != workload:
        return None
    try:
        with open(os.path.join(ROOT, t["src"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
                return None
    except OSError:
        return None
    return t["bytes"]


def measure_matmul_peaks(dev):
    """TF32 and FP64 dense rates of this GPU, measured here the way the bf16 peaks of
    MEASURED_PEAKS.json were: cuBLAS through torch.matmul, best of 5 after warm-up, CUDA events
    (TF32: 8192^3 with TF32 tensor cores allowed; FP64: 4096^3).  Used only as roofline
    denominators: the library itself calls no cuBLAS."""
    import torch
    out = {}
    cases = (("tf32_tflops", torch.float32, 8192), ("fp64_tflops", torch.float64, 4096))
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        torch.backends.cuda.matmul.allow_tf32 = True
        for key, dt, n in cases:
            a = torch.randn(n, n, device=dev, dtype=dt)
            b = torch.randn(n, n, device=dev, dtype=dt)
            for _ in range(2):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[key] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    out["how"] = ("torch.matmul (cuBLAS), best of 5: TF32 8192^3 with allow_tf32, FP64 4096^3; "
                  "2 n^3 flops / CUDA-event time")
    return out


def roofline(stats, w, walkers, precision, peaks, src, rank, workload="n5k", steps=None,
             recompute=False, kernel=None, n_ell_useful=None, tiles=None):
    """Roofline of one kernel of the profiled steps (default: the longest).  `achieved` is the
    method's useful work (algorithmic_work) per launch over the kernel's average CUDA-event time,
    and `frac` is that over the measured peak of the kernel's arithmetic (bf16 burst from
    MEASURED_PEAKS.json for the split-bf16 GEMMs; TF32 and FP64 matmul rates measured in this run).
    `pipe_occupancy` counts every compensated product the kernel executes (useful x products):
    how busy the tensor pipe is, not how fast the method runs.  When the multipoles run in chunks
    (a memory budget) a launch covers one chunk, so the work per launch is the step's work over
    the step's launches of that kernel; with Delta recomputed in the VJP, the forward contraction
    runs twice per step."""
    if not stats:
        return None
    if kernel is None:
        name, (launches, ms) = max(stats.items(), key=lambda kv: kv[1][1])
    else:
        if kernel not in stats:
            return None
        name, (launches, ms) = kernel, stats[kernel]
    work = algorithmic_work(w, walkers, rank, n_ell_useful)
    bound, flops, products = work.get(name, ("alu", None, 1))
    avg_s = ms / launches / 1e3
    if flops is None:
        return {"kernel": name, "bound": None, "avg_ms": ms / launches, "note": "no algorithmic count"}
    per_step = launches / steps if steps else 1.0
    reps = 2 if recompute and name in ("basis gemm fwd", "contract fp64") else 1
    flops = flops * reps / per_step
    useful = flops / avg_s / 1e12
    if bound == "tensor":
        if products is None:
            products = {"3xtf32": 3, "tf32x6": 6, "bf16x9": 9}[precision]
        if precision in ("3xtf32", "tf32x6") and not name.startswith("basis"):
            if peaks.get("tf32_tflops"):
                peak, note = peaks["tf32_tflops"], "tf32 dense rate measured in this run (cuBLAS)"
            else:
                peak = peaks["bf16_tflops"] * TF32_OVER_BF16
                note = "tf32 peak = measured bf16 burst x nominal tf32/bf16 ratio"
        else:
            peak, note = peaks["bf16_tflops"], "bf16 burst peak (%s)" % src
        return {"kernel": name, "bound": "tensor", "achieved": useful, "peak": peak, "unit": "TFLOP/s",
                "frac": useful / peak, "pipe_occupancy": useful * products / peak,
                "products": products, "traffic": traffic_for(name, walkers, workload, tiles),
                "avg_ms": ms / launches, "launches": launches, "peak_source": note,
                "work": "4 n_h N_tr N_k N_ell useful flops per evaluation (%.3g per launch)" % flops}
    if peaks.get("fp64_tflops"):
        peak = peaks["fp64_tflops"]
        note = "FP64 dense rate measured in this run (cuBLAS DGEMM); derived DFMA pipe %.2f TF/s" % FP64_PEAK_TFLOPS
    else:
        peak = FP64_PEAK_TFLOPS
        note = "FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived)"
    return {"kernel": name, "bound": "alu", "achieved": useful, "peak": peak, "unit": "TFLOP/s",
            "frac": useful / peak, "traffic": traffic_for(name, walkers, workload, tiles),
            "avg_ms": ms / launches, "launches": launches, "peak_source": note,
            "work": "%.3g useful flops per launch" % flops}


# ------------------------------------------------------------------ clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle ----

def oracle_grids(w, tracers=None):
    """The oracle's grids for the workload (or for a subset of its tracers), with its numpy.fft
    form of the Eq. 3.2 sum (a pinned library step, the fastest form the oracle has)."""
    from oracle import fftlog as O
    sel = slice(None) if tracers is None else tracers
    return O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind[sel], w.fft_bias[sel],
                   fft="numpy")


def oracle_eval(w, cbar, g=None):
    from oracle import fftlog as O
    if g is None:
        g = oracle_grids(w)
    W = w.W if w.W.ndim == 2 else w.W[0]
    P = w.P if w.P.ndim == 1 else w.P[0]
    A = w.amp if w.amp.ndim == 1 else w.amp[0]
    f = O.forward(g, W, w.D, P, A, w.B)
    O.vjp(g, f, cbar[0], W, w.D, P, A, w.B)
    return g, f


def cpu_baseline(w, cbar, n_eval=8):
    g = oracle_grids(w)
    for b in np.unique(w.fft_bias):
        g.mtable(b)  # the paper excludes the Gamma-ratio precomputation from its timings
    t0 = time.perf_counter()
    f = None
    for _ in range(n_eval):
        _, f = oracle_eval(w, cbar, g)
    dt = time.perf_counter() - t0
    return {"value": n_eval / dt, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d full forward+VJP evaluations of one parameter point (Gamma/phase tables "
                      "precomputed, as the paper excludes them), NumPy/SciPy FP64 with numpy.fft for "
                      "the FFTLog sum, BLAS threads = all cores" % n_eval}, f


class TracerSample:
    """A bounded sample of one evaluation for the reference arm: step t evaluates the forward pass
    and the VJP of tracer t mod N_tr alone (its FFTLog at every knot, Delta at every multipole,
    its auto-spectrum and the reverse mode) with the oracle as it stands; N_tr steps stand for one
    evaluation (the cross-spectra's quadrature, a few per cent of the oracle's time, is left out,
    so the scaled rate slightly overstates the oracle's)."""

    def __init__(self, w, cbar):
        self.w = w
        self.cb = cbar[0]
        self.grids = [oracle_grids(w, slice(i, i + 1)) for i in range(w.n_tr)]
        for i, g in enumerate(self.grids):
            g.mtable(w.fft_bias[i])
        self.t = 0

    def step(self):
        from oracle import fftlog as O
        w = self.w
        i = self.t % w.n_tr
        self.t += 1
        g = self.grids[i]
        W = (w.W if w.W.ndim == 2 else w.W[0])[i:i + 1]
        P = w.P if w.P.ndim == 1 else w.P[0]
        A = (w.amp if w.amp.ndim == 1 else w.amp[0])[i:i + 1]
        B = None if w.B is None else w.B[i:i + 1]
        f = O.forward(g, W, w.D, P, A, B)
        O.vjp(g, f, self.cb[:, i:i + 1, i:i + 1], W, w.D, P, A, B)


def cpu_baseline_sweep_child(threads):
    """The CPU-baseline leg at every workload size, one JSON line per workload: the oracle as it
    stands, timed on the host cores with the BLAS thread count the parent pinned.  tiny2 and n5k
    forward, n5k_vjp forward + VJP, and (all cores only) one forward pass of the large workload;
    the Gamma-ratio tables are built before the timed region, as the paper excludes them."""
    from oracle import fftlog as O
    from workloads import make_workload
    cases = [("tiny2", False, 3.0), ("n5k", False, 3.0), ("n5k_vjp", True, 3.0)]
    if threads > 1:
        cases.append(("large", False, 0.0))
    for name, vjp, budget in cases:
        w = make_workload(name)
        g = oracle_grids(w)
        for b in np.unique(w.fft_bias):
            g.mtable(b)
        W = w.W if w.W.ndim == 2 else w.W[0]
        cb = None
        if vjp:
            cb = w.C_bar if w.C_bar.ndim == 3 else w.C_bar[0]
        n = 0
        t0 = time.perf_counter()
        while True:
            f = O.forward(g, W, w.D, w.P, w.amp, w.B)
            if vjp:
                O.vjp(g, f, cb, W, w.D, w.P, w.amp, w.B)
            n += 1
            if time.perf_counter() - t0 >= budget:
                break
        dt = time.perf_counter() - t0
        print(json.dumps({"sweep": "cpu", "workload": name, "pass": "fwd+vjp" if vjp else "fwd",
                          "blas_threads": threads, "cores": os.cpu_count(), "evals": n,
                          "s_per_eval": dt / n, "evals_per_s": n / dt,
                          "shape": {"n_tr": w.n_tr, "N": w.N, "n_k": len(w.k), "n_ell": len(w.ells),
                                    "n_knots": len(w.knots)}}), flush=True)
    return 0


def cpu_baseline_sweep():
    """The oracle's CPU cost per workload size with BLAS pinned to one thread and to all cores;
    each setting runs in a child process, since BLAS fixes its thread count when it loads."""
    for threads in (1, os.cpu_count() or 1):
        env = dict(os.environ)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[var] = str(threads)
        env["SWCL_CPU_SWEEP_THREADS"] = str(threads)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--sweep", "cpu-child"], env=env)
        if r.returncode != 0:
            return r.returncode
    return 0


# ----------------------------------------------------------------- our arm ----

class Step:
    """The library calls of one timed step on device buffers: forward + VJP (or forward only) of
    every walker as one CUDA-graph replay, and the same kernels launched one by one for per-kernel
    CUDA-event timing."""

    def __init__(self, swcl, ctx, C, Cb, Pb, Ab, Wb):
        self.swcl, self.ctx = swcl, ctx
        self.C, self.Cb, self.Pb, self.Ab, self.Wb = C, Cb, Pb, Ab, Wb

    def full(self, p):
        self.swcl.swcl_compute_batched(self.ctx.ptr, p, self.C, self.Cb, self.Pb, self.Ab, self.Wb)
        return self.ctx.query(self.swcl.SWCL_Q_KERNEL_LAUNCHES)

    def fwd(self, p):
        self.swcl.swcl_compute_batched(self.ctx.ptr, p, self.C)
        return self.ctx.query(self.swcl.SWCL_Q_KERNEL_LAUNCHES)

    def profiled(self, p):
        # per-kernel event timing needs the kernels launched one by one (not from a graph)
        self.swcl.swcl_compute_cl(self.ctx.ptr, p, self.C)
        n1 = self.ctx.query(self.swcl.SWCL_Q_KERNEL_LAUNCHES)
        self.swcl.swcl_vjp(self.ctx.ptr, p, self.Cb, self.Pb, self.Ab, self.Wb)
        return n1 + self.ctx.query(self.swcl.SWCL_Q_KERNEL_LAUNCHES)


def device_inputs(swcl, ctx, w, cbar, dev, with_grids=True):
    """Sets the workload on the context from device tensors and returns the Step buffers."""
    import torch
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    if with_grids:
        ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots)
        ctx.set_tracers(w.kind, w.fft_bias)
    ctx.set_windows(t(w.W), t(w.D), None if w.B is None else t(w.B))
    ctx.set_power(t(w.P), t(w.amp))
    nw = n_walk(w)
    if w.ell_lists is not None:
        ctx.set_ell_lists(w.ell_lists)
        n_out = sum(len(x) for x in w.ell_lists)
    else:
        n_out = nw * len(w.ells)
    C = torch.empty((n_out, w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
    Cb = t(np.asarray(cbar).reshape(C.shape))
    Pb = torch.empty((nw, len(w.k)), dtype=torch.float64, device=dev)
    Ab = torch.empty((nw, w.n_tr), dtype=torch.float64, device=dev)
    Wb = torch.empty((nw, w.n_tr, w.N), dtype=torch.float64, device=dev)
    return Step(swcl, ctx, C, Cb, Pb, Ab, Wb)


def run_ours(args, rank, world, device):
    import torch
    import paper_2505_22718_gb300 as swcl
    from paper_2505_22718_gb300.sharding import max_over_ranks

    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    prec = swcl.PRECISIONS[args.precision]
    w, cbar = make_inputs(args.walkers, rank, world, args.workload)
    nw = n_walk(w)
    # one dedicated stream: the library's kernels, the L2 flush and the timing events are
    # all ordered on it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = swcl.Context(device, int(args.budget_gb * (1 << 30)), stream.cuda_stream)
    # the per-grid tables (Gamma ratios, phases, tracer powers) are built once, outside the step,
    # as the paper excludes them from its timings; their cost is reported beside the step
    torch.cuda.synchronize(dev)
    t_tab = time.perf_counter()
    ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots)
    ctx.set_tracers(w.kind, w.fft_bias)
    torch.cuda.synchronize(dev)
    tables_ms = (time.perf_counter() - t_tab) * 1e3
    st = device_inputs(swcl, ctx, w, cbar, dev, with_grids=False)
    if args.limber:
        ctx.set_limber(args.limber)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    last = {}

    def timed(fn, steps, warmup, profile_ctx=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        if profile_ctx is not None:
            swcl.swcl_profile_reset(profile_ctx.ptr)
            swcl.swcl_profile_enable(profile_ctx.ptr, True)
        evs = []
        launches = 0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launches += fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        stats = None
        if profile_ctx is not None:
            stats = swcl.swcl_profile_read(profile_ctx.ptr)
            swcl.swcl_profile_enable(profile_ctx.ptr, False)
        per = [a.elapsed_time(b) for a, b in evs]
        last["median_ms"] = statistics.median(per)
        ms = sum(per)
        if world > 1:
            ms = max_over_ranks(ms, dev)
            torch.distributed.barrier()
        return ms, launches, stats

    out = {}
    clocks = ClockSampler(device) if rank == 0 else None
    if clocks:
        clocks.start()
    ms, launches, _ = timed(lambda: st.full(prec), args.steps, args.warmup)
    clk = clocks.stop() if clocks else None
    ms_step = ms / args.steps
    out["ms_per_step_median"] = last["median_ms"]
    out["tables_ms"] = tables_ms
    peaks, src = load_peaks()
    if rank == 0 and not args.no_extra:
        peaks = dict(peaks)
        peaks.update(measure_matmul_peaks(dev))
        out["peaks_measured_here"] = {k: peaks[k] for k in ("tf32_tflops", "fp64_tflops", "how")}
    # per-kernel device times for the roofline: the same step launched kernel by kernel with
    # CUDA events around each kernel on the library's stream
    k_prof = max(3, min(args.steps, 200))
    _, _, stats = timed(lambda: st.profiled(prec), k_prof, 2, profile_ctx=ctx)
    value = nw * world / (ms_step / 1e3)
    out["value"] = value
    out["ms_per_step"] = ms_step
    out["gpu_launches"] = launches    # kernels of the graph replays in the timed region
    out["kernels_per_step"] = launches // max(args.steps, 1)
    out["clocks"] = clk
    out["kernel_ms"] = {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in (stats or {}).items()}
    rank_r = ctx.query(swcl.SWCL_Q_PROFILE_RANK)
    out["tiles"] = {"fwd": ctx.query(swcl.SWCL_Q_TILE_FWD), "adj": ctx.query(swcl.SWCL_Q_TILE_ADJ)}
    out["recompute"] = ctx.query(swcl.SWCL_Q_RECOMPUTE)
    out["roofline"] = roofline(stats, w, nw, args.precision, peaks, src, rank_r, args.workload,
                               k_prof, bool(out["recompute"]), tiles=out["tiles"])
    out["profile_rank"] = rank_r
    msf, _, _ = timed(lambda: st.fwd(prec), args.steps, max(3, args.warmup // 2))
    out["fwd_only"] = {"value": nw * world / (msf / args.steps / 1e3), "unit": "evals/s",
                       "ms_per_step": msf / args.steps}
    if not args.no_fp64_compare and args.precision != "fp64":
        k64 = max(3, args.steps // 20)
        ms64, _, _ = timed(lambda: st.full(swcl.SWCL_FP64), k64, 2)
        _, _, st64 = timed(lambda: st.profiled(swcl.SWCL_FP64), 3, 1, profile_ctx=ctx)
        out["fp64_gpu_path"] = {"value": nw * world / (ms64 / k64 / 1e3), "unit": "evals/s",
                                "ms_per_step": ms64 / k64,
                                "roofline": roofline(st64, w, nw, "fp64", peaks, src, rank_r,
                                                     args.workload, 3, bool(out["recompute"]))}
    # result of this precision (rank 0, walker 0) for the accuracy check against the oracle
    st.full(prec)
    torch.cuda.synchronize(dev)
    out["_C0"] = st.C[:len(w.ells)].cpu().numpy()

    # end to end through the public API with pinned host buffers: the per-step inputs of a
    # sampler (window samples, P(k), amplitudes, cotangent) go host -> device, the graph replays,
    # and every result comes back; D (growth at the knots) was set once with the windows
    if not args.no_e2e:
        def pinned(a):
            h = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
            h.numpy()[...] = a
            return h
        W_h, P_h, A_h = pinned(w.W), pinned(w.P), pinned(w.amp)
        Cb_h = pinned(np.asarray(cbar).reshape(st.C.shape))
        C_h = torch.empty(st.C.shape, dtype=torch.float64, pin_memory=True)
        Pb_h = torch.empty(st.Pb.shape, dtype=torch.float64, pin_memory=True)
        Ab_h = torch.empty(st.Ab.shape, dtype=torch.float64, pin_memory=True)
        Wb_h = torch.empty(st.Wb.shape, dtype=torch.float64, pin_memory=True)

        # one call per step: inputs host -> device, forward + VJP, results device -> host, in
        # one graph replay; returns when the host outputs are written
        e2e_step = swcl.HostStep(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)

        for _ in range(max(3, args.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        if world > 1:
            el = max_over_ranks(el, dev)
        h2d = sum(x.numel() * 8 for x in (W_h, P_h, A_h, Cb_h))
        d2h = sum(x.numel() * 8 for x in (C_h, Pb_h, Ab_h, Wb_h))
        out["e2e"] = {"value": nw * world * args.steps / el, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h,
                      "calls": "swcl_step_host (HostStep, arguments prepared once): window "
                               "samples, P, amplitudes and cotangent "
                               "host -> device, forward + VJP, C and the gradients device -> host, "
                               "one graph replay and one wait per step"}
    ctx.close()
    del st
    if rank == 0 and world == 1 and args.workload == "n5k" and not args.no_extra:
        out["general_profile"] = run_general_profile(args, dev, stream, flush, timed, peaks, src)
        out["batched"] = run_batched(args, dev, stream, timed, peaks, src)
        out["large"] = run_large(args, dev, stream, timed, peaks, src)
    return out, w, cbar


def run_general_profile(args, dev, stream, flush, timed, peaks, src):
    """Sub-record for a growth that is not of low rank (n5k_general): one FFTLog per k-knot and
    the knot-stencil tcgen05 kernels (Sec. 3.2's interpolation along k in their producers).
    Forward + VJP and forward-only evals/s, the FP64 GPU path on the same inputs, the roofline
    of both contraction kernels, and the normalised C error against the oracle."""
    import torch
    import paper_2505_22718_gb300 as swcl
    from workloads import make_workload
    w = make_workload("n5k_general")
    prec = swcl.PRECISIONS[args.precision]
    ctx = swcl.Context(dev.index, 0, stream.cuda_stream)
    st = device_inputs(swcl, ctx, w, w.C_bar[None], dev)
    steps = max(3, min(args.steps, 200))
    ms, launches, _ = timed(lambda: st.full(prec), steps, 3)
    msf, _, _ = timed(lambda: st.fwd(prec), steps, 3)
    _, _, stats = timed(lambda: st.profiled(prec), 10, 2, profile_ctx=ctx)
    rank_r = ctx.query(swcl.SWCL_Q_PROFILE_RANK)
    rec = {"workload": "N5K shape with D(k,z) = (1+z)^-1 exp(0.02 ln(k/0.1) g(z)) (profiles of high "
                       "rank: one FFTLog per knot, 150 knots per tracer)",
           "profile_rank": rank_r, "value": 1e3 * steps / ms, "unit": "evals/s", "ms_per_step": ms / steps,
           "fwd_only": {"value": 1e3 * steps / msf, "ms_per_step": msf / steps},
           "kernels_per_step": launches // steps,
           "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in stats.items()},
           "roofline": roofline(stats, w, 1, args.precision, peaks, src, rank_r, "n5k_general", 10),
           "roofline_fwd_contraction": roofline(stats, w, 1, args.precision, peaks, src, rank_r,
                                                "n5k_general", 10, kernel="contract tc"),
           "roofline_adj_contraction": roofline(stats, w, 1, args.precision, peaks, src, rank_r,
                                                "n5k_general", 10, kernel="contract adj tc")}
    if not args.no_fp64_compare:
        ms64, _, _ = timed(lambda: st.full(swcl.SWCL_FP64), 3, 1)
        rec["fp64_gpu_path"] = {"value": 3e3 / ms64, "unit": "evals/s", "ms_per_step": ms64 / 3}
    st.full(prec)
    torch.cuda.synchronize(dev)
    C = st.C.cpu().numpy()
    ctx.close()
    if not args.no_cpu_baseline:
        from oracle import fftlog as O
        g = oracle_grids(w)
        Co = O.forward(g, w.W, w.D, w.P, w.amp, w.B)["C"]
        dg = np.abs(np.einsum("lii->li", Co))
        floor = 1e-3 * np.sqrt(dg[:, :, None] * dg[:, None, :])
        rec["accuracy"] = {"max_norm_err_vs_oracle": float(np.max(np.abs(C - Co) / np.maximum(np.abs(Co), floor))),
                           "gate": 1e-4}
    return rec


def run_large(args, dev, stream, timed, peaks, src):
    """Sub-record for the large configuration (30 tracers, every ell in [2, 3000], N = N_k = 4096,
    200 knots, B(k, z)): one evaluation per step, forward + VJP and forward only, under a 40 GiB
    memory budget, and the roofline of the dominant kernel."""
    import paper_2505_22718_gb300 as swcl
    from workloads import make_workload
    w = make_workload("large")
    cbar = np.random.default_rng(31).standard_normal((1, len(w.ells), w.n_tr, w.n_tr))
    prec = swcl.PRECISIONS[args.precision]
    ctx = swcl.Context(dev.index, 40 << 30, stream.cuda_stream)
    st = device_inputs(swcl, ctx, w, cbar, dev)
    ms, _, _ = timed(lambda: st.full(prec), 5, 3)
    msf, _, _ = timed(lambda: st.fwd(prec), 5, 2)
    _, _, stats = timed(lambda: st.profiled(prec), 3, 1, profile_ctx=ctx)
    rank_r = ctx.query(swcl.SWCL_Q_PROFILE_RANK)
    rec = {"workload": WORKLOAD_LARGE, "budget_gb": 40, "delta_recomputed": bool(ctx.query(swcl.SWCL_Q_RECOMPUTE)),
           "value": 1e3 * 5 / ms, "unit": "evals/s", "ms_per_step": ms / 5,
           "fwd_only": {"value": 1e3 * 5 / msf, "ms_per_step": msf / 5},
           "tiles": {"fwd": ctx.query(swcl.SWCL_Q_TILE_FWD), "adj": ctx.query(swcl.SWCL_Q_TILE_ADJ)},
           "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in stats.items()},
           "roofline": roofline(stats, w, 1, args.precision, peaks, src, rank_r, "large", 3)}
    ctx.close()
    return rec


def run_batched(args, dev, stream, timed, peaks, src, n_walkers=256):
    """Sub-record for the batched configuration: 256 parameter points with their own P(k)
    amplitude and tilt, clustering amplitudes and window shifts, and ragged multipole lists
    (50-103 of the 103), forward + VJP and forward-only as one CUDA-graph replay per step.
    evals/s counts parameter points; the roofline counts only the listed multipoles as useful."""
    import paper_2505_22718_gb300 as swcl
    from workloads import make_workload
    w = make_workload("walkers", n_walkers=n_walkers)
    n_out = sum(len(x) for x in w.ell_lists)
    cbar = np.random.default_rng(99).standard_normal((n_out, w.n_tr, w.n_tr))
    prec = swcl.PRECISIONS[args.precision]
    ctx = swcl.Context(dev.index, 0, stream.cuda_stream)
    st = device_inputs(swcl, ctx, w, cbar, dev)
    steps = max(3, min(args.steps // 40, 50))
    ms, launches, _ = timed(lambda: st.full(prec), steps, 3)
    msf, _, _ = timed(lambda: st.fwd(prec), steps, 3)
    _, _, stats = timed(lambda: st.profiled(prec), 3, 1, profile_ctx=ctx)
    rank_r = ctx.query(swcl.SWCL_Q_PROFILE_RANK)
    rec = {"walkers": n_walkers, "listed_multipoles": n_out,
           "value": n_walkers * 1e3 * steps / ms, "unit": "evals/s", "ms_per_step": ms / steps,
           "fwd_only": {"value": n_walkers * 1e3 * steps / msf, "ms_per_step": msf / steps},
           "kernels_per_step": launches // steps, "tiles": {"fwd": ctx.query(swcl.SWCL_Q_TILE_FWD),
                                                            "adj": ctx.query(swcl.SWCL_Q_TILE_ADJ)},
           "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / max(v[0], 1)} for k, v in stats.items()},
           "roofline": roofline(stats, w, n_walkers, args.precision, peaks, src, rank_r, "walkers", 3,
                                n_ell_useful=n_out)}
    if not args.no_fp64_compare:
        ms64, _, _ = timed(lambda: st.full(swcl.SWCL_FP64), 2, 1)
        rec["fp64_gpu_path"] = {"value": n_walkers * 2e3 / ms64, "unit": "evals/s", "ms_per_step": ms64 / 2}
    ctx.close()
    return rec


def run_sweep_nell(args, device):
    """Forward and forward+VJP time per evaluation of the N5K-shaped workload for N_ell
    log-spaced multipoles in [2, 2000] (the running-time study of Sec. 5 / Appendix A), one
    CUDA-graph replay per step, L2 flushed before each timed step, CUDA events on the stream."""
    import torch
    import paper_2505_22718_gb300 as swcl
    from workloads import make_workload, ell_list
    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    prec = swcl.PRECISIONS[args.precision]
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    steps = max(3, min(args.steps, 200))
    pts = []
    for n in (10, 30, 103, 300, 1000, 1999):
        w = make_workload("n5k")
        w.ells = ell_list(2, 2000, n)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
        ctx = swcl.Context(device, 0, stream.cuda_stream)
        ctx.set_grids(w.chi_min, w.chi_max, w.N, w.k, w.ells, w.knots)
        ctx.set_tracers(w.kind, w.fft_bias)
        ctx.set_windows(t(w.W), t(w.D), None)
        ctx.set_power(t(w.P), t(w.amp))
        if args.limber:
            ctx.set_limber(args.limber)
        C = torch.empty((n, w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
        Cb = torch.randn((n, w.n_tr, w.n_tr), dtype=torch.float64, device=dev)
        Pb = torch.empty((1, len(w.k)), dtype=torch.float64, device=dev)
        Ab = torch.empty((1, w.n_tr), dtype=torch.float64, device=dev)
        Wb = torch.empty((1, w.n_tr, w.N), dtype=torch.float64, device=dev)
        res = {}
        for name, fn in (("fwd", lambda: swcl.swcl_compute_batched(ctx.ptr, prec, C)),
                         ("fwd_vjp", lambda: swcl.swcl_compute_batched(ctx.ptr, prec, C, Cb, Pb, Ab, Wb))):
            for _ in range(max(3, args.warmup)):
                fn()
            torch.cuda.synchronize(dev)
            tot = 0.0
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                tot += e0.elapsed_time(e1)
            res[name] = tot / steps
        ctx.close()
        line = {"sweep": "n_ell", "n_ell": n, "ms_fwd": res["fwd"], "ms_fwd_vjp": res["fwd_vjp"],
                "precision": args.precision, "limber_switch": args.limber, "steps": steps,
                "workload": WORKLOAD}
        print(json.dumps(line))
        pts.append((n, res["fwd"], res["fwd_vjp"]))
    a = np.array(pts)
    fit = {}
    for col, name in ((1, "fwd"), (2, "fwd_vjp")):
        slope, icpt = np.polyfit(a[:, 0], a[:, col], 1)
        fit[name] = {"ms_per_ell": slope, "ms_fixed": icpt}
    print(json.dumps({"sweep": "n_ell", "fit_t_equals_a_nell_plus_b": fit, "precision": args.precision,
                      "limber_switch": args.limber}))
    return 0


def run_sweep_e2e(args, device):
    """Where the end-to-end step's time goes, one parameter point of the N5K-shaped workload, one
    process: per step (host wall time over the timed steps, no L2 flush), the device-pointer graph
    followed by a host synchronisation; swcl_step_host through the Python binding; and the same
    C entry point called through ctypes with its arguments prepared once."""
    import ctypes
    import torch
    import paper_2505_22718_gb300 as swcl
    from paper_2505_22718_gb300 import _lib
    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    prec = swcl.PRECISIONS[args.precision]
    w, cbar = make_inputs(1, 0, 1)
    ctx = swcl.Context(device)
    st = device_inputs(swcl, ctx, w, cbar, dev)

    def pinned(a, shape):
        h = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        h.numpy()[...] = np.asarray(a).reshape(shape)
        return h
    W_h, P_h, A_h = pinned(w.W, st.Wb.shape), pinned(w.P, st.Pb.shape), pinned(w.amp, st.Ab.shape)
    Cb_h = pinned(cbar, st.C.shape)
    C_h, Pb_h, Ab_h, Wb_h = (torch.empty(x.shape, dtype=torch.float64, pin_memory=True)
                             for x in (st.C, st.Pb, st.Ab, st.Wb))
    lib = _lib.load()
    args_c = [ctypes.c_void_p(t.data_ptr()) for t in (W_h, P_h, A_h, Cb_h, C_h, Pb_h, Ab_h, Wb_h)]

    def device_graph():
        st.full(prec)
        ctx.sync()

    def step_binding():
        swcl.swcl_step_host(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)

    def step_ctypes():
        if lib.swcl_step_host(ctx.ptr, prec, *args_c) != 0:
            raise RuntimeError("swcl_step_host failed")
    steps = max(100, args.steps)
    out = {"sweep": "e2e", "workload": WORKLOAD, "precision": args.precision, "steps": steps}
    step_prepared = swcl.HostStep(ctx.ptr, prec, C_h, W_h, P_h, A_h, Cb_h, Pb_h, Ab_h, Wb_h)
    for name, fn in (("device_graph_and_sync_us", device_graph), ("step_host_binding_us", step_binding),
                     ("step_host_ctypes_us", step_ctypes), ("host_step_object_us", step_prepared)):
        for _ in range(max(3, args.warmup)):
            fn()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        out[name] = (time.perf_counter() - t0) / steps * 1e6
    ctx.close()
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.sweep == "cpu":
        return cpu_baseline_sweep() if rank == 0 else 0
    if args.sweep == "cpu-child":
        return cpu_baseline_sweep_child(int(os.environ.get("SWCL_CPU_SWEEP_THREADS", os.cpu_count() or 1)))
    if args.impl == "reference":
        if rank != 0:
            return 0
        w, cbar = make_inputs(1, 0, 1)
        sample = TracerSample(w, cbar)
        for _ in range(args.warmup):
            sample.step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sample.step()
        dt = time.perf_counter() - t0
        v = args.steps / w.n_tr / dt
        line = {"metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": WORKLOAD, "walkers_per_gpu": 1, "precision": "fp64 oracle"},
                "cpu_baseline": {"value": v, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": "one tracer's forward+VJP per step (FFTLog at all 150 knots, "
                                           "all 103 multipoles, its auto-spectrum), %d tracer steps = "
                                           "one evaluation; Gamma tables precomputed; numpy.fft form"
                                           % w.n_tr},
                "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if args.sweep == "nell":
        if rank != 0:
            return 0
        import __graft_entry__
        __graft_entry__.build()
        return run_sweep_nell(args, local)
    if args.sweep == "e2e":
        if rank != 0:
            return 0
        import __graft_entry__
        __graft_entry__.build()
        return run_sweep_e2e(args, local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    out, w, cbar = run_ours(args, rank, world, local)
    if rank == 0:
        cpu = None
        acc = None
        if world == 1 and not args.no_cpu_baseline and args.workload == "n5k":
            cpu, f = cpu_baseline(w if n_walk(w) == 1 else w, cbar[:1] if cbar.ndim == 4 else cbar)
            if n_walk(w) == 1 and not args.limber:
                Co = f["C"]
                C0 = out["_C0"]
                dg = np.abs(np.einsum("lii->li", Co))
                floor = 1e-3 * np.sqrt(dg[:, :, None] * dg[:, None, :])
                acc = {"max_norm_err_vs_oracle": float(np.max(np.abs(C0 - Co) / np.maximum(np.abs(Co), floor))),
                       "gate": 1e-10 if args.precision == "fp64" else 1e-4}
        dtype = {"fp64": "f64",
                 "3xtf32": "tf32x3 tensor-core contraction (f32 accumulate) + f64 FFT/Gamma/k-sum",
                 "tf32x6": "tf32x6 tensor-core contraction (f32 accumulate) + f64 FFT/Gamma/k-sum",
                 "bf16x9": "split-bf16 tensor-core contraction (3+3 planes, 6 products in basis mode; "
                           "f32 accumulate) + f64 FFT/Gamma/k-sum"}[args.precision]
        line = {"metric": METRIC, "value": out["value"], "unit": "evals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
                "data": "synthetic",
                "config": {"workload": WORKLOAD if args.workload == "n5k" else WORKLOAD_LARGE,
                           "walkers_per_gpu": n_walk(w), "precision": args.precision,
                           "budget_gb": args.budget_gb or None, "delta_recomputed": bool(out["recompute"]),
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": "walkers sharded across ranks" if world > 1 else "1 GPU",
                           "profile_rank": out.get("profile_rank"), "gemm_tiles": out.get("tiles"),
                           "limber_switch": args.limber or None},
                "roofline": out["roofline"], "cpu_baseline": cpu, "e2e": out.get("e2e"),
                "clocks": out["clocks"], "gpu_launches": out["gpu_launches"],
                "ms_per_step_median": out["ms_per_step_median"], "tables_ms": out["tables_ms"],
                "fwd_only": out["fwd_only"], "fp64_gpu_path": out.get("fp64_gpu_path"),
                "accuracy": acc, "kernel_ms": out["kernel_ms"],
                "kernels_per_step": out["kernels_per_step"],
                "peaks_measured_here": out.get("peaks_measured_here"),
                "general_profile": out.get("general_profile"), "batched": out.get("batched"),
                "large": out.get("large")}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
