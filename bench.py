#!/usr/bin/env python
"""Benchmark of the recycled shifted solves on GB300.

Workload: the 2048 x 2048 image (sigma 4, radius 12, 3 % noise), 64 shifts
log-spaced over 1e-6..1, 8 outer reweighting steps, principal recycle dimension
100, 8 local Ritz vectors, mixed precision (FP32 Krylov vectors and matvecs,
FP64 Grams, small solves and iterative-refinement residuals), every system
solved to a true relative residual of 1e-8. All of it runs through librecyc's
C ABI.

A step is one outer reweighting step of that job: rs_set_weights(w_k),
rs_update_recycle (k = 0: principal space from two seeding solves; k >= 1:
update by Eq. delta), rs_solve_shifts over all 64 shifts, and the L-curve corner
and IRN weights w_{k+1}. Steps cycle through k = 0..7; after k = 7 the next step
starts the job again on a new problem. The timed steps and the end-to-end steps
both start at k = 0.

Metric: shifted solves per second over the timed steps (and matvecs per
second), inputs resident in HBM. `e2e` repeats the same steps with the data
image and each step's weights copied in from pinned host memory and every
step's solutions (and next weights) copied back. `roofline` is the MINRES
kernel's achieved rate from CUDA events around its launches in the timed
region. The other keys put the number in context: the FP64 GPU solver and the
unrecycled solver on the same workload, solution differences, the other
workloads, and the FP64 oracle on the host cores (`cpu_baseline`).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "shifted solves/sec & matvecs/sec at rel. residual 1e-8; HBM GB/s vs roofline"
FP64_NOMINAL_GFLOPS = 152 * 2070e6 * 4 / 1e9   # 152 SMs x 2 FP64 FMA/clk x 2070 MHz (1.26 TF)
CSRC = os.path.join(ROOT, "paper_2306_15049_gb300", "csrc")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic byte of a
# MINRES kernel, from one ncu capture of `python bench.py --profile-case small` (the same
# kernel on the same image and radius, four shifts on a random 12-column principal
# basis, 24 steps each: about 1.3 GB on the device); scaled to a launch of the timed
# workload by its algorithmic bytes. `src` is the SHA-256 (first 16 hex digits) of the
# kernel's sources at the capture: a kernel changed since reports traffic null.
TRAFFIC = {
    # 2048 x 2048, radius 12, mixed, two-pass stencil (RS_TMA=2): two 24-step launches read
    # 10.25 + 11.08 GB and wrote 2.00 + 2.00 GB against 11.27 + 12.08 GB algorithmic (s = 8, 9)
    "k_mr_tma<float,12>": {"dram_per_alg": 1.085, "src": "1c2c3fff45f90c26"},
}


OUTER_KEYS = ("init_solves", "update_vnew", "principal_setup", "shift_setup", "shift_minres",
              "fp64_residuals")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--workload", default="C5")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the unrecycled comparison solver (every shift from x0 = 0)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (512x512, four images, differentiation, 64x64 oracle parity)")
    ap.add_argument("--profile-case", nargs="?", const="step", choices=["step", "job", "small"],
                    help="run once for a profiler and exit (step: the first two outer steps of the workload; "
                         "job: all its outer steps; "
                         "small: four shifts of the same image on a random 12-column principal basis, "
                         "24 MINRES steps each)")
    return ap.parse_args()


def workload_config(wl, precision):
    return {
        "workload": f"{wl.height}x{wl.width} image, sigma {wl.sigma}, radius {wl.radius}, "
                    f"{int(round(wl.eta * 100))}% noise; {wl.M} shifts 1e{int(wl.log_lo)}..1e{int(wl.log_hi)}; "
                    f"{wl.K} outer IRN steps; p={wl.p}, |J|={wl.n_ritz_local}; tol {wl.tol:g}",
        "n": wl.n, "shifts": wl.M, "outer_steps": wl.K, "p": wl.p, "local_ritz": wl.n_ritz_local,
        "precision": precision,
        "step": "one outer reweighting step (set_weights, update_recycle, all shifts, L-curve and "
                "next weights); steps cycle k = 0..K-1 from k = 0",
        "parallelism": "replicas (one independent workload per GPU)",
    }


def kernel_src_sha():
    h = hashlib.sha256()
    for f in ("mrtma.cu", "tma.cuh", "mrpersist.cu", "mrcommon.cuh", "optile.cuh", "gridsync.cuh"):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (test infrastructure, timed as it stands)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    """In a spawned process with one BLAS thread: time the oracle's recycled MINRES
    (its own operator, a 10-column local space) on the workload's image for about
    `seconds`; returns (steps, seconds)."""
    name, seconds, seed = args
    import numpy as np

    import synth
    from oracle.minres import recycled_minres
    from oracle.operator import Operator, make_data
    wl = synth.WORKLOADS[name]
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    _, b = make_data(op, x, z, wl.eta)
    K, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((wl.n, 10)))
    w = np.ones(2 * wl.n)
    g = float(wl.gammas()[wl.M // 2])
    steps, t0 = 0, time.perf_counter()
    while True:
        res = recycled_minres(lambda v: op.apply(v, g, w), b, K, 0.0, 3)
        steps += res.iters
        el = time.perf_counter() - t0
        if el >= seconds:
            return steps, el


def _oracle_setup_sample(name, frac):
    """The oracle's per-step dense work (Algorithm "Stabilized U" on the 2p-column
    pre-stabilize basis and the QR of Eq. establishU on p columns) on 1/frac of the
    rows; returns its seconds scaled to all rows (both are linear in the rows)."""
    import numpy as np

    import synth
    from oracle.recycle import stabilize
    wl = synth.WORKLOADS[name]
    rows = max(1024, wl.n // frac)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((rows, 2 * wl.p))
    t0 = time.perf_counter()
    Q = stabilize(U, wl.p)
    np.linalg.qr(Q + 1e-3 * rng.standard_normal(Q.shape))
    return (time.perf_counter() - t0) * wl.n / rows


def _blas_env(threads):
    return {k: str(threads) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}


def _spawn_pool(procs, threads):
    """A spawned process pool whose workers start with `threads` BLAS threads."""
    import multiprocessing as mp
    env = _blas_env(threads)
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return mp.get_context("spawn").Pool(procs)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def setup_seconds(name, threads):
    """_oracle_setup_sample in a fresh process with `threads` BLAS threads."""
    pool = _spawn_pool(1, threads)
    try:
        return pool.apply(_oracle_setup_sample, (name, 16))
    finally:
        pool.close()
        pool.join()


class OracleSampler:
    """Spawned worker processes (one BLAS thread each) that time the oracle."""

    def __init__(self, name, procs):
        self.name = name
        self.procs = procs
        self.pool = _spawn_pool(procs, 1)

    def rate(self, seconds):
        """Aggregate oracle MINRES steps per second of all workers over ~seconds."""
        res = self.pool.map(_oracle_worker, [(self.name, seconds, 7 + i) for i in range(self.procs)])
        return sum(s / el for s, el in res), sum(s for s, _ in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def usable_procs():
    n = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 1e9
        n = max(1, min(n, int(avail / 2.0)))     # about 1 GB per worker at 2048 x 2048
    except (ValueError, OSError, AttributeError):
        pass
    return n


def oracle_solves_per_s(steps_per_s, setup_s, mv_per_solve, solves_per_step):
    """Oracle solves/s from its MINRES-step rate (a step = one operator application
    plus its projections and updates) and its dense set-up per outer step."""
    per_step_s = solves_per_step * mv_per_solve / steps_per_s + setup_s
    return solves_per_step / per_step_s, per_step_s


# Work of the timed workload per solve, used to scale the oracle's sampled rate when no
# GPU run of the same process supplies it (the reference arm): operator applications per
# solve of the 2048 x 2048 workload (seeding solves, V^(new), images, local images,
# MINRES steps and FP64 residuals included), counted by the recycled solver on GB300.
MV_PER_SOLVE = {"C5": 351.5, "C2": 218.5}


def cpu_baseline(name, seconds, mv_per_solve, solves_per_step, procs):
    """The oracle on 1 and on all usable host cores (a bounded sample, extrapolated)."""
    out = {}
    model = cpu_model()
    for label, p in (("1", 1), ("all", procs)):
        smp = OracleSampler(name, p)
        try:
            smp.rate(1.0)                           # worker start-up and first touch
            rate, steps = smp.rate(seconds)
        finally:
            smp.close()
        setup = setup_seconds(name, p)
        value, per_step = oracle_solves_per_s(rate, setup, mv_per_solve, solves_per_step)
        out[label] = {"value": value, "unit": "solves/s", "cores": p, "kind": "oracle",
                      "cpu_model": model, "host_cores": os.cpu_count(),
                      "oracle_minres_steps_per_s": rate, "extrapolated_s_per_outer_step": per_step,
                      "sample": (f"{steps} recycled-MINRES steps of the FP64 oracle on this image "
                                 f"({p} process(es), one BLAS thread each, ~{seconds:.0f} s) at "
                                 f"{mv_per_solve:.1f} operator applications per solve, plus its "
                                 f"stabilize SVD and principal QR timed on 1/16 of the rows and scaled "
                                 f"({setup:.1f} s per outer step); {solves_per_step} solves per outer step")}
    return out


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------
def clocks_start(dev_index):
    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), f"--query-gpu={q}",
                              "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (FileNotFoundError, OSError):
        return None, path
    return p, path


def clocks_stop(p, path):
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [s.strip() for s in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
            "samples": len(sm)}


def fp64_fma_peak(dev):
    """FP64 FMA rate of this GPU's CUDA cores from the library's microbenchmark
    (rs_measure_fp64_fma), GFLOP/s; the nominal figure if it cannot run."""
    import ctypes

    import torch
    from paper_2306_15049_gb300 import recyc
    lib = recyc.load()
    props = torch.cuda.get_device_properties(dev)
    scratch = torch.empty(8 * props.multi_processor_count * 256, dtype=torch.float64, device=dev)
    out = ctypes.c_double(0.0)
    best = 0.0
    for _ in range(3):
        st = lib.rs_measure_fp64_fma(scratch.data_ptr(), scratch.numel() * 8,
                                     ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream), ctypes.byref(out))
        if st == recyc.RS_OK:
            best = max(best, out.value)
    return (best, "measured (rs_measure_fp64_fma: independent FMA chains on every SM)") if best > 0 else \
        (FP64_NOMINAL_GFLOPS, "nominal: 152 SMs x 4 flop/clk x 2070 MHz")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def reduce_over_ranks(dist, ms, counts, device):
    """Whole-job aggregation of the replicas: the slowest rank's time (max over
    ranks) and the work of all ranks (sum of the counts)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), [int(round(v)) for v in c.tolist()]


class Job:
    """One replica of the workload's outer loop on one GPU, through the C ABI.
    step() runs the next outer step k; after k = K-1 the job starts again."""

    def __init__(self, wl, precision, dev, plain=False, batched_local=0):
        import torch

        import synth
        from paper_2306_15049_gb300 import recyc
        from paper_2306_15049_gb300.workloads import desc_for
        self.torch, self.recyc, self.wl, self.dev = torch, recyc, wl, dev
        self.precision = precision
        self.desc = desc_for(wl, precision=recyc.RS_MIXED if precision == "mixed" else recyc.RS_FP64,
                             batched_local=batched_local)
        x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed).reshape(-1)
        z = synth.noise_direction(wl.height, wl.width, wl.seed).reshape(-1)
        xt = torch.tensor(x, dtype=torch.float64, device=dev)
        zt = torch.tensor(z, dtype=torch.float64, device=dev)
        self.d = torch.empty_like(xt)
        recyc.rs_synthesize_data(self.desc[0], xt, zt, wl.eta, self.d,
                                 torch.empty(1 << 20, dtype=torch.uint8, device=dev))
        del xt, zt
        self.workspace = torch.empty(recyc.rs_workspace_bytes(self.desc[0]), dtype=torch.uint8, device=dev)
        self.X = torch.empty(wl.M, wl.n, dtype=torch.float64, device=dev)
        self.w = torch.ones(2 * wl.n, dtype=torch.float64, device=dev)
        self.w_next = torch.empty_like(self.w)
        self.d_host = self.d.cpu().pin_memory()
        self.w_host = torch.ones(2 * wl.n, dtype=torch.float64).pin_memory()
        self.X_host = None
        self.plain = plain
        self.P = None
        self.k = 0
        self.stream = torch.cuda.current_stream(dev)
        self.timing = {"launches": [0, 0], "ms": [0.0, 0.0], "pixels": [0, 0], "bytes": [0.0, 0.0],
                       "flops": [0.0, 0.0], "phase_ms": {}}
        self.timing_on = False
        self.launches = 0
        self.h2d = self.d2h = 0

    def _collect_timing(self):
        if self.P is None or not self.timing_on:
            return
        t = self.P.rs_get_timing()
        for c in range(2):
            for key in ("launches", "ms", "pixels", "bytes", "flops"):
                self.timing[key][c] += t[key][c]
        for key, v in t["phase_ms"].items():
            self.timing["phase_ms"][key] = self.timing["phase_ms"].get(key, 0.0) + v
        self.P.rs_set_timing(True)            # resets the accumulated times

    def set_timing(self, on):
        self._collect_timing()
        self.timing_on = on
        if self.P is not None:
            self.P.rs_set_timing(on)

    def reset_timing(self):
        self._collect_timing()
        self.timing = {"launches": [0, 0], "ms": [0.0, 0.0], "pixels": [0, 0], "bytes": [0.0, 0.0],
                       "flops": [0.0, 0.0], "phase_ms": {}}

    def restart(self):
        """The next step starts the job at k = 0 on a new problem."""
        self._collect_timing()
        if self.P is not None:
            self.P.close()
            self.P = None
        self.k = 0

    def prepare_e2e(self):
        """The pinned host buffer for the solutions: allocated once, outside any timed
        region (a caller keeps its host buffers across steps)."""
        if self.X_host is None:
            self.X_host = self.torch.empty(self.wl.M, self.wl.n, dtype=self.torch.float64).pin_memory()

    def step(self, e2e=False):
        torch, recyc, wl = self.torch, self.recyc, self.wl
        if self.P is not None and self.k >= wl.K:
            self.restart()
        if self.P is None:
            if e2e:
                self.d.copy_(self.d_host, non_blocking=True)
                self.h2d += self.d.numel() * 8
            self.P = recyc.Problem(self.desc, self.d, workspace=self.workspace)
            self.P.rs_set_timing(self.timing_on)
            self.w.fill_(1.0)
            self.w_host.fill_(1.0)
        if e2e:
            self.w.copy_(self.w_host, non_blocking=True)
            self.h2d += self.w.numel() * 8
        P, k = self.P, self.k
        info0 = P.rs_get_info()
        P.rs_set_weights(self.w)
        if e2e and self.X_host is None:
            self.prepare_e2e()
        if self.plain:
            stats = P.rs_solve_plain(self.X)
            if e2e:
                self.X_host.copy_(self.X, non_blocking=True)
        else:
            P.rs_update_recycle(recyc.RS_INIT if k == 0 else recyc.RS_UPDATE)
            if e2e:
                # every solution lands in the pinned host buffer as soon as it is final
                # (the library's copy stream), while the next shifts solve; the call
                # returns once the last one has landed
                stats = P.rs_solve_shifts_host(self.X, self.X_host)
            else:
                stats = P.rs_solve_shifts(self.X)
        _, _, ls = P.rs_lcurve(self.X, wl.M)
        P.rs_irn_weights(self.X[ls], wl.beta, self.w_next)
        self.w, self.w_next = self.w_next, self.w
        if e2e:
            # on the job's stream: the step's closing event follows the copy
            self.w_host.copy_(self.w, non_blocking=True)
            self.d2h += (self.X.numel() + self.w.numel()) * 8
        info = P.rs_get_info()
        self.k += 1
        return {"k": k, "solves": wl.M, "matvecs": info["matvecs_total"] - info0["matvecs_total"],
                "iters": sum(s["iters"] for s in stats),
                "worst_relres": max(s["relres_true"] for s in stats), "nc": info["nc"],
                "minres_kernel": info["minres_kernel"], "tuned_variant": info["tuned_variant"],
                "kernel_launches": info["kernel_launches"],
                "launches_before": info0["kernel_launches"], "lstar": ls}


def run_steps(job, steps, e2e=False, keep_X_of_step0=False):
    """`steps` outer steps from k = 0, each bracketed by CUDA events on the job's stream
    (inputs far larger than L2: no flush needed between steps)."""
    torch = job.torch
    job.restart()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    res = []
    x0 = None
    torch.cuda.synchronize(job.dev)
    ev[0].record(job.stream)
    for i in range(steps):
        r = job.step(e2e=e2e)
        ev[i + 1].record(job.stream)
        res.append(r)
        if keep_X_of_step0 and r["k"] == 0 and x0 is None:
            x0 = job.X.clone()
    torch.cuda.synchronize(job.dev)
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[steps]), step_ms, res, x0


def per_k(step_ms, res):
    out = {}
    for ms, r in zip(step_ms, res):
        out.setdefault(r["k"], []).append(ms)
    return {str(k): round(sum(v) / len(v), 3) for k, v in sorted(out.items())}


def roofline_entry(job, ms_total, minres_kernel, wl, precision, fp64_peak, tuned_variant=-1):
    peaks, peak_kind = measured_peaks()
    tm = job.timing
    cat = 0 if tm["ms"][0] >= tm["ms"][1] else 1
    launches = max(1, tm["launches"][cat])
    tname = "float" if precision == "mixed" else "double"
    names = {3: f"k_mr_batch<{tname},{wl.radius}>", 2: f"k_mr_tma<{tname},{wl.radius}>",
             1: f"k_mr_resident<{tname},{wl.radius}>", 0: f"k_mr_persist<{tname},{wl.radius}>"}
    kname = names.get(minres_kernel, f"k_mr_matvec<{tname}>") if cat == 0 else \
        "k_op_apply<double> (FP64 true / refinement residual matvec)"
    entry = {"kernel": kname, "launches": tm["launches"][cat],
             "avg_launch_us": tm["ms"][cat] * 1000.0 / launches,
             "kernel_time_share_of_step": tm["ms"][cat] / ms_total if ms_total > 0 else None}
    if cat == 0 and minres_kernel == 2 and tuned_variant in (1, 2):
        entry["stencil"] = "A as two autocorrelation passes" if tuned_variant == 2 else "A as four blur passes"
    steps = tm["pixels"][cat] / wl.n
    if cat == 0 and precision == "mixed" and minres_kernel != 1:
        achieved = tm["bytes"][cat] / (tm["ms"][cat] / 1000.0) / 1e9
        bytes_per_launch = tm["bytes"][cat] / launches
        cap = TRAFFIC.get(kname)
        traffic, why = None, f"no ncu capture recorded for {kname}"
        if cap is not None:
            if cap["src"] == kernel_src_sha():
                traffic = cap["dram_per_alg"] * bytes_per_launch
                why = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of `bench.py --profile-case small` "
                       f"({cap['dram_per_alg']:.3f} of the algorithmic bytes), scaled to the timed launches")
            else:
                why = "kernel sources changed since the ncu capture"
        entry.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": why,
                      "peak_source": f"{peak_kind} hbm_gbs",
                      "algorithmic_bytes_per_launch": bytes_per_launch,
                      "us_per_minres_step": tm["ms"][cat] * 1000.0 / max(1.0, steps),
                      "bytes_per_step": "(12 + 2 s) n 4 (one recycled-MINRES iteration, s = local "
                                        "dimension: K_l read twice, 12 vectors of n floats)"})
    elif cat == 0 and minres_kernel == 1:
        # vectors of one solve fit in L2: bound by the grid barriers, reported per step
        entry.update({"bound": "latency", "us_per_minres_step": tm["ms"][cat] * 1000.0 / max(1.0, steps),
                      "achieved": None, "peak": None, "unit": "us/step", "frac": None, "traffic": None})
    else:
        achieved = tm["flops"][cat] / (tm["ms"][cat] / 1000.0) / 1e9
        entry.update({"bound": "alu", "achieved": achieved / 1e3, "peak": fp64_peak[0] / 1e3,
                      "unit": "TFLOP/s", "frac": achieved / fp64_peak[0], "traffic": None,
                      "peak_source": "FP64 FMA, " + fp64_peak[1],
                      "algorithmic_flops_per_launch": tm["flops"][cat] / launches})
    return entry


def rel_diff(a, b):
    import torch
    num = torch.linalg.vector_norm(a - b, dim=1)
    den = torch.linalg.vector_norm(b, dim=1).clamp_min(1e-300)
    return float((num / den).max().item())


def oracle_relres(wl, x_dev, gamma, w_dev):
    """||b - (A + gamma E) x|| / ||b|| recomputed on the host by the FP64 oracle's operator."""
    import numpy as np

    import synth
    from oracle.operator import Operator, make_data
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x_true = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    _, b = make_data(op, x_true, z, wl.eta)
    x = x_dev.cpu().numpy()
    w = w_dev.cpu().numpy()
    return float(np.linalg.norm(b - op.apply(x, gamma, w)) / np.linalg.norm(b))


def adjoint_rate(precision, dev, reps=2):
    """Differentiation workload (1024 x 1024, sigma 3, radius 10, 16 shifts): one
    forward pass (k = 0 principal space and all shifted solves) plus the adjoint
    solves on the same recycle space and d loss / d gamma, d loss / d w for the
    loss sum_l ||x_l - x_true||^2, passes per second (CUDA events, after one
    untimed pass)."""
    import torch

    import synth
    from paper_2306_15049_gb300 import recyc
    from paper_2306_15049_gb300.workloads import desc_for
    wl = synth.C4
    desc = desc_for(wl, precision=recyc.RS_MIXED if precision == "mixed" else recyc.RS_FP64)
    x = torch.tensor(synth.piecewise_constant_image(wl.height, wl.width, wl.seed).reshape(-1),
                     dtype=torch.float64, device=dev)
    z = torch.tensor(synth.noise_direction(wl.height, wl.width, wl.seed).reshape(-1),
                     dtype=torch.float64, device=dev)
    d = torch.empty_like(x)
    recyc.rs_synthesize_data(desc[0], x, z, wl.eta, d, torch.empty(1 << 20, dtype=torch.uint8, device=dev))
    ws = torch.empty(recyc.rs_workspace_bytes(desc[0]), dtype=torch.uint8, device=dev)
    w = torch.ones(2 * wl.n, dtype=torch.float64, device=dev)
    X = torch.empty(wl.M, wl.n, dtype=torch.float64, device=dev)
    G = torch.empty_like(X)
    Lam = torch.empty_like(X)
    dw = torch.empty(2 * wl.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def one():
        P = recyc.Problem(desc, d, workspace=ws)
        P.rs_set_weights(w)
        P.rs_update_recycle(recyc.RS_INIT)
        P.rs_solve_shifts(X)
        torch.sub(X, x, out=G)
        G.mul_(2.0)
        st = P.rs_solve_adjoint(G, Lam)
        P.rs_shift_gradients(X, Lam, dw)
        P.close()
        return st

    one()
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        st = one()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / reps
    return {"value": 1000.0 / ms, "unit": "forward+adjoint gradient passes/s", "ms_per_pass": ms,
            "precision": precision,
            "workload": "1024x1024, sigma 3, radius 10, 16 shifts 1e-5..1, p=40, |J|=8, k=0; "
                        "loss sum_l ||x_l - x_true||^2; gradients w.r.t. the 16 shifts and the 2n weights",
            "adjoint_iters": sum(s_["iters"] for s_ in st),
            "worst_adjoint_relres": max(s_["relres_true"] for s_ in st)}


def batched_images_rate(precision, dev, reps=2):
    """The four images of uneven size (256^2 .. 1024^2, sigma 1.5 .. 3, radius
    4 .. 10), 32 shifts each, batched local spaces; one outer step (k = 0) of all
    four solved jointly (every shift of every image in one persistent launch)
    against the four solved one after another (solves/s, CUDA events)."""
    import torch

    import synth
    from paper_2306_15049_gb300 import recyc
    from paper_2306_15049_gb300.workloads import desc_for
    prec = recyc.RS_MIXED if precision == "mixed" else recyc.RS_FP64
    items = []
    for wl in synth.C3:
        desc = desc_for(wl, precision=prec, batched_local=1)
        x = torch.tensor(synth.piecewise_constant_image(wl.height, wl.width, wl.seed).reshape(-1),
                         dtype=torch.float64, device=dev)
        z = torch.tensor(synth.noise_direction(wl.height, wl.width, wl.seed).reshape(-1),
                         dtype=torch.float64, device=dev)
        d = torch.empty_like(x)
        recyc.rs_synthesize_data(desc[0], x, z, wl.eta, d, torch.empty(1 << 20, dtype=torch.uint8, device=dev))
        ws = torch.empty(recyc.rs_workspace_bytes(desc[0]), dtype=torch.uint8, device=dev)
        X = torch.empty(wl.M, wl.n, dtype=torch.float64, device=dev)
        w = torch.ones(2 * wl.n, dtype=torch.float64, device=dev)
        items.append((wl, desc, d, ws, X, w))
    stream = torch.cuda.current_stream(dev)

    def one(joint):
        probs = []
        for wl, desc, d, ws, X, w in items:
            P = recyc.Problem(desc, d, workspace=ws)
            P.rs_set_weights(w)
            P.rs_update_recycle(recyc.RS_INIT)
            probs.append(P)
        if joint:
            st = recyc.rs_solve_shifts_batched(probs, [it[4] for it in items])
        else:
            st = [P.rs_solve_shifts(it[4]) for P, it in zip(probs, items)]
        for P in probs:
            P.close()
        return st

    out = {}
    # joint: the library call pinned to one launch for all shifts (RS_BATCH_JOINT=1);
    # tuned: the library call as it stands (after its first two calls have timed the
    # joint and the per-problem launches); one_by_one: rs_solve_shifts per image
    for name, joint, env in (("joint", True, "1"), ("tuned", True, None), ("one_by_one", False, None)):
        old = os.environ.get("RS_BATCH_JOINT")
        if env is None:
            os.environ.pop("RS_BATCH_JOINT", None)
        else:
            os.environ["RS_BATCH_JOINT"] = env
        try:
            for _ in range(3 if name == "tuned" else 1):
                one(joint)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                st = one(joint)
            b.record(stream)
            torch.cuda.synchronize(dev)
        finally:
            if old is None:
                os.environ.pop("RS_BATCH_JOINT", None)
            else:
                os.environ["RS_BATCH_JOINT"] = old
        ms = a.elapsed_time(b) / reps
        solves = sum(len(x) for x in st)
        out[name] = {"value": solves / (ms / 1000.0), "unit": "solves/s", "ms_per_step": ms,
                     "worst_true_relres": max(s_["relres_true"] for x in st for s_ in x)}
    out["workload"] = ("images 256^2, 384^2, 512^2, 1024^2 (sigma 1.5, 2, 2.5, 3; radius 4, 6, 8, 10), "
                       "32 shifts 1e-5..1 each, p=40, |J|=8, batched local spaces, k=0; a step = "
                       "principal spaces of the four images + all 128 shifted solves")
    out["precision"] = precision
    return out


def whole_job(wl, precision, dev, reps=2, plain=False, batched_local=0):
    """The whole outer loop of a small workload (K steps) per pass, solves/s."""
    job = Job(wl, precision, dev, plain=plain, batched_local=batched_local)
    run_steps(job, wl.K)
    job.set_timing(True)
    job.reset_timing()
    ms, step_ms, res, _ = run_steps(job, wl.K * reps)
    job.restart()
    solves = sum(r["solves"] for r in res)
    out = {"value": solves / (ms / 1000.0), "unit": "solves/s", "ms_per_job": ms / reps,
           "matvecs_per_solve": sum(r["matvecs"] for r in res) / solves,
           "iters_per_job": sum(r["iters"] for r in res) / reps,
           "worst_true_relres": max(r["worst_relres"] for r in res)}
    if not plain:
        tm = job.timing
        steps = tm["pixels"][0] / wl.n
        out["minres_kernel_us_per_step"] = tm["ms"][0] * 1000.0 / max(1.0, steps)
        out["minres_bound"] = ("latency (one solve's vectors stay in L2; two grid barriers and the "
                               "cross-CTA reductions per step)" if res[-1]["minres_kernel"] == 1 else "hbm")
    return out


def oracle_parity_c1(dev):
    """The 64 x 64 workload (3 outer steps, 8 shifts) solved by the FP64 oracle on the
    host and by the GPU in FP64 and in mixed precision from the oracle's weights:
    the largest relative solution difference over all systems."""
    import numpy as np
    import torch

    import synth
    from oracle.operator import Operator, irn_weights, make_data
    from oracle.outer import run as oracle_run
    from oracle.recycle import Params
    from paper_2306_15049_gb300 import recyc
    from paper_2306_15049_gb300.workloads import desc_for
    wl = synth.C1
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    prm = Params.from_workload(wl)
    prm.maxit = min(prm.maxit, 100_000)
    steps, lstars = oracle_run(op, b, d, wl.gammas(), prm, wl.K, wl.beta)
    weights = [np.ones(2 * wl.n)] + [irn_weights(op, steps[k].X[lstars[k]], wl.beta) for k in range(wl.K - 1)]
    out = {"workload": "64x64, sigma 1.5, radius 4, 8 shifts 1e-4..1, 3 outer steps, p=10 "
                       "(oracle's weights at every step)"}
    for precision in ("fp64", "mixed"):
        desc = desc_for(wl, precision=recyc.RS_MIXED if precision == "mixed" else recyc.RS_FP64,
                        maxit=prm.maxit)
        dg = torch.tensor(d, dtype=torch.float64, device=dev)
        P = recyc.Problem(desc, dg)
        worst, worst_res = 0.0, 0.0
        for k, w in enumerate(weights):
            P.rs_set_weights(torch.tensor(w, dtype=torch.float64, device=dev))
            P.rs_update_recycle(recyc.RS_INIT if k == 0 else recyc.RS_UPDATE)
            X = torch.empty(wl.M, wl.n, dtype=torch.float64, device=dev)
            st = P.rs_solve_shifts(X)
            Xn = X.cpu().numpy()
            for l in range(wl.M):
                worst = max(worst, float(np.linalg.norm(Xn[l] - steps[k].X[l]) / np.linalg.norm(steps[k].X[l])))
                worst_res = max(worst_res, st[l]["relres_true"])
        P.close()
        out[precision] = {"max_rel_err_vs_oracle": worst, "worst_true_relres": worst_res}
    return out


def profile_case(args, wl, dev):
    import torch

    import synth
    from paper_2306_15049_gb300 import recyc
    if args.profile_case in ("step", "job"):
        # the first two outer steps (k = 0: seeding solves; k = 1: Eq. delta update), or all K
        job = Job(wl, args.precision, dev)
        rs = [job.step() for _ in range(2 if args.profile_case == "step" else wl.K)]
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": args.profile_case, "workload": wl.name, "precision": args.precision,
                          "steps": rs}), flush=True)
        return
    small = synth.tiny(wl.height, wl.width, sigma=wl.sigma, radius=wl.radius, M=4, p=12,
                       n_ritz_local=wl.n_ritz_local, seed=wl.seed, tol=wl.tol, log_lo=wl.log_lo,
                       eta=wl.eta)
    job = Job(small, args.precision, dev)
    P = recyc.Problem(job.desc, job.d, workspace=job.workspace)
    P.rs_set_weights(job.w)
    g = torch.Generator(device=dev).manual_seed(5)
    U = torch.randn(12, small.n, dtype=torch.float64, device=dev, generator=g)
    P.rs_set_recycle_basis(U, 12)
    stats = P.rs_solve_shifts(job.X, iters_override=[24] * small.M)
    torch.cuda.synchronize(dev)
    info = P.rs_get_info()
    print(json.dumps({"profile_case": "small", "precision": args.precision, "image": [wl.height, wl.width],
                      "radius": wl.radius, "iters": sum(s["iters"] for s in stats),
                      "local_dims": [s["local_dim"] for s in stats],
                      "minres_kernel": info["minres_kernel"], "kernel_launches": info["kernel_launches"],
                      "device_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2)}), flush=True)


def reference_arm(args, wl, config, rank):
    """The FP64 oracle on the host cores, timed as it stands: each step a bounded
    sample of the workload (its recycled MINRES steps on the workload's image, all
    usable cores), extrapolated to the solves of one outer step."""
    if rank != 0:
        return
    procs = usable_procs()
    mv = MV_PER_SOLVE.get(args.workload, 300.0)
    per = max(1.0, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    setup = setup_seconds(args.workload, procs)
    smp = OracleSampler(args.workload, procs)
    try:
        for _ in range(max(1, args.warmup)):
            smp.rate(per)
        rates, total = [], 0
        for _ in range(args.steps):
            r, s = smp.rate(per)
            rates.append(r)
            total += s
    finally:
        smp.close()
    rate = sum(rates) / len(rates)
    value, per_step = oracle_solves_per_s(rate, setup, mv, wl.M)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config, precision="fp64 (oracle)"),
        "oracle_minres_steps_per_s": rate,
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": procs, "kind": "oracle",
                         "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
                         "sample": f"{args.steps} samples of ~{per:.0f} s: {total} recycled-MINRES steps of "
                                   f"the FP64 oracle on this image in {procs} processes (one BLAS thread each), "
                                   f"at {mv:.1f} operator applications per solve, plus the stabilize SVD and "
                                   f"principal QR timed on 1/16 of the rows and scaled ({setup:.1f} s per outer "
                                   f"step); ms_per_step is that extrapolation to one outer step"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    import synth
    wl = synth.WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    config = workload_config(wl, args.precision)
    if args.impl == "reference":
        reference_arm(args, wl, config, rank)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if args.profile_case:
        profile_case(args, wl, dev)
        return
    fp64_peak = fp64_fma_peak(dev)
    job = Job(wl, args.precision, dev)
    config["device_workspace_gb"] = round(job.workspace.numel() / 1e9, 3)
    config["l2"] = f"inputs larger than L2 (a {config['device_workspace_gb']} GB workspace; no flush)"

    run_steps(job, max(3, args.warmup))
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    props = torch.cuda.get_device_properties(dev)
    smi_id = str(getattr(props, "uuid", local))
    if smi_id and not smi_id.startswith("GPU-") and len(smi_id) > 8:
        smi_id = "GPU-" + smi_id
    job.set_timing(True)
    job.reset_timing()
    clk_p, clk_path = clocks_start(smi_id)
    ms, step_ms, res, X_k0 = run_steps(job, args.steps, keep_X_of_step0=True)
    clocks = clocks_stop(clk_p, clk_path)
    job.set_timing(False)
    # the library's own process-wide launch counter across the timed steps
    launches_timed = res[-1]["kernel_launches"] - res[0]["launches_before"]
    solves = sum(r["solves"] for r in res)
    mvs = sum(r["matvecs"] for r in res)
    if dist:
        torch.cuda.synchronize(dev)
        dist.barrier()
        ms, (solves, mvs) = reduce_over_ranks(dist, ms, [solves, mvs], dev)
    value = solves / (ms / 1000.0)
    w_k0 = torch.ones(2 * wl.n, dtype=torch.float64, device=dev)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 Krylov + f64 refinement" if args.precision == "mixed" else "f64",
        "data": "synthetic", "config": config,
        "matvecs_per_s": mvs / (ms / 1000.0),
        "run": {"ms_per_outer_step_by_k": per_k(step_ms, res),
                "matvecs_per_solve": mvs / max(1, solves),
                "minres_iters_per_solve": sum(r["iters"] for r in res) / max(1, solves),
                "worst_true_relres": max(r["worst_relres"] for r in res), "n_c": res[-1]["nc"],
                "tuned_variant": res[-1]["tuned_variant"],
                "phases_ms_per_step": {k: v / args.steps for k, v in job.timing["phase_ms"].items()}},
        "gpu_launches": int(launches_timed), "clocks": clocks,
        "roofline": roofline_entry(job, ms, res[-1]["minres_kernel"], wl, args.precision, fp64_peak,
                                   res[-1]["tuned_variant"]),
        "fp64_fma_peak": {"value": fp64_peak[0] / 1e3, "unit": "TFLOP/s", "source": fp64_peak[1]},
    }

    if not args.no_e2e:
        job.prepare_e2e()
        job.h2d = job.d2h = 0
        e_ms, e_step_ms, e_res, _ = run_steps(job, args.steps, e2e=True)
        e_solves = sum(r["solves"] for r in e_res)
        if dist:
            e_ms, (e_solves,) = reduce_over_ranks(dist, e_ms, [e_solves], dev)
        line["e2e"] = {"value": e_solves / (e_ms / 1000.0), "unit": "solves/s",
                       "h2d_bytes_per_step": job.h2d // args.steps, "d2h_bytes_per_step": job.d2h // args.steps,
                       "what": "data image (at k = 0) and weights w_k copied in from pinned host memory, all "
                               "solutions x^(k,.) and w_{k+1} copied back into pinned host memory, every step; "
                               "each solution copied by rs_solve_shifts_host as soon as it is final while the "
                               "next shifts solve, the step ending when every copy has landed",
                       "ms_per_outer_step_by_k": per_k(e_step_ms, e_res),
                       "matvecs_per_solve": sum(r["matvecs"] for r in e_res) /
                       max(1, sum(r["solves"] for r in e_res))}
    job.restart()

    if world == 1 and rank == 0:
        acc = {}
        # the FP64 oracle's own operator recomputes two solutions' residuals (host)
        try:
            g = wl.gammas()
            acc["oracle_operator_relres"] = {
                f"gamma_{l + 1}": oracle_relres(wl, X_k0[l], float(g[l]), w_k0) for l in (0, wl.M - 1)}
        except Exception as e:                       # the oracle is context here, never the result
            acc["oracle_operator_relres"] = f"unavailable: {e}"
        if not args.no_fp64_compare and args.precision == "mixed":
            j64 = Job(wl, "fp64", dev)
            f_ms, _, f_res, X64 = run_steps(j64, 1, keep_X_of_step0=True)
            k0_ms = [m for m, r in zip(step_ms, res) if r["k"] == 0]
            line["fp64_gpu"] = {"value": wl.M / (f_ms / 1000.0), "unit": "solves/s", "ms_per_step": f_ms,
                                "step": "k = 0 (seeding solves, principal space, 64 shifts)",
                                "mixed_ms_same_step": sum(k0_ms) / len(k0_ms) if k0_ms else None,
                                "matvecs": f_res[0]["matvecs"], "iters": f_res[0]["iters"],
                                "worst_true_relres": f_res[0]["worst_relres"]}
            acc["max_rel_diff_mixed_vs_fp64_gpu_k0"] = rel_diff(X_k0, X64)
            j64.restart()
            del j64, X64
        line["accuracy"] = acc
        if not args.no_plain:
            jp = Job(wl, args.precision, dev, plain=True)
            p_ms, p_step, p_res, _ = run_steps(jp, 2)
            jp.restart()
            rec = [m for m, r in zip(step_ms, res) if r["k"] in (0, 1)]
            line["no_recycling"] = {
                "value": sum(r["solves"] for r in p_res) / (p_ms / 1000.0), "unit": "solves/s",
                "ms_per_step": p_ms / 2, "steps": "k = 0, 1 (weights from its own L-curve)",
                "recycled_ms_per_step_same_k": sum(rec) / len(rec) if rec else None,
                "matvecs_per_solve": sum(r["matvecs"] for r in p_res) / sum(r["solves"] for r in p_res),
                "iters": sum(r["iters"] for r in p_res),
                "worst_true_relres": max(r["worst_relres"] for r in p_res)}
            del jp
        del X_k0
        torch.cuda.empty_cache()
        if not args.no_extras:
            line["C2"] = {"workload": "512x512, sigma 2.5, radius 8, 2% noise, 16 shifts 1e-5..1, 5 outer "
                                      "steps, p=40, |J|=8; a pass is the whole 5-step job",
                          "mixed": whole_job(synth.C2, "mixed", dev),
                          "mixed_batched_local": whole_job(synth.C2, "mixed", dev, batched_local=1),
                          "fp64": whole_job(synth.C2, "fp64", dev, reps=1),
                          "no_recycling": whole_job(synth.C2, "mixed", dev, plain=True, reps=1)}
            line["C1_oracle_parity"] = oracle_parity_c1(dev)
            line["batched_images_C3"] = batched_images_rate("mixed", dev)
            line["adjoint_C4"] = {"mixed": adjoint_rate("mixed", dev), "fp64": adjoint_rate("fp64", dev, reps=1)}
        if not args.no_cpu_baseline:
            cb = cpu_baseline(args.workload, args.cpu_seconds, mvs / max(1, solves), wl.M, usable_procs())
            line["cpu_baseline"] = cb["1"]
            line["cpu_baseline_all_cores"] = cb["all"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
