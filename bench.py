#!/usr/bin/env python
"""Benchmark of the recycled shifted solves on GB300.

Workload (one step): the 512 x 512 image of the single-image workload
(sigma 2.5, radius 8, 2 % noise), 16 shifts log-spaced over 1e-5..1, 5 outer
reweighting steps (k = 0: principal space from two MINRES solves; k >= 1:
update by Eq. delta; the IRN weights from the L-curve corner), principal
recycle dimension 40, 8 local Ritz vectors, every system solved to a true
relative residual of 1e-8. All of it runs through librecyc's C ABI.

Metric: shifted solves per second (and matvecs per second) over the whole job,
inputs resident in HBM; `e2e` repeats it with the data image copied in from
pinned host memory and every step's solutions copied back. `roofline` is the
dominant kernel's achieved rate from CUDA events around its launches in the
timed region; `cpu_baseline` is the FP64 oracle on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "shifted solves/sec & matvecs/sec at rel. residual 1e-8; HBM GB/s vs roofline"
FP64_PEAK_GFLOPS = 152 * 2070e6 * 4 / 1e9   # 152 SMs x 2 FP64 FMA/clk x 2070 MHz (nominal 1.25 TF)
# DRAM bytes (read + write) per MINRES step of k_mr_resident<float, 8> on a 512 x 512
# image, from one ncu capture of 24-step launches (profiles/k_mr_resident_float_r8_512x512.md:
# 15.79 MB + 0.04 MB per launch); scaled to a launch by its steps
MR_RESIDENT_DRAM_BYTES_PER_STEP = {(512, 512, 8, "float"): (15.795e6 + 0.042e6) / 24}
# The same for the streaming kernel k_mr_persist<float, 12> on a 2048 x 2048 image
# (profiles/k_mr_persist_float_r12_2048x2048_dram.md: 10.46 GB + 2.10 GB per 24-step launch)
MR_PERSIST_DRAM_BYTES_PER_STEP = {(2048, 2048, 12, "float"): (10.46e9 + 2.10e9) / 24}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--workload", default="C2")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-local-space measurement of the same workload")
    ap.add_argument("--batched-local", action="store_true",
                    help="run the workload with batched local spaces (all shifts of a step in one launch)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the unrecycled comparison solver (every shift from x0 = 0)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the differentiation measurement on the 1024x1024 workload")
    ap.add_argument("--profile-case", nargs="?", const="full", choices=["full", "small"],
                    help="run the workload once for a profiler and exit (small: every shift of "
                         "the first outer step on a random principal basis, 24 MINRES steps each)")
    return ap.parse_args()


def workload_config(wl, precision):
    return {
        "workload": f"{wl.height}x{wl.width} image, sigma {wl.sigma}, radius {wl.radius}, "
                    f"{int(wl.eta * 100)}% noise; {wl.M} shifts 1e{int(wl.log_lo)}..1e{int(wl.log_hi)}; "
                    f"{wl.K} outer IRN steps; p={wl.p}, |J|={wl.n_ritz_local}; tol {wl.tol:g}",
        "n": wl.n, "shifts": wl.M, "outer_steps": wl.K, "p": wl.p, "local_ritz": wl.n_ritz_local,
        "precision": precision,
        "l2": "flushed between timed steps (256 MB write)",
        "parallelism": "replicas (one independent workload per GPU)",
    }


def oracle_counts(name):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_counts_{name}.json")
    with open(path) as f:
        return json.load(f)


def oracle_matvec_rate(wl, seconds):
    """FP64 oracle matvecs per second on this workload's operator (host cores)."""
    import numpy as np

    import synth
    from oracle.operator import Operator, make_data
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    w = synth.random_weights(wl.n, 1, lo=1.0, hi=1000.0)
    v = b.copy()
    count = 0
    t0 = time.perf_counter()
    c0 = time.process_time()
    while True:
        v = op.apply(v, 1e-3, w)
        v /= np.abs(v).max()      # keeps the iterate scaled (a ufunc reduction: no BLAS threads)
        count += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            oracle_matvec_rate.cpu_per_wall = (time.process_time() - c0) / el
            return count / el, count, el


def cpu_baseline(wl, name, seconds):
    rate, count, el = oracle_matvec_rate(wl, seconds)
    oc = oracle_counts(name)
    solves_per_s = rate * oc["total_solves"] / oc["total_matvecs"]
    return {
        "value": solves_per_s, "unit": "solves/s", "cores": 1, "kind": "oracle",
        "matvecs_per_s": rate,
        "process_cpu_s_per_wall_s": round(getattr(oracle_matvec_rate, "cpu_per_wall", float("nan")), 2),
        "sample": (f"FP64 NumPy oracle: {count} matvecs of this workload's operator in {el:.1f} s "
                   f"(1 thread), scaled by the oracle's own count for the whole workload "
                   f"({oc['total_matvecs']} matvecs for {oc['total_solves']} solves, "
                   f"tests/golden/oracle_counts_{name}.json)"),
    }, oc


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


def adjoint_rate(precision, dev, reps=2):
    """Differentiation workload (1024 x 1024, sigma 3, radius 10, 16 shifts): one
    forward pass (k = 0 principal space and all shifted solves) plus the adjoint
    solves on the same recycle space and d loss / d gamma, d loss / d w for the
    loss sum_l ||x_l - x_true||^2. Returns forward+backward passes per second
    (CUDA events, after one untimed pass) and the solve counts."""
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
        dg = P.rs_shift_gradients(X, Lam, dw)
        P.close()
        return st, dg

    one()
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        st, dg = one()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / reps
    return {"value": 1000.0 / ms, "unit": "forward+adjoint gradient passes/s",
            "ms_per_pass": ms, "precision": precision,
            "workload": "1024x1024, sigma 3, radius 10, 16 shifts 1e-5..1, p=40, |J|=8, k=0; "
                        "loss sum_l ||x_l - x_true||^2; gradients w.r.t. the 16 shifts and the 2n weights",
            "adjoint_iters": sum(s_["iters"] for s_ in st),
            "worst_adjoint_relres": max(s_["relres_true"] for s_ in st)}


def batched_images_rate(precision, dev, reps=2):
    """Batched workload: the four images of uneven size (256^2 .. 1024^2, sigma
    1.5 .. 3, radius 4 .. 10), 32 shifts each, batched local spaces; one outer step
    (k = 0) of all four solved jointly (every shift of every image in one
    persistent launch) against the four solved one after another. Returns
    solves per second of both (CUDA events, after one untimed pass)."""
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
    for joint in (True, False):
        one(joint)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            st = one(joint)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / reps
        solves = sum(len(x) for x in st)
        out["joint" if joint else "one_by_one"] = {
            "value": solves / (ms / 1000.0), "unit": "solves/s", "ms_per_step": ms,
            "worst_true_relres": max(s_["relres_true"] for x in st for s_ in x)}
    out["workload"] = ("images 256^2, 384^2, 512^2, 1024^2 (sigma 1.5, 2, 2.5, 3; radius 4, 6, 8, 10), "
                       "32 shifts 1e-5..1 each, p=40, |J|=8, batched local spaces, k=0; a step = "
                       "principal spaces of the four images + all 128 shifted solves")
    out["precision"] = precision
    return out


def reduce_over_ranks(dist, ms, counts, device):
    """Whole-job aggregation of the replicas: the slowest rank's time (max over
    ranks) and the work of all ranks (sum of the counts)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), [int(round(v)) for v in c.tolist()]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Runner:
    """One replica of the workload on one GPU, through the C ABI."""

    def __init__(self, wl, precision, dev, batched_local=0, plain=False):
        import numpy as np
        import torch

        import synth
        from paper_2306_15049_gb300 import recyc
        from paper_2306_15049_gb300.workloads import desc_for
        self.torch, self.recyc, self.wl, self.dev = torch, recyc, wl, dev
        self.desc = desc_for(wl, precision=recyc.RS_MIXED if precision == "mixed" else recyc.RS_FP64,
                             batched_local=batched_local)
        x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed).reshape(-1)
        z = synth.noise_direction(wl.height, wl.width, wl.seed).reshape(-1)
        xt = torch.tensor(x, dtype=torch.float64, device=dev)
        zt = torch.tensor(z, dtype=torch.float64, device=dev)
        self.d = torch.empty_like(xt)
        scratch = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
        recyc.rs_synthesize_data(self.desc[0], xt, zt, wl.eta, self.d, scratch)
        self.workspace = torch.empty(recyc.rs_workspace_bytes(self.desc[0]), dtype=torch.uint8, device=dev)
        self.X = torch.empty(wl.M, wl.n, dtype=torch.float64, device=dev)
        self.w = torch.ones(2 * wl.n, dtype=torch.float64, device=dev)
        self.w_next = torch.empty_like(self.w)
        self.d_host = self.d.cpu().pin_memory()
        self.w0_host = torch.ones(2 * wl.n, dtype=torch.float64).pin_memory()
        self.X_host = torch.empty(wl.M, wl.n, dtype=torch.float64).pin_memory()
        self.timing = {"launches": [0, 0], "ms": [0.0, 0.0], "pixels": [0, 0], "bytes": [0.0, 0.0],
                       "flops": [0.0, 0.0], "phase_ms": {}}
        self.last = None
        self.np = np
        # plain: the paper's comparison solver (every shift from x0 = 0, no recycling)
        self.plain = plain

    def step(self, timing=False, e2e=False):
        """The whole workload: K outer steps of all M shifts. Returns work counts."""
        torch, recyc, wl = self.torch, self.recyc, self.wl
        if e2e:
            self.d.copy_(self.d_host, non_blocking=True)
            self.w.copy_(self.w0_host, non_blocking=True)
        else:
            self.w.fill_(1.0)
        P = recyc.Problem(self.desc, self.d, workspace=self.workspace)
        if timing:
            P.rs_set_timing(True)
        solves, worst, iters = 0, 0.0, 0
        for k in range(wl.K):
            P.rs_set_weights(self.w)
            if self.plain:
                stats = P.rs_solve_plain(self.X)
            else:
                P.rs_update_recycle(recyc.RS_INIT if k == 0 else recyc.RS_UPDATE)
                stats = P.rs_solve_shifts(self.X)
            if e2e:
                self.X_host.copy_(self.X, non_blocking=True)
            solves += wl.M
            worst = max(worst, max(s["relres_true"] for s in stats))
            iters += sum(s["iters"] for s in stats)
            if k + 1 < wl.K:
                _, _, ls = P.rs_lcurve(self.X, wl.M)
                P.rs_irn_weights(self.X[ls], wl.beta, self.w_next)
                self.w, self.w_next = self.w_next, self.w
        info = P.rs_get_info()
        if timing:
            t = P.rs_get_timing()
            for c in range(2):
                self.timing["launches"][c] += t["launches"][c]
                self.timing["ms"][c] += t["ms"][c]
                self.timing["pixels"][c] += t["pixels"][c]
                self.timing["bytes"][c] += t["bytes"][c]
                self.timing["flops"][c] += t["flops"][c]
            for k, v in t["phase_ms"].items():
                self.timing["phase_ms"][k] = self.timing["phase_ms"].get(k, 0.0) + v
        P.close()
        self.last = {"solves": solves, "matvecs": info["matvecs_total"], "worst_relres": worst,
                     "iters": iters, "nc": info["nc"], "kernel_launches": info["kernel_launches"],
                     "minres_kernel": info["minres_kernel"]}
        return self.last


def timed(runner, steps, flush, timing=False, e2e=False):
    """Run `steps` steps; each bracketed by CUDA events; L2 flushed in between."""
    torch = runner.torch
    stream = torch.cuda.current_stream(runner.dev)
    tot_ms, solves, mvs = 0.0, 0, 0
    launches0 = None
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(runner.dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = runner.step(timing=timing, e2e=e2e)
        b.record(stream)
        torch.cuda.synchronize(runner.dev)
        tot_ms += a.elapsed_time(b)
        solves += r["solves"]
        mvs += r["matvecs"]
        if launches0 is None:
            launches0 = r["kernel_launches"]
    return tot_ms, solves, mvs


def main():
    args = parse()
    import synth
    wl = synth.WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    config = workload_config(wl, args.precision)
    if args.batched_local:
        config["local_spaces"] = "batched: [W, g^(k-1,l), g^(k-1,l-1)], every shift of a step in one launch"

    if args.impl == "reference":
        # the FP64 oracle on the host cores; under torchrun only rank 0 works
        if rank != 0:
            return
        rate_w, _, _ = oracle_matvec_rate(wl, 1.0) if args.warmup > 0 else (0, 0, 0)
        for _ in range(max(0, args.warmup - 1)):
            oracle_matvec_rate(wl, 0.5)
        oc = oracle_counts(args.workload)
        per = max(2.0, min(20.0, 90.0 / max(1, args.steps)))
        rates = []
        samples = 0
        for _ in range(args.steps):
            r, c, el = oracle_matvec_rate(wl, per)
            rates.append(r)
            samples += c
        rate = sum(rates) / len(rates)
        value = rate * oc["total_solves"] / oc["total_matvecs"]
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * oc["total_matvecs"] / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config, precision="fp64 (oracle)"),
            "matvecs_per_s": rate,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} samples of {per:.0f} s of oracle FP64 matvecs "
                                       f"({samples} matvecs, 1 thread) scaled by the oracle's own "
                                       f"{oc['total_matvecs']} matvecs for {oc['total_solves']} solves; "
                                       "ms_per_step is that extrapolation"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
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
    runner = Runner(wl, args.precision, dev, batched_local=int(args.batched_local))
    config["device_workspace_gb"] = round(runner.workspace.numel() / 1e9, 3)
    if args.profile_case == "full":
        r = runner.step()
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": wl.name, "precision": args.precision, **r}), flush=True)
        return
    if args.profile_case == "small":
        from paper_2306_15049_gb300 import recyc
        P = recyc.Problem(runner.desc, runner.d, workspace=runner.workspace)
        P.rs_set_weights(runner.w)
        g = torch.Generator(device=dev).manual_seed(5)
        U = torch.randn(wl.p, wl.n, dtype=torch.float64, device=dev, generator=g)
        P.rs_set_recycle_basis(U, wl.p)
        stats = P.rs_solve_shifts(runner.X, iters_override=[24] * wl.M)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": "small", "precision": args.precision,
                          "iters": sum(s["iters"] for s in stats),
                          "kernel_launches": P.rs_get_info()["kernel_launches"]}), flush=True)
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    for _ in range(max(3, args.warmup)):
        runner.step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    props = torch.cuda.get_device_properties(dev)
    smi_id = str(getattr(props, "uuid", local))
    if smi_id and not smi_id.startswith("GPU-") and len(smi_id) > 8:
        smi_id = "GPU-" + smi_id
    launches_before = runner.last["kernel_launches"]
    clk_p, clk_path = clocks_start(smi_id)
    ms, solves, mvs = timed(runner, args.steps, flush, timing=True)
    clocks = clocks_stop(clk_p, clk_path)
    launches_timed = runner.last["kernel_launches"] - launches_before
    run_stats = dict(runner.last)
    if dist:
        ms, (solves, mvs) = reduce_over_ranks(dist, ms, [solves, mvs], dev)
    ms_per_step = ms / args.steps
    value = solves / (ms / 1000.0)

    # end to end: host data in, every step's solutions out
    runner.step(e2e=True)
    e_ms, e_solves, _ = timed(runner, args.steps, flush, e2e=True)
    if dist:
        e_ms, (e_solves,) = reduce_over_ranks(dist, e_ms, [e_solves], dev)
    e2e = {"value": e_solves / (e_ms / 1000.0), "unit": "solves/s",
           "h2d_bytes_per_step": 8 * (wl.n + 2 * wl.n),
           "d2h_bytes_per_step": 8 * wl.K * wl.M * wl.n}

    # roofline of the dominant kernel (live CUDA-event times from the timed region)
    peaks, peak_kind = measured_peaks()
    tm = runner.timing
    cat = 0 if tm["ms"][0] >= tm["ms"][1] else 1
    launches = max(1, tm["launches"][cat])
    avg_s = tm["ms"][cat] / 1000.0 / launches
    tname = "float" if args.precision == "mixed" else "double"
    mk = runner.last.get("minres_kernel", -1)
    if cat == 1:
        kname = "k_op_apply<double> (FP64 true / refinement residual matvec)"
    elif mk == 3:
        kname = ("k_mr_batch<%s,%d> (one cooperative launch for all shifts of a step, "
                 "convergence masks)" % (tname, wl.radius))
    elif mk == 1:
        kname = ("k_mr_resident<%s,%d> (one cooperative launch per solve, one CTA per 32x32 tile, "
                 "two grid-wide barriers per MINRES step)" % (tname, wl.radius))
    elif mk == 0:
        kname = ("k_mr_persist<%s,%d> (one cooperative launch per solve, tiles streamed through "
                 "memory)" % (tname, wl.radius))
    else:
        kname = ("k_mr_matvec<%s> (fused MINRES step: direction update, v_j, (A+gamma E) v_j, K^T y)"
                 % tname)
    traffic = None
    per_step = (MR_RESIDENT_DRAM_BYTES_PER_STEP if mk == 1 else MR_PERSIST_DRAM_BYTES_PER_STEP if mk == 0
                else {}).get((wl.height, wl.width, wl.radius, tname))
    if cat == 0 and per_step is not None:
        traffic = per_step * tm["pixels"][0] / wl.n / launches
    if cat == 0 and args.precision == "mixed":
        achieved = tm["bytes"][cat] / (tm["ms"][cat] / 1000.0) / 1e9
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": tm["bytes"][cat] / launches}
    else:
        achieved = tm["flops"][cat] / (tm["ms"][cat] / 1000.0) / 1e9
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved / 1e3,
                "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": None, "peak_source": "nominal FP64: 152 SMs x 4 flop/clk x 2070 MHz",
                "algorithmic_flops_per_launch": tm["flops"][cat] / launches}
    if traffic is not None:
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of 24-step launches "
                                  "of the same kernel, scaled by the timed launches' steps per launch")
    roof["launches"] = tm["launches"][cat]
    roof["avg_launch_us"] = avg_s * 1e6
    roof["kernel_time_share_of_step"] = tm["ms"][cat] / ms if ms > 0 else None

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 Krylov + f64 refinement" if args.precision == "mixed" else "f64",
        "data": "synthetic", "config": config,
        "matvecs_per_s": mvs / (ms / 1000.0),
        "run": {"matvecs_per_step": run_stats["matvecs"], "iters_per_step": run_stats["iters"],
                "worst_true_relres": run_stats["worst_relres"], "n_c": run_stats["nc"],
                "phases_ms_per_step": {k: v / args.steps for k, v in tm["phase_ms"].items()}},
        # kernels the library launched inside the timed region (its own counter)
        "gpu_launches": int(launches_timed), "clocks": clocks, "roofline": roof, "e2e": e2e,
    }

    if not args.no_batched:
        # the same workload with batched local spaces: all 16 shifts of a step in
        # one cooperative launch (convergence masks), against the shift-by-shift path
        rb = Runner(wl, args.precision, dev, batched_local=1)
        rb.step()
        b_ms, b_solves, b_mvs = timed(rb, max(1, args.steps), flush)
        line["batched_local"] = {"value": b_solves / (b_ms / 1000.0), "unit": "solves/s",
                                 "ms_per_step": b_ms / max(1, args.steps),
                                 "matvecs_per_s": b_mvs / (b_ms / 1000.0),
                                 "worst_true_relres": rb.last["worst_relres"],
                                 "iters_per_step": rb.last["iters"],
                                 "variant": "local spaces [W, g^(k-1,l), g^(k-1,l-1)]; every shift "
                                            "of a step in one persistent cooperative launch"}
    if not args.no_batched and world == 1:
        line["batched_images_C3"] = batched_images_rate(args.precision, dev)
    if not args.no_adjoint and world == 1:
        line["adjoint_C4"] = {"mixed": adjoint_rate("mixed", dev), "fp64": adjoint_rate("fp64", dev, reps=1)}
    if not args.no_fp64_compare and args.precision == "mixed":
        r64 = Runner(wl, "fp64", dev)
        r64.step()
        f_ms, f_solves, f_mvs = timed(r64, 1, flush)
        line["fp64_gpu"] = {"value": f_solves / (f_ms / 1000.0), "unit": "solves/s",
                            "ms_per_step": f_ms, "matvecs_per_s": f_mvs / (f_ms / 1000.0),
                            "worst_true_relres": r64.last["worst_relres"]}
    if not args.no_plain and world == 1:
        # the paper's comparison: the same outer iteration with every shift solved
        # from x0 = 0 without recycling (same inner solver, tolerance and precision)
        rp = Runner(wl, args.precision, dev, plain=True)
        rp.step()
        p_ms, p_solves, p_mvs = timed(rp, 1, flush)
        line["no_recycling"] = {"value": p_solves / (p_ms / 1000.0), "unit": "solves/s",
                                "ms_per_step": p_ms, "matvecs_per_solve": p_mvs / p_solves,
                                "recycled_matvecs_per_solve": run_stats["matvecs"] / run_stats["solves"],
                                "iters_per_step": rp.last["iters"],
                                "worst_true_relres": rp.last["worst_relres"],
                                "note": "recycled matvecs include the recycle space's own "
                                        "(seeding solves, V_new steps, AU/EU images, local images)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(wl, args.workload, args.cpu_seconds)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
