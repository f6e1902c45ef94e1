"""Record the oracle's own work counts for a workload (run by hand, once).

Runs the full outer loop of the FP64 oracle (L-curve + reweighting) on a
workload and writes its per-step matvec and solve counts to
``tests/golden/oracle_counts_<name>.json``. The CPU baseline of the benchmark
scales a timed, bounded sample of oracle matvecs by these counts.

Usage: python -m oracle.record_counts C2
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

import synth
from oracle.operator import Operator, make_data
from oracle.outer import run
from oracle.recycle import Params


def main(name: str) -> str:
    wl = synth.WORKLOADS[name]
    op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
    x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
    z = synth.noise_direction(wl.height, wl.width, wl.seed)
    d, b = make_data(op, x, z, wl.eta)
    prm = Params.from_workload(wl)
    t0 = time.time()
    steps, lstars = run(op, b, d, wl.gammas(), prm, wl.K, wl.beta)
    out = {
        "workload": wl.name,
        "generated_by": "python -m oracle.record_counts " + name,
        "seconds": time.time() - t0,
        "steps": [{"k": k, "nc": int(s.nc), "overhead_matvecs": int(s.overhead_matvecs),
                   "shift_matvecs": [int(v) for v in s.matvecs],
                   "iters": [int(v) for v in s.iters],
                   "relres_true": [float(v) for v in s.relres_true],
                   "lstar": int(lstars[k])} for k, s in enumerate(steps)],
    }
    out["total_matvecs"] = int(sum(s["overhead_matvecs"] + sum(s["shift_matvecs"]) for s in out["steps"]))
    out["total_solves"] = int(wl.K * wl.M)
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        f"oracle_counts_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return path


if __name__ == "__main__":
    print(main(sys.argv[1] if len(sys.argv) > 1 else "C2"))
