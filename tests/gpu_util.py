"""Helpers shared by the GPU parity tests: one workload set up twice, once in
the FP64 oracle (CPU) and once through the C ABI (GPU), from the same seeded
synthetic inputs."""
import numpy as np

import synth
from oracle.operator import Operator, RadonOperator, make_data
from oracle.recycle import Params


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def lib_ready():
    from paper_2306_15049_gb300 import build, recyc
    build.build()
    return recyc.load()


class Pair:
    """Oracle and GPU views of one workload."""

    def __init__(self, wl, precision=0, batched_local=0, maxit=None, x_image=None, guess=0, inner=0):
        torch = torch_cuda()
        lib_ready()
        from paper_2306_15049_gb300 import recyc
        from paper_2306_15049_gb300.workloads import desc_for
        self.wl = wl
        if wl.radon_angles:
            self.op = RadonOperator(wl.height, wl.width, wl.radon_angles)
        else:
            self.op = Operator(wl.height, wl.width, wl.sigma, wl.radius)
        x = synth.piecewise_constant_image(wl.height, wl.width, wl.seed)
        if x_image is not None:
            x = np.asarray(x_image, dtype=np.float64).reshape(wl.height, wl.width)
        if wl.radon_angles:
            z = synth.sinogram_noise(self.op.m, wl.seed)
        else:
            z = synth.noise_direction(wl.height, wl.width, wl.seed)
        self.x_true = x.reshape(-1)
        self.d, self.b = make_data(self.op, x, z, wl.eta)
        self.prm = Params.from_workload(wl, batched_local=bool(batched_local))
        self.prm.inner = "cg" if inner else "minres"
        # every workload here converges in a few thousand steps; a cap keeps a
        # regression from running for hours
        self.prm.maxit = min(self.prm.maxit, 20000) if maxit is None else maxit
        self.gammas = wl.gammas()
        self.desc = desc_for(wl, precision=precision, batched_local=batched_local,
                             maxit=self.prm.maxit, guess=guess, inner=inner)
        dev = torch.device("cuda:0")
        xt = torch.tensor(self.x_true, dtype=torch.float64, device=dev)
        zt = torch.tensor(z.reshape(-1), dtype=torch.float64, device=dev)
        dg = torch.empty(self.d.shape[0], dtype=torch.float64, device=dev)
        ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
        recyc.rs_synthesize_data(self.desc[0], xt, zt, wl.eta, dg, ws)
        self.d_gpu = dg
        self.P = recyc.Problem(self.desc, dg)
        self.torch = torch
        self.dev = dev

    def t(self, a):
        return self.torch.tensor(np.ascontiguousarray(a), dtype=self.torch.float64, device=self.dev)

    def n(self, t):
        return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
