"""The allocation-free data synthesis entry point, for callers that cannot
allocate device memory (for example a process whose device memory is held by
another allocator, so that it cannot set aside a workspace).

rs_synthesize_data_noalloc keeps its scratch in a fixed device array inside
the library instead of a caller workspace. Through the C ABI, two calls in a
row must give the same data image as rs_synthesize_data with a workspace,
within the FP64 tolerance of the operator tests. The first call is small (13
partial sums); the second is large enough that its reduction uses all 304
partial-sum slots the array is sized for, so stale slots of the first call
would show. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_synthesis_matches_the_workspace_entry_point_on_two_calls():
    import torch

    from paper_2306_15049_gb300 import build, recyc
    from paper_2306_15049_gb300.workloads import desc_for
    assert torch.cuda.is_available()
    build.build()
    lib = recyc.load()
    dev = torch.device("cuda:0")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    for call, (h, w, sigma, r, eta, seed) in enumerate([(130, 97, 2.0, 6, 0.02, 11),
                                                        (640, 512, 1.5, 4, 0.05, 12)]):
        wl = synth.tiny(h, w, sigma=sigma, radius=r, M=4, p=4, n_ritz_local=1, seed=seed)
        desc, keep = desc_for(wl)
        x = torch.tensor(synth.piecewise_constant_image(h, w, seed).reshape(-1), dtype=torch.float64,
                         device=dev)
        z = torch.tensor(synth.noise_direction(h, w, seed).reshape(-1), dtype=torch.float64, device=dev)
        d_ref = torch.empty_like(x)
        d_na = torch.full_like(x, float("nan"))
        st = lib.rs_synthesize_data(ctypes.byref(desc), x.data_ptr(), z.data_ptr(), eta,
                                    d_ref.data_ptr(), ws.data_ptr(), ws.numel(), None)
        assert st == recyc.RS_OK, lib.rs_last_error(None)
        st = lib.rs_synthesize_data_noalloc(ctypes.byref(desc), x.data_ptr(), z.data_ptr(), eta,
                                            d_na.data_ptr(), None)
        assert st == recyc.RS_OK, lib.rs_last_error(None)
        a, b = d_na.cpu().numpy(), d_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(b), call


def test_noalloc_synthesis_rejects_bad_sizes_without_touching_the_gpu():
    from paper_2306_15049_gb300 import build, recyc
    from paper_2306_15049_gb300.workloads import desc_for
    build.build()
    lib = recyc.load()
    desc, keep = desc_for(synth.tiny(8, 8, M=4, p=4, n_ritz_local=1))
    desc.height, desc.width = 1 << 15, 1 << 14      # 2^29 pixels: above the stated maximum
    st = lib.rs_synthesize_data_noalloc(ctypes.byref(desc), 1, 1, 0.01, 1, None)
    assert st == recyc.RS_EINVAL
    assert b"2^28" in lib.rs_last_error(None)
