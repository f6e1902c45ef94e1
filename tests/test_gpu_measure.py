"""The FP64 FMA-rate microbenchmark that bench.py takes as the peak of the FP64
kernels (rs_measure_fp64_fma, through the C ABI): a positive rate, below what
any GPU of this class could reach, and stable across calls."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_measured():
    import torch

    from paper_2306_15049_gb300 import build, recyc
    build.build()
    lib = recyc.load()
    dev = torch.device("cuda:0")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    scratch = torch.empty(8 * sms * 256, dtype=torch.float64, device=dev)
    rates = []
    for _ in range(2):
        out = ctypes.c_double(0.0)
        st = lib.rs_measure_fp64_fma(scratch.data_ptr(), scratch.numel() * 8, None, ctypes.byref(out))
        assert st == recyc.RS_OK, lib.rs_last_error(None)
        rates.append(out.value)
    assert all(10.0 < r < 100_000.0 for r in rates), rates          # GFLOP/s
    assert max(rates) < 1.5 * min(rates), rates
    bad = lib.rs_measure_fp64_fma(scratch.data_ptr(), 8, None, ctypes.byref(ctypes.c_double()))
    assert bad == recyc.RS_EINVAL
