"""The throughput microbenchmarks behind the roofline denominators (ges_peak_run): the atomic
kernel adds exactly the operations it reports, and the measured rates are plausible for the
device's SM count and clock (128 FP32 lanes per SM, and 32 special-function results per clock
and SM, the ex2 rate measured on this GB300, bound them from above)."""
import pytest
import torch

from paper_2411_09156_gb300 import _lib, peaks

pytestmark = pytest.mark.gpu


def test_atomic_kernel_adds_what_it_reports():
    sink = torch.zeros(16 * 4096, dtype=torch.float32, device="cuda")
    ops = peaks.run(peaks.KINDS["l2_atomic_add"], 1, 7, sink)
    torch.cuda.synchronize()
    assert ops > 0
    assert float(sink.double().sum()) == float(ops)


def test_measured_rates_are_below_the_nominal_per_sm_rates():
    pk = peaks.measure(reps=2)
    sms = pk["sm_count"]
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    ghz = 2.2  # above the GPU's maximum SM clock
    assert 0.3 * sms * 128 * 2 * 1.0e9 / 1e12 < pk["fp32_tflops"] <= sms * 128 * 2 * ghz * 1e9 / 1e12
    for k in ("mufu_ex2_gops", "mufu_rcp_gops"):
        assert 0.3 * sms * 16 * 1.0 < pk[k] <= sms * 32 * ghz, (k, pk[k])
    assert pk["l2_atomic_gops"] > 0


def test_bad_arguments_are_rejected():
    import ctypes
    sink = torch.zeros(256, dtype=torch.float32, device="cuda")
    ops = ctypes.c_uint64()
    lib = _lib.lib()
    for kind, bps, iters, n in ((4, 1, 1, 256), (0, 0, 1, 256), (0, 1, 0, 256), (0, 1, 1, 255), (3, 1, 1, 250)):
        st = lib.ges_peak_run(kind, bps, iters, ctypes.c_void_p(sink.data_ptr()), n, None, ctypes.byref(ops))
        assert st == _lib.GES_ERR_INVALID_ARG, (kind, bps, iters, n)
