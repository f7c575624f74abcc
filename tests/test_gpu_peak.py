"""The binary64 pipe measurement (fdlb_measure_fp64_pipe), the roofline
denominator of the binary64 stage kernels: a positive rate no higher than
the nominal 2 DFMA lanes per clock per SM at the device's maximum clock (a
rate above it would mean the timed kernel is not doing its work), and within
reach of it (8 independent chains per thread on 2048 threads per SM), stable
from call to call."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_pipe_rate_is_physical():
    import torch
    from paper_1909_08390_gb300 import build as B, fdlb
    B.build()
    fdlb.load()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    clock_ghz = 2.07  # the part's maximum SM clock
    nominal = sms * 2 * clock_ghz * 1e9
    rates = []
    for _ in range(3):
        r, ms = fdlb.fdlb_measure_fp64_pipe()
        assert ms > 0.0
        rates.append(r)
    print("DFMA/s: " + ", ".join("%.4g" % r for r in rates) + " (nominal %.4g)" % nominal)
    for r in rates:
        assert 0.5 * nominal < r <= 1.02 * nominal, (r, nominal)
    assert max(rates) / min(rates) < 1.05
