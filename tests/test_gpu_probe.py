"""The FP32 and FP64 throughput probes. The FP32 one (g6x_fp32_probe): its measured rate lies
between half of and 1.05x the rate derived from the unit counts at GB300's
maximum SM clock (SMs x 128 FP32 lanes x 2 flop x 2070 MHz), which is the
force kernel's roofline denominator; bad arguments are refused."""
import pytest

from paper_0902_4463_gb300 import g6gb as g6

pytestmark = pytest.mark.gpu


def test_fp32_probe_against_derived_peak():
    import torch
    from paper_0902_4463_gb300 import build
    build.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2070e6 / 1e12
    tf, ms = g6.g6x_fp32_probe(4000)
    assert ms > 0 and 0.5 * derived <= tf <= 1.05 * derived, (tf, derived, ms)
    for bad in (0, -1, 1 << 25):
        with pytest.raises(g6.G6Error):
            g6.g6x_fp32_probe(bad)


def test_fp64_probe_is_a_small_fraction_of_fp32():
    """GB300's FP64 pipe is far narrower than its FP32 pipe (nominally about
    1/60 of the rate); the probe must land in that range, not near FP32."""
    from paper_0902_4463_gb300 import build
    build.build()
    tf32, _ = g6.g6x_fp32_probe(2000)
    tf64, ms = g6.g6x_fp64_probe(100)
    assert ms > 0 and 0.0 < tf64 < tf32 / 8, (tf64, tf32)
    for bad in (0, -1, 1 << 25):
        with pytest.raises(g6.G6Error):
            g6.g6x_fp64_probe(bad)
