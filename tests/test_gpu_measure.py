"""The measured FP32 peak (the degridding roofline's denominator) is
plausible: below the unit-count bound at the maximum SM clock, and not far
below it (a kernel that did less work than it counts would read above the
bound; one that failed to fill the SMs would read far below it)."""
import pytest

torch = pytest.importorskip("torch")

import paper_2102_12739_gb300 as dg  # noqa: E402

pytestmark = pytest.mark.gpu

FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0         # GB300 maximum SM clock


def test_measured_fp32_peak_is_within_the_unit_count_bound():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
    for packed in (True, False):
        t = dg.measure_fp32_peak(0, packed=packed)
        assert 0.5 * bound < t <= 1.01 * bound, (packed, t, bound)


def test_measure_fp32_peak_rejects_bad_arguments():
    with pytest.raises(dg.DegridError):
        dg.measure_fp32_peak(-1)
