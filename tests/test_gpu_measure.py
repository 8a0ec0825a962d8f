"""The measured device peaks are plausible.  The FP32 peak (the degridding
roofline's denominator) lies below the unit-count bound at the maximum SM
clock and not far below it: a kernel that did less work than it counts would
read above the bound, one that failed to fill the SMs far below it.  The L2
read bandwidth lies above the HBM copy rate (the buffer is L2-resident) and
below what the SMs' load paths could take in (128 bytes per SM per clock)."""
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


def test_measured_l2_read_bandwidth_is_between_hbm_and_the_load_path_bound():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    upper = sms * 128 * MAX_SM_MHZ * 1e6 / 1e9
    bw = dg.measure_l2_read_bw(0)
    assert 7000.0 < bw <= upper, (bw, upper)
    with pytest.raises(dg.DegridError):
        dg.measure_l2_read_bw(-1)


def test_measured_l2_reduce_rate_is_plausible():
    # the copy engines' reduce-adds of footprint tiles into an L2-resident
    # stack: above 1 TB/s of added data (else the kernel did not keep them
    # busy) and below what the SMs' paths to L2 could carry (128 bytes per SM
    # per clock)
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    upper = sms * 128 * MAX_SM_MHZ * 1e6 / 1e9
    bw = dg.measure_l2_reduce_bw(0)
    assert 1000.0 < bw <= upper, (bw, upper)
    with pytest.raises(dg.DegridError):
        dg.measure_l2_reduce_bw(-1)
