"""The library's throughput probes against the unit counts the roofline denominators are derived
from, at no more than the 2070 MHz maximum SM clock (a loaded clock can be lower, hence the lower
bounds): 128 FP32 FMA lanes and 16 lg2 results per SM per clock."""
import pytest

pytestmark = pytest.mark.gpu

SM_MAX_HZ = 2070e6


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2009_00767_gb300 import binding
    return binding


def test_probes_match_the_unit_counts(lib):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = lib.fmm_probe_peak(lib.FMM_PROBE_FP32_FMA)
    lg2 = lib.fmm_probe_peak(lib.FMM_PROBE_MUFU_LG2)
    f64 = lib.fmm_probe_peak(lib.FMM_PROBE_FP64_FMA)
    r32 = f32 / (sms * 128 * 2 * SM_MAX_HZ)
    rlg = lg2 / (sms * 16 * SM_MAX_HZ)
    assert 0.6 < r32 < 1.05, r32
    assert 0.6 < rlg < 1.05, rlg
    assert 0 < f64 < f32 / 8           # the FP64 pipe is a small fraction of the FP32 one on this part
