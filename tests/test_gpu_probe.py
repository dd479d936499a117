"""The pipe-rate probe behind the roofline denominators (needs a GB300): every
rate is measured and positive, fma.rn.f32 issues at most one instruction per
lane per clock (4 x 32 lanes per SM), and the transcendental unit is slower
than the FMA pipe."""
import pytest

from paper_2002_02481_gb300 import build, lv

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lib = lv.load()
    peaks = lv.measure_pipe_peaks(lib)
    assert set(peaks) == set(lv.PIPES)
    assert all(v > 0 for v in peaks.values()), peaks
    props = torch.cuda.get_device_properties(0)
    max_mhz = 2070.0
    issue_cap = props.multi_processor_count * 128 * max_mhz * 1e6
    assert 0.5 * issue_cap <= peaks["ffma"] <= 1.05 * issue_cap, (peaks["ffma"], issue_cap)
    for k in ("mufu_ex2", "mufu_lg2", "mufu_sin", "mufu_cos", "mufu_sqrt"):
        assert peaks[k] < peaks["ffma"], (k, peaks[k], peaks["ffma"])
    for k in ("imad", "imad_wide", "lop3"):
        assert peaks[k] <= 1.05 * issue_cap, (k, peaks[k])
