"""The instruction-rate microbenchmark behind the filter rooflines, on the GPU:
every rate is positive and below what the SM can issue, and the mixed tap loop
of the paired form does not beat the bound computed from its parts."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_01210_gb300 import alu_peaks, build
    build.build()
    r = alu_peaks.measure(0, warm_s=0.2)
    per = r["rate_per_sm_clk"]
    for k, v in per.items():
        assert v > 0, k
    # one FMA a lane per clock at most, 4 schedulers x 32 lanes (5 % for clock sampling noise)
    assert per["ffma"] <= 128 * 1.05 and per["ffma2"] <= 128 * 1.05
    assert per["ffma"] >= 32                          # issue-bound, not latency-bound
    mixed = per["tap_paired"]
    bound = r["tap_peaks"]["fp32_expanded_pairs"]["taps_per_sm_clk"]
    assert mixed <= bound * 1.05
