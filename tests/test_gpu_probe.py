"""The roofline probe (rbf_probe_peaks): rates are positive, below what an SM can issue,
and ordered as the hardware orders them (float64 FMA far below float32 FMA)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    import paper_1305_5179_b300 as rbf
    r = rbf.probe_peaks(0)
    assert r["num_sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 < r["sm_mhz"] < 4000.0
    # an SM issues at most 4 warp instructions (128 lanes) per clock
    assert 4.0 <= r["ex2_per_clk_sm"] <= 128.0
    assert 32.0 <= r["ffma_per_clk_sm"] <= 128.5
    assert 32.0 <= r["ffma2_lanes_per_clk_sm"] <= 257.0
    assert 0.1 <= r["dfma_per_clk_sm"] <= r["ffma_per_clk_sm"] / 2
    assert 0.0 < r["mma_commit_cycles"] <= r["mma_commit4_cycles"]
