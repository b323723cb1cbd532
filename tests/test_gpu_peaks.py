"""The throughput probes behind the scoring kernel's roofline terms: each
measured peak is positive and no larger than what the device's unit counts
allow at its reported maximum clock (128 FP32 lanes per SM and cycle; 32 ex2
results per SM and cycle, twice the special-function rate of earlier parts,
as measured on GB300), and the L2 gather rate is far above what DRAM alone
could serve for random 16-byte loads."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_peaks_within_unit_limits():
    from paper_2007_03678_gb300 import adg
    ctx = adg.Context(0)
    p = adg.probe_peaks(ctx)
    ctx.close()
    ghz = p["sm_clock_mhz"] / 1e3
    fp32_nominal = p["sms"] * 128 * 2 * ghz / 1e3  # TFLOP/s
    mufu_nominal = p["sms"] * 32 * ghz  # G results/s
    print({k: round(v, 1) if isinstance(v, float) else v for k, v in p.items()})
    assert p["sms"] > 0 and p["sm_clock_mhz"] > 0
    assert p["fp32_tflops"] == max(p["fp32_scalar_tflops"], p["fp32x2_tflops"])
    # a probe can run a little above the reported clock's figure only through
    # timer granularity; 5 % is the margin
    assert 0.3 * fp32_nominal < p["fp32_tflops"] <= 1.05 * fp32_nominal
    assert 0.3 * mufu_nominal < p["mufu_gops"] <= 1.05 * mufu_nominal
    assert 0.15 * mufu_nominal < p["mufu_rsqrt_gops"] <= 1.05 * mufu_nominal
    assert p["l2_gather_gbs"] > 1000.0
    assert p["gather_bytes"] == 8 << 20
