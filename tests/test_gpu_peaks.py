"""The measured ALU peaks (art_measure_alu_peaks) that sit beside the derived peak in the tracer's
roofline: FP32 fused multiply-add throughput at most the derived 152 SMs x 128 lanes x 2 flops at
the 2.07 GHz maximum clock (with 5 % for timer granularity) and at least half of it; FP64 between
a quarter and twice GB300's nominal 1.25 TFLOP/s, and far below FP32."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_alu_peaks():
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    try:
        m = ctx.art_measure_alu_peaks()
    finally:
        ctx.close()
    derived = 152 * 128 * 2 * 2.07e9 / 1e12
    print(m, "derived FP32", derived)
    assert 0.5 * derived <= m["fp32_tflops"] <= 1.05 * derived, m
    assert 0.25 * 1.25 <= m["fp64_tflops"] <= 2.0 * 1.25, m
    assert m["fp64_tflops"] < 0.1 * m["fp32_tflops"], m


def test_fp64_issue_cost():
    """The FP64 issue cost behind the tracer's FP64 kernel form: one warp issues FP64 at well under
    the SM's rate whatever its independent chains (so a ray's latency is its warp's FP64
    instruction count), and four warps reach the SM rate that the measured FP64 throughput
    implies (a warp instruction per 32 lanes / (throughput per SM and cycle))."""
    from paper_2103_07417_gb300 import art
    ctx = art.Context(0)
    try:
        c = ctx.art_measure_fp64_issue()
        m = ctx.art_measure_alu_peaks()
    finally:
        ctx.close()
    lanes_per_cycle = m["fp64_tflops"] * 1e12 / (2 * 152 * 2.07e9)
    sm_cycles = 32.0 / lanes_per_cycle
    print(c, "implied SM cycles per warp instruction", sm_cycles)
    assert c["one_warp_chain"] >= 4.0, c
    assert c["one_warp_8_chains"] > 2.0 * c["four_warps_per_sm"], c
    assert 0.6 * sm_cycles <= c["four_warps_per_sm"] <= 1.6 * sm_cycles, (c, sm_cycles)
