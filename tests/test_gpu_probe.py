"""The FMA throughput probe returns rates in the range this class of GPU can reach."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_rates_are_plausible():
    import paper_2402_08296_b300 as ddg
    r = ddg.ddg_probe_fma_peaks(0)
    # B300: 148 SMs x 128 FP32 lanes x 2 FLOP x up to 2,032 MHz = 77.0 TFLOP/s; FP64 at about 1/64 of it
    assert 20.0 < r["fp32_tflops"] < 90.0, r
    assert 0.2 < r["fp64_tflops"] < 5.0, r
    assert r["fp32_tflops"] > 8.0 * r["fp64_tflops"], r
