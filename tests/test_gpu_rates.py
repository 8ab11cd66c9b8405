"""The instruction-rate probe behind the walk's roofline (gt_measure_fp32_rates): the
rates must be those of a working GPU and consistent with each other, and the flop count of
an rsqrt by the paper's rule (Sec. 4: add/multiply throughput over rsqrt throughput) must
lie in the range of the GPUs the paper names (4 to 8) or near it."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_rates_are_consistent():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_07279_gb300 import build
    build.build()
    from paper_1610_07279_gb300 import gothic as g
    g.load()
    r = g.gt_measure_fp32_rates(torch.cuda.current_stream().cuda_stream)
    props = torch.cuda.get_device_properties(0)
    lanes = props.multi_processor_count * 128
    for k in ("fma_per_s", "fma2_per_s", "add_per_s", "mul_per_s"):
        # at least a fifth of the lanes' rate at 1 GHz, at most the lanes' rate at 3 GHz
        assert 0.2 * lanes * 1e9 < r[k] < lanes * 3e9, (k, r[k])
    assert 0.5 < r["fma2_per_s"] / r["fma_per_s"] < 2.5
    assert r["peak_flops"] == pytest.approx(2 * max(r["fma_per_s"], r["fma2_per_s"]))
    assert 2.0 <= r["rsqrt_flops"] <= 32.0
    assert 0 < r["fp64_fma_per_s"] < r["fma_per_s"]
    assert g.gt_measure_fp32_peak(torch.cuda.current_stream().cuda_stream) == pytest.approx(2 * r["fma_per_s"], rel=0.2)
