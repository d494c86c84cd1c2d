"""The measured ALU peaks that the roofline fractions divide by
(rt_measure_alu_peak): plausible for a GB300 (152 SMs, up to 2070 MHz; FP64
4 flop/clk/SM nominal, FP32 256 flop/clk/SM nominal) and stable between two
calls."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2309_08655_gb300 import rt  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2309_08655_gb300.build import build
    build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_measured_peaks_are_plausible_and_repeatable():
    a = rt.rt_measure_alu_peak(2000, 150000)
    b = rt.rt_measure_alu_peak(2000, 150000)
    props = torch.cuda.get_device_properties(0)
    nominal64 = props.multi_processor_count * 4 * 2.07e9
    nominal32 = props.multi_processor_count * 256 * 2.07e9
    for m in (a, b):
        assert 0.3 * nominal64 < m["fp64_flops"] < 1.3 * nominal64, m
        assert 0.3 * nominal32 < m["fp32_flops"] < 1.3 * nominal32, m
        assert m["fp64_ms"] > 1.0 and m["fp32_ms"] > 1.0
    assert abs(a["fp64_flops"] / b["fp64_flops"] - 1) < 0.2
    assert abs(a["fp32_flops"] / b["fp32_flops"] - 1) < 0.2
    with pytest.raises(rt.RtError):
        rt.rt_measure_alu_peak(0, 10)
