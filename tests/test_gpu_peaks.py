"""hom_alu_peak: the measured FMA rate the bench divides the kinetic passes'
FP32 work by.  Checked for plausibility against the GPU's own unit counts
(at most 128 FP32 lanes x 2 flops per SM per clock; FP64 far below FP32) and
for its argument checks."""

import pytest

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible_and_checked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import binding as H
    from paper_1903_02581_gb300 import build

    build.build()
    sink = torch.zeros(4, dtype=torch.float64, device="cuda")
    props = torch.cuda.get_device_properties(0)
    f32 = H.hom_alu_peak(0, sink.data_ptr())
    f64 = H.hom_alu_peak(1, sink.data_ptr())
    # 2.2 GHz bounds every clock this part runs at
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9
    assert 0.3 * ceiling < f32 <= ceiling, (f32, ceiling)
    assert 0.0 < f64 < 0.5 * f32, (f64, f32)
    assert float(sink.abs().sum()) == 0.0          # never written
    with pytest.raises(H.HomError):
        H.hom_alu_peak(2, sink.data_ptr())
    with pytest.raises(H.HomError):
        H.hom_alu_peak(0, 0)
