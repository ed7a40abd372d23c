"""The FMA throughput probe behind the arithmetic rooflines (lb_ch_alu_peak)."""
import pytest

from paper_1805_00007_gb300 import abi

pytestmark = pytest.mark.gpu


def test_alu_peak_is_plausible():
    """FP32: below the unit-count bound of 152 SMs x 128 lanes x 2 flop x 2.1 GHz (82 TFLOP/s) and above a
    quarter of it; FP64: a small fraction of FP32 on this part (nominally 1/64)."""
    f32 = abi.lb_ch_alu_peak(abi.LBCH_F32)
    f64 = abi.lb_ch_alu_peak(abi.LBCH_F64)
    assert 20e12 < f32 < 82e12
    assert 0.05e12 < f64 < 0.5 * f32


def test_alu_peak_rejects_other_precisions():
    with pytest.raises(abi.LbchError) as ei:
        abi.lb_ch_alu_peak(abi.LBCH_F16S)
    assert ei.value.status == abi.LBCH_EINVAL
