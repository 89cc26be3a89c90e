"""The measured FMA peak that the benchmark's arithmetic rooflines divide by
(ffsat_alu_peak): positive, FP64 below FP32 on this part, argument errors
reported, and no device memory left allocated."""
import pytest

torch = pytest.importorskip("torch")

from paper_2308_15020_gb300 import ffsat  # noqa: E402

pytestmark = pytest.mark.gpu


def test_fp32_and_fp64_peaks_are_measured():
    tf32, ms32 = ffsat.alu_peak(ffsat.FFSAT_F32, target_ms=20.0)
    tf64, ms64 = ffsat.alu_peak(ffsat.FFSAT_F64, target_ms=20.0)
    # a GB300 runs 152 SMs x 128 FP32 lanes x 2 flops at up to 2.07 GHz = 80.5 TFLOP/s
    assert 5.0 < tf32 < 120.0
    assert 0.0 < tf64 < tf32
    assert ms32 > 5.0 and ms64 > 5.0


def test_peak_arguments_are_checked():
    with pytest.raises(ffsat.FFSatError) as e:
        ffsat.alu_peak(7)
    assert e.value.code == -1
    with pytest.raises(ffsat.FFSatError):
        ffsat.alu_peak(ffsat.FFSAT_F32, target_ms=0.0)


def test_peak_frees_its_buffer():
    torch.cuda.synchronize()
    ffsat.alu_peak(ffsat.FFSAT_F32, target_ms=5.0)
    free0, _ = torch.cuda.mem_get_info()
    ffsat.alu_peak(ffsat.FFSAT_F32, target_ms=5.0)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
