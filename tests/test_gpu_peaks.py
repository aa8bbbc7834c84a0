"""The measured FMA rates that serve as the roofline's denominators (fmm_measure_fma_rate): both
pipes report a positive rate no higher than the part's nominal one allows, and the FP32 pipe is
far faster than the FP64 pipe (nominally 64 times on this part); packed FP32 pairs (one
instruction per two FMAs) retire FMAs at least about as fast as single FP32 FMAs."""
import pytest

from paper_2101_08226_gb300 import _lib, api, build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f64, ms64 = api.measure_fma_rate(64, 2)
    f32, ms32 = api.measure_fma_rate(32, 2)
    # nominal: 2 FP64 and 128 FP32 FMAs per clock per SM, at most 2.1 GHz, 2 flops per FMA
    assert 0.0 < f64 <= 1.05 * sms * 2 * 2 * 2.1e9 / 1e12
    assert 0.0 < f32 <= 1.05 * sms * 128 * 2 * 2.1e9 / 1e12
    assert 20.0 < f32 / f64 < 100.0
    assert ms64 > 5.0 and ms32 > 5.0   # long enough launches that the launch overhead is noise
    f2, ms2 = api.measure_fma_rate(_lib.FMM_FMA_F32X2, 2)
    assert 0.9 * f32 < f2 <= 1.05 * sms * 256 * 2 * 2.1e9 / 1e12 and ms2 > 5.0


def test_fma_rate_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    for bits, reps in ((16, 1), (64, 0), (-64, 1)):
        with pytest.raises(_lib.FmmError) as e:
            api.measure_fma_rate(bits, reps)
        assert e.value.code == _lib.FMM_ERR_ARG
