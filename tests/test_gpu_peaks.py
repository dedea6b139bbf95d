"""The library's peak-rate microbenchmark (skm_measure_peak), whose FP32 and
FP64 FMA rates are the roofs the benchmark reports the SIMT kernels against."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_04074_gb300 import skm  # noqa: E402


def test_measured_peaks_are_plausible():
    """skm_measure_peak's FP32 and FP64 FMA rates lie in the range a GB300
    can reach (152 SMs at up to ~2 GHz: FP32 below ~90 TFLOP/s; FP64 a small
    fraction of it), and an unknown kind is refused."""
    f32 = skm.measure_peak("fp32")
    f64 = skm.measure_peak("fp64")
    f32x2 = skm.measure_peak("fp32x2")  # packed pairs: at least the scalar rate's neighbourhood
    assert 20.0 < f32 < 120.0, f32
    assert 0.1 < f64 < f32, f64
    assert 0.8 * f32 < f32x2 < 250.0, (f32, f32x2)
    g = skm.measure_peak("l2_gather")  # TB/s of gathered bytes, L2-resident table
    assert 1.0 < g < 100.0, g
    import ctypes
    out = ctypes.c_double(0)
    assert skm.load().skm_measure_peak(7, ctypes.byref(out), None) == skm.EINVAL
