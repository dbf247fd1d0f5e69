"""qram_measure_peaks: the measured roofline denominators.

The FP64 FMA rate of this part is about two lanes per clock per SM (148 SMs
at up to 2032 MHz: about 1.2 TFLOP/s), and 32-bit integer add/logic issue is
tens of Tops/s.  The test checks that the measurement lands in those ranges
and that two measurements agree, so a broken timer or a kernel the compiler
emptied cannot pass for a peak."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_plausible_and_repeatable():
    import paper_2609_34935_b300 as Q
    a = Q.measure_peaks(0)
    b = Q.measure_peaks(0)
    for p in (a, b):
        assert math.isfinite(p["fp64_flops"]) and math.isfinite(p["int32_ops"])
        assert 3e11 < p["fp64_flops"] < 5e12
        assert 5e12 < p["int32_ops"] < 1e14
    assert abs(a["fp64_flops"] / b["fp64_flops"] - 1.0) < 0.2
    assert abs(a["int32_ops"] / b["int32_ops"] - 1.0) < 0.2


def test_measure_peaks_rejects_null_outputs():
    import ctypes as C
    from paper_2609_34935_b300 import load_library
    L = load_library()
    x = C.c_double()
    assert L.qram_measure_peaks(0, None, C.byref(x)) != 0
    assert L.qram_measure_peaks(0, C.byref(x), None) != 0
