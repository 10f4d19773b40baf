"""Measured lane-arithmetic rates (qew_measure_alu_peaks): the denominators of the relaxation
kernels' rooflines.  The FP32 FMA rate must come out near its nominal value, SMs x 128 lanes x the
SM clock measured during the same run; the other two rates must lie in the ranges that their
instruction counts allow."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qew():
    import paper_1211_7275_gb300 as q
    q.load()
    return q


def test_rates_against_unit_counts(qew):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = qew.measure_alu_peaks()
    print(r)
    assert 500.0 <= r["sm_mhz"] <= 2300.0
    nominal = sms * 128 * r["sm_mhz"] * 1e6
    assert 0.8 * nominal <= r["fp32_fma_per_s"] <= 1.05 * nominal
    assert 0.0 < r["fp64_fma_per_s"] < r["fp32_fma_per_s"]
    # a Philox4x32-10 block is ten rounds of two wide multiplies and two three-way XORs
    assert r["fp32_fma_per_s"] / 200 <= r["philox_blocks_per_s"] <= r["fp32_fma_per_s"] / 20


def test_short_output_array_is_rejected(qew):
    from paper_1211_7275_gb300 import _capi
    lib = _capi.load()
    out = np.zeros(2)
    rc = lib.qew_measure_alu_peaks(out.ctypes.data_as(ctypes.c_void_p), 2)
    assert rc == -1
    assert b"4 values" in lib.qew_last_error(None)
