"""The FP32 peak measurement behind the FFT passes' FP32 fraction: both forms
run, give a plausible figure for a 152-SM part (nominal 128 FP32 lanes per
SM at up to 2.07 GHz: ~80 TFLOP/s), and the entry point rejects null outputs.
GPU only."""
import ctypes

import pytest

from paper_2304_05639_gb300 import build, lenia
from gpu_util import torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    torch_mod()


def test_fp32_peak_is_plausible():
    scalar, pair = lenia.lenia_measure_fp32_peak()
    print("fp32 peak TFLOP/s: scalar", scalar, "packed pairs", pair)
    assert 10.0 < scalar < 400.0
    assert 10.0 < pair < 800.0


def test_fp32_peak_rejects_null_outputs():
    d = ctypes.c_double(0.0)
    assert lenia.load().lenia_measure_fp32_peak(None, ctypes.byref(d), None) == lenia.LENIA_EINVAL
