"""Host-side arithmetic of bench.py's report, checked by hand: the FFT flop
count behind the FP32 fraction, the FP32 line built from per-kernel times,
the algorithmic bytes of the headline workload, and the config object that
both arms print.  CPU only."""
import math

import bench


def test_fft_flop_count_by_hand():
    # one 64 x 64 channel, one kernel: rows 64 * 2.5 * 64 * 6, columns 33 * 5 * 64 * 6
    rows = 64 * 2.5 * 64 * 6
    cols = 33 * 5.0 * 64 * 6
    want = (rows + cols) + (33 * 64 * 2.0 + cols + rows)
    assert math.isclose(bench.fft_flops(64, 64, 1, 1), want, rel_tol=0, abs_tol=1e-6)
    # the headline workload: ~1005 flop per site-step
    per_site = bench.fft_flops(2048, 2048, 3, 15) / 2048 ** 2
    assert 1000 < per_site < 1010


def test_fp32_line_from_kernel_times():
    prof = {"rows_r2c": (0.35, 10), "cols_conv": (0.87, 10), "rows_c2r": (0.96, 10), "epilogue": (2.4, 10)}
    line = bench.fp32_line(prof, 2048, 2048, 77.0, 78.8)
    assert line["peak_tflops"] == 78.8
    assert math.isclose(line["fft_passes"]["ms"], 0.218, rel_tol=1e-9)
    want = bench.fft_flops(2048, 2048, 3, 15) / 0.218e-3 / 1e12
    assert math.isclose(line["fft_passes"]["achieved_tflops"], want, rel_tol=1e-9)
    assert math.isclose(line["fft_passes"]["frac"], want / 78.8, rel_tol=1e-9)


def test_algorithmic_bytes_and_shared_config():
    # A in and out (3 channels) and 30 gene planes in and out, FP32
    assert bench.ALG_BYTES_PER_SITE == 3 * 4 * 2 + 30 * 4 * 2 == 264
    a, b = bench.workload_config(1), bench.workload_config(1)
    assert a == b and "conv_path" not in a
    assert a["height"] == a["width"] == 2048 and a["channels"] == 3 and a["kernels"] == 15
    assert bench.workload_config(4)["worlds"] == 4 and bench.workload_config(4)["parallelism"] == "replicas"
