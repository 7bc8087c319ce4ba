"""lenia_stats_noalloc: the statistics reduction for callers that cannot
allocate device memory (for example code whose GPU memory is all reserved
by another framework's allocator, or code that must avoid the device-wide
synchronisation of cudaMalloc/cudaFree).  Its scratch is a static device
array inside the library.  Its output is compared with lenia_stats (the
context path) and with the FP64 oracle's statistics, on two calls in a row.
This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia

pytestmark = pytest.mark.gpu


def _circ(d, n):
    d = np.abs(d)
    return np.minimum(d, n - d)


def _check(got, ref, H, W, rtol=2e-6):
    # same tolerances as the other stats parity tests (FP32 outputs of FP64 sums)
    assert np.allclose(got[:, 0], ref[:, 0], rtol=rtol, atol=1e-4), (got, ref)
    assert _circ(got[:, 1] - ref[:, 1], H).max() <= 1e-3, (got, ref)
    assert _circ(got[:, 2] - ref[:, 2], W).max() <= 1e-3, (got, ref)


def _noalloc_twice(torch, A, C, H, W):
    outs = []
    for _ in range(2):                      # two calls in a row share the scratch
        out = torch.full((C, 3), -1.0, device="cuda")
        lenia.lenia_stats_noalloc(A, C, H, W, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().astype(np.float64))
    return outs


def test_stats_noalloc_matches_lenia_stats_and_oracle():
    import torch
    assert torch.cuda.is_available()
    build.build()
    oracle.build()
    worlds = [inputs.multi_channel(H=128, W=256, R=9, patch=40, n_geno=4, live=True),
              inputs.localized_single_channel(H=96, W=160, R=6, patch=32, n_geno=3),
              # ragged: neither side a multiple of the 32 x 32 block
              inputs.multi_channel(H=100, W=76, R=5, patch=24, n_geno=2, n_channels=2, live=True)]
    for w in worlds:
        cfg, ks = lenia.config_from_world(w, lenia.CONV_DIRECT)
        ctx = lenia.lenia_init(cfg, ks)
        try:
            A = torch.from_numpy(w.A).cuda()
            ref = torch.zeros((w.n_channels, 3), device="cuda")
            lenia.lenia_stats(ctx, A, ref)
            torch.cuda.synchronize()
            ref = ref.cpu().numpy().astype(np.float64)
            ora = oracle.stats(w.A)
            for got in _noalloc_twice(torch, A, w.n_channels, w.height, w.width):
                _check(got, ref, w.height, w.width)
                _check(got, ora, w.height, w.width)
        finally:
            lenia.lenia_destroy(ctx)


@pytest.mark.parametrize("C,H,W", [(3, 2048, 2048), (1, 8192, 8192)])
def test_stats_noalloc_large_worlds_match_oracle(C, H, W):
    """2048^2 x 3 (the headline world) and 8192^2 x 1, whose 65536 block
    records fill the static scratch exactly."""
    import torch
    build.build()
    oracle.build()
    A = np.zeros((C, H, W), np.float32)
    rng = inputs.Rng(4242 + C)
    for c in range(C):
        y0 = int(rng.integers(1, 0, H - 1)[0])
        x0 = int(rng.integers(1, 0, W - 1)[0])
        side = H // 4
        blob = rng.uniform(side * side).reshape(side, side)
        A[c] = np.roll(np.pad(blob, ((0, H - side), (0, W - side))), (y0, x0), axis=(0, 1))
    ora = oracle.stats(A)
    Ad = torch.from_numpy(A).cuda()
    for got in _noalloc_twice(torch, Ad, C, H, W):
        # masses up to ~1e6 summed in FP64 and rounded to FP32
        _check(got, ora, H, W, rtol=1e-6)


def test_stats_noalloc_rejects_oversize():
    import torch
    build.build()
    A = torch.zeros(8, device="cuda")
    out = torch.zeros(3, device="cuda")
    with pytest.raises(lenia.LeniaError) as e:
        lenia.lenia_stats_noalloc(A, 1, 16384, 64, out)
    assert e.value.status == lenia.LENIA_EINVAL
    with pytest.raises(lenia.LeniaError) as e:
        lenia.lenia_stats_noalloc(A, 2, 8192, 8192, out)         # 131072 records
    assert e.value.status == lenia.LENIA_EINVAL
