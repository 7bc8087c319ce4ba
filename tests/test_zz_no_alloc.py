"""lenia_stats_noalloc: the statistics reduction for callers that cannot
allocate device memory (for example code whose GPU memory is all reserved
by another framework's allocator, or code that must avoid the device-wide
synchronisation of cudaMalloc/cudaFree).  Its scratch is a static device
array inside the library.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2304_05639_gb300 import build, inputs, lenia

pytestmark = pytest.mark.gpu


def _circ(d, n):
    d = np.abs(d)
    return np.minimum(d, n - d)


def _check(got, ref, H, W):
    # same tolerances as the other stats parity tests
    assert np.allclose(got[:, 0], ref[:, 0], rtol=2e-6, atol=1e-4)
    assert _circ(got[:, 1] - ref[:, 1], H).max() <= 1e-3
    assert _circ(got[:, 2] - ref[:, 2], W).max() <= 1e-3


def test_stats_noalloc_matches_lenia_stats():
    import torch
    assert torch.cuda.is_available()
    build.build()
    worlds = [inputs.multi_channel(H=128, W=256, R=9, patch=40, n_geno=4, live=True),
              inputs.localized_single_channel(H=96, W=160, R=6, patch=32, n_geno=3)]
    for w in worlds:
        cfg, ks = lenia.config_from_world(w, lenia.CONV_DIRECT)
        ctx = lenia.lenia_init(cfg, ks)
        try:
            A = torch.from_numpy(w.A).cuda()
            ref = torch.zeros((w.n_channels, 3), device="cuda")
            lenia.lenia_stats(ctx, A, ref)
            for _ in range(2):                      # two calls in a row share the scratch
                out = torch.full((w.n_channels, 3), -1.0, device="cuda")
                lenia.lenia_stats_noalloc(A, w.n_channels, w.height, w.width, out)
                torch.cuda.synchronize()
                _check(out.cpu().numpy(), ref.cpu().numpy(), w.height, w.width)
        finally:
            lenia.lenia_destroy(ctx)


def test_stats_noalloc_rejects_oversize():
    import torch
    build.build()
    A = torch.zeros(8, device="cuda")
    out = torch.zeros(3, device="cuda")
    with pytest.raises(lenia.LeniaError) as e:
        lenia.lenia_stats_noalloc(A, 1, 16384, 64, out)
    assert e.value.status == lenia.LENIA_EINVAL
    with pytest.raises(lenia.LeniaError) as e:
        lenia.lenia_stats_noalloc(A, 8, 8192, 8192, out)
    assert e.value.status == lenia.LENIA_EINVAL
