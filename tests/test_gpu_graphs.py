"""Rollouts and backward passes replayed from cached CUDA graphs: results
equal direct launches (the same kernels), a new set of genes invalidates the
captured graphs, and other buffers get their own capture.  GPU only."""
import numpy as np
import pytest

from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import to_dev, torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    torch_mod()


def _world():
    w = inputs.global_multi_channel(H=64, W=64, R=9, patch=24)
    for i, k in enumerate(w.kernels):
        k.mu = float(0.1 + 0.01 * i)
        k.sigma = float(0.05 + 0.003 * i)
    return w


def _genes(w, scale=1.0):
    return np.array([[k.mu * scale, k.sigma, k.h] for k in w.kernels], np.float32)


def _steps(ctx, A, n):
    torch = torch_mod()
    for _ in range(n):
        B = torch.empty_like(A)
        lenia.lenia_step(ctx, A, None, B, None)
        A = B
    return A


def test_rollout_graph_equals_steps_and_follows_new_genes():
    torch = torch_mod()
    w = _world()
    cfg, ks = lenia.config_from_world(w)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A0 = to_dev(w.A)
        a = A0.clone()
        lenia.lenia_rollout(ctx, a, None, 6)          # captured, then replayed
        lenia.lenia_rollout(ctx, a, None, 7)          # replayed, odd tail direct
        ref = _steps(ctx, A0.clone(), 13)
        old8 = _steps(ctx, A0.clone(), 8)
        torch.cuda.synchronize()
        assert torch.equal(a, ref)
        # other genes: the cached graph must not be reused
        lenia.lenia_set_genes(ctx, _genes(w, 1.1))
        b = A0.clone()
        lenia.lenia_rollout(ctx, b, None, 8)
        ref2 = _steps(ctx, A0.clone(), 8)
        torch.cuda.synchronize()
        assert torch.equal(b, ref2)
        assert not torch.equal(b, old8)
        # another buffer: its own capture
        c = A0.clone()
        lenia.lenia_rollout(ctx, c, None, 8)
        torch.cuda.synchronize()
        assert torch.equal(c, b)
    finally:
        lenia.lenia_destroy(ctx)


def test_backward_graph_tracks_genes_and_fresh_tensors():
    torch = torch_mod()
    w = _world()
    n = 6
    cfg, ks = lenia.config_from_world(w, max_rollout_steps=n, ckpt_every=2)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A0 = to_dev(w.A)
        out = []
        for rep in range(3):                          # fresh gradient tensors every call
            gT = torch.ones_like(A0)
            gA0 = torch.empty_like(A0)
            gg = torch.empty((w.n_kernels, 3), dtype=torch.float32, device="cuda")
            lenia.lenia_backward(ctx, A0, None, n, gT, gA0, gg)
            out.append((gA0, gg))
        torch.cuda.synchronize()
        for gA0, gg in out[1:]:
            assert torch.equal(gA0, out[0][0]) and torch.equal(gg, out[0][1])
        # new genes: the result must equal a context made with them
        g2 = _genes(w, 1.1)
        lenia.lenia_set_genes(ctx, g2)
        gA0 = torch.empty_like(A0)
        gg = torch.empty((w.n_kernels, 3), dtype=torch.float32, device="cuda")
        lenia.lenia_backward(ctx, A0, None, n, torch.ones_like(A0), gA0, gg)
        for k, kd in enumerate(w.kernels):
            kd.mu = float(g2[k, 0])
        cfg2, ks2 = lenia.config_from_world(w, max_rollout_steps=n, ckpt_every=2)
        ctx2 = lenia.lenia_init(cfg2, ks2)
        try:
            gA0b = torch.empty_like(A0)
            ggb = torch.empty((w.n_kernels, 3), dtype=torch.float32, device="cuda")
            lenia.lenia_backward(ctx2, A0, None, n, torch.ones_like(A0), gA0b, ggb)
            torch.cuda.synchronize()
            assert torch.equal(gA0, gA0b) and torch.equal(gg, ggb)
            assert not torch.equal(gg, out[0][1])
        finally:
            lenia.lenia_destroy(ctx2)
    finally:
        lenia.lenia_destroy(ctx)
