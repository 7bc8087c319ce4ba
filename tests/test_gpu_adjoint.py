"""Adjoint of the rollout (lenia_backward) against FP64 finite differences of
the oracle: per-kernel gene gradients (mu, sigma, h) and dL/dA0, for a
linear loss and for the centroid-displacement loss through the autograd
wrapper.  GPU only.

Finite differences: central, step 2e-8 on FP64 oracle rollouts (small enough
that no site crosses the clip at 0 or 1 between the two evaluations; FP64
rounding then contributes about 1e-6 of the gradient).  Tolerance:
the GPU runs in FP32, so each gradient vector must match within 2e-3 of its
largest entry."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import to_dev, torch_mod

pytestmark = pytest.mark.gpu

EPS = 2e-8
REL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


def _world(W=64, R=9, patch=24):
    w = inputs.global_multi_channel(H=64, W=W, R=R, patch=patch)
    # potentials near the growth peak keep the update away from the clip
    rng = inputs.Rng(5)
    A = np.zeros_like(w.A)
    y0, x0 = 32 - patch // 2, W // 2 - patch // 2
    for c in range(3):
        A[c, y0:y0 + patch, x0:x0 + patch] = rng.uniform(patch * patch, 0.1, 0.5).reshape(patch, patch)
    w.A = A
    for i, k in enumerate(w.kernels):
        k.mu = float(0.1 + 0.01 * i)
        k.sigma = float(0.05 + 0.003 * i)
    return w


def _oracle_final(world, n, A=None):
    A_T, _, _ = oracle.rollout(world, n, A=A)
    return A_T


def _fd_gene(world, n, loss, k, which):
    kd = world.kernels[k]
    v0 = getattr(kd, which)
    setattr(kd, which, v0 + EPS)
    lp = loss(_oracle_final(world, n))
    setattr(kd, which, v0 - EPS)
    lm = loss(_oracle_final(world, n))
    setattr(kd, which, v0)
    return (lp - lm) / (2 * EPS)


def _fd_site(world, n, loss, c, y, x):
    A = world.A.astype(np.float64)
    Ap, Am = A.copy(), A.copy()
    Ap[c, y, x] += EPS
    Am[c, y, x] -= EPS
    return (loss(_oracle_final(world, n, Ap)) - loss(_oracle_final(world, n, Am))) / (2 * EPS)


def _close(got, ref, name):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    scale = max(np.max(np.abs(ref)), 1e-9)
    err = np.max(np.abs(got - ref))
    print(f"{name}: max|grad| {scale:.4e}, max err {err:.3e} ({err / scale:.2e} relative)")
    assert err <= REL * scale, (name, got, ref)


@pytest.mark.parametrize("path,n,ckpt", [(1, 6, 4), (2, 6, 4), (1, 5, 8), (1, 6, 1), (2, 5, 1)])
def test_backward_linear_loss_matches_fd(path, n, ckpt):
    torch = torch_mod()
    w = _world()
    wts = inputs.random_field(21, w.A.shape, -1.0, 1.0).astype(np.float64)
    loss = lambda A: float(np.sum(wts * A))
    cfg, ks = lenia.config_from_world(w, path, max_rollout_steps=n, ckpt_every=ckpt)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A0 = to_dev(w.A)
        gA_T = to_dev(wts.astype(np.float32))
        gA0 = torch.empty_like(A0)
        gg = torch.empty((w.n_kernels, 3), dtype=torch.float32, device="cuda")
        lenia.lenia_backward(ctx, A0, None, n, gA_T, gA0, gg)
        lenia.lenia_check(ctx)
        gA0, gg = gA0.cpu().numpy(), gg.cpu().numpy()
    finally:
        lenia.lenia_destroy(ctx)
    ks_probe = [0, 4, 9, 14]
    for j, which in enumerate(("mu", "sigma", "h")):
        ref = [_fd_gene(w, n, loss, k, which) for k in ks_probe]
        _close(gg[ks_probe, j], ref, f"d/d{which}")
    sites = [(0, 30, 30), (1, 25, 38), (2, 36, 27), (0, 41, 22)]
    ref = [_fd_site(w, n, loss, *s) for s in sites]
    _close([gA0[s] for s in sites], ref, "dL/dA0")


def _centroid(A, torch=None):
    """Circular-mean centre (y, x) of channel 0 of A [C, H, W]."""
    H, W = A.shape[1:]
    if torch is None:
        ty = 2 * np.pi * np.arange(H) / H
        tx = 2 * np.pi * np.arange(W) / W
        a = A[0]
        cy = math.atan2(float((a.sum(1) * np.sin(ty)).sum()), float((a.sum(1) * np.cos(ty)).sum())) * H / (2 * np.pi)
        cx = math.atan2(float((a.sum(0) * np.sin(tx)).sum()), float((a.sum(0) * np.cos(tx)).sum())) * W / (2 * np.pi)
        return cy, cx
    ty = 2 * math.pi * torch.arange(H, device=A.device, dtype=A.dtype) / H
    tx = 2 * math.pi * torch.arange(W, device=A.device, dtype=A.dtype) / W
    a = A[0]
    cy = torch.atan2((a.sum(1) * torch.sin(ty)).sum(), (a.sum(1) * torch.cos(ty)).sum()) * H / (2 * math.pi)
    cx = torch.atan2((a.sum(0) * torch.sin(tx)).sum(), (a.sum(0) * torch.cos(tx)).sum()) * W / (2 * math.pi)
    return cy, cx


def test_autograd_centroid_loss_matches_fd():
    """Centroid-displacement loss |c(A_T) - (c(A_0) + (8, 0))|^2 through the
    torch.autograd wrapper; the loss itself is plain torch."""
    torch = torch_mod()
    w = _world(W=256, R=13, patch=40)
    n = 8
    cy0, cx0 = _centroid(w.A.astype(np.float64))
    target = (cy0 + 8.0, cx0)

    def loss_np(A):
        cy, cx = _centroid(A)
        return (cy - target[0]) ** 2 + (cx - target[1]) ** 2

    roll = lenia.LeniaRollout(w, n, ckpt_every=4)
    try:
        A0 = to_dev(w.A).requires_grad_(True)
        genes = torch.tensor(lenia.genes_of(w), device="cuda", requires_grad=True)
        A_T = roll(A0, genes)
        cy, cx = _centroid(A_T.double(), torch)
        L = (cy - target[0]) ** 2 + (cx - target[1]) ** 2
        L.backward()
        assert abs(float(L) - loss_np(_oracle_final(w, n))) < 1e-3 * max(1.0, float(L))
        gg = genes.grad.cpu().numpy()
        gA0 = A0.grad.cpu().numpy()
    finally:
        roll.close()
    ks_probe = [0, 7, 12]
    for j, which in enumerate(("mu", "sigma", "h")):
        ref = [_fd_gene(w, n, loss_np, k, which) for k in ks_probe]
        _close(gg[ks_probe, j], ref, f"centroid d/d{which}")
    sites = [(0, 32, 128), (0, 28, 140), (1, 34, 118)]
    ref = [_fd_site(w, n, loss_np, *s) for s in sites]
    _close([gA0[s] for s in sites], ref, "centroid dL/dA0")


def test_backward_rejects_unsupported():
    torch = torch_mod()
    w = _world()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)                  # no adjoint buffers
    try:
        A0 = to_dev(w.A)
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_backward(ctx, A0, None, 2, A0, None, None)
        assert e.value.status == lenia.LENIA_ENOTSUP
    finally:
        lenia.lenia_destroy(ctx)
    cfg, ks = lenia.config_from_world(w, 1, max_rollout_steps=4)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A0 = to_dev(w.A)
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_backward(ctx, A0, None, 5, A0, None, None)     # beyond max_rollout_steps
        assert e.value.status == lenia.LENIA_EINVAL
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_set_genes(ctx, np.zeros((w.n_kernels, 3)))     # sigma = 0
        assert e.value.status == lenia.LENIA_EINVAL
    finally:
        lenia.lenia_destroy(ctx)
    # gene maps: no adjoint buffers are made, backward is not supported
    wl = inputs.localized_single_channel(H=64, W=64, R=6, patch=16, n_geno=2)
    cfg, ks = lenia.config_from_world(wl, 1, max_rollout_steps=4)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A0 = to_dev(wl.A)
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_backward(ctx, A0, None, 2, A0, None, None)
        assert e.value.status == lenia.LENIA_ENOTSUP
    finally:
        lenia.lenia_destroy(ctx)


def test_set_genes_changes_the_step():
    """lenia_set_genes replaces mu/sigma/h: the step then matches the oracle
    with the new genes."""
    torch = torch_mod()
    w = _world()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        for k in w.kernels:
            k.mu, k.sigma, k.h = k.mu + 0.05, k.sigma * 1.3, k.h * 0.7
        lenia.lenia_set_genes(ctx, lenia.genes_of(w))
        A = to_dev(w.A)
        A2 = torch.empty_like(A)
        lenia.lenia_step(ctx, A, None, A2, None)
        torch.cuda.synchronize()
        ref, _ = oracle.step(w)
        assert np.max(np.abs(A2.cpu().numpy() - ref)) <= 1e-5
    finally:
        lenia.lenia_destroy(ctx)
