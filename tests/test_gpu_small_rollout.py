"""Rollouts of small worlds with global genes on the direct route run as one
cooperative launch (every block keeps an 8 x 8 tile for the whole rollout and
meets the others at a bounded grid barrier after each step), the smallest of
them in one thread-block cluster that keeps the world in shared memory.
Against the FP64 oracle's rollout (the 1e-3 gate after 10 steps) and against
repeated lenia_step calls (FP32 rounding).  GPU only."""
import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import to_dev, torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


def _live(w):
    # global genes near the noise level, so that the world stays alive for the
    # compared steps (random global genes let these worlds die within a step)
    for i, k in enumerate(w.kernels):
        k.mu = float(0.1 + 0.01 * i)
        k.sigma = float(0.05 + 0.003 * i)
    return w


WORLDS = {
    "c1": lambda: inputs.single_kernel_global(),                                    # 64^2, R = 13
    "c5s": lambda: _live(inputs.global_multi_channel(H=64, W=64, R=13, patch=24)),  # 3 channels, 15 kernels
    "rect": lambda: _live(inputs.global_multi_channel(H=32, W=120, R=7, patch=16)), # 15 x 4 tiles
    "max": lambda: inputs.single_kernel_global(H=128, W=128, R=18, patch=40),       # the largest size taken
    "q8": lambda: _live(inputs.single_kernel_global(H=40, W=64, R=9, patch=16)),    # a cluster of 8
    "r3": lambda: _live(inputs.single_kernel_global(H=64, W=96, R=3, patch=20)),    # a small radius
}

# the form lenia_rollout takes for each world (16-byte aligned A)
ROUTES = {"c1": lenia.ROUTE_CLUSTER, "c5s": lenia.ROUTE_CLUSTER, "rect": lenia.ROUTE_COOPERATIVE,
          "max": lenia.ROUTE_COOPERATIVE, "q8": lenia.ROUTE_CLUSTER, "r3": lenia.ROUTE_CLUSTER}


@pytest.mark.parametrize("name", list(WORLDS))
@pytest.mark.parametrize("n", [2, 7, 10])
def test_small_rollout_matches_oracle_and_steps(name, n):
    torch = torch_mod()
    w = WORLDS[name]()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_DIRECT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        assert lenia.lenia_rollout_route(ctx) == ROUTES[name]
        A = to_dev(w.A)
        lenia.lenia_rollout(ctx, A, None, n)
        lenia.lenia_check(ctx)
        got = A.cpu().numpy()
        # the same steps one launch sequence at a time
        B = to_dev(w.A)
        for _ in range(n):
            B2 = torch.empty_like(B)
            lenia.lenia_step(ctx, B, None, B2, None)
            B = B2
        torch.cuda.synchronize()
        steps = B.cpu().numpy()
    finally:
        lenia.lenia_destroy(ctx)
    ref, _, _ = oracle.rollout(w, n)
    err = np.abs(got - ref).max()
    d_steps = np.abs(got - steps).max()
    print(f"{name} n={n}: max|dA| vs oracle {err:.2e}, vs repeated steps {d_steps:.2e}")
    assert err <= 1e-3
    assert d_steps <= 1e-5 * n
    assert got.max() > 0                      # the compared state is not empty


def test_cluster_rollout_unaligned_state_takes_the_cooperative_launch():
    """A caller's A that is not 16-byte aligned runs the cooperative launch
    (scalar accesses); both forms give the same state to FP32 rounding."""
    torch = torch_mod()
    w = WORLDS["c1"]()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_DIRECT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A = to_dev(w.A)
        store = torch.zeros(w.A.size + 1, dtype=torch.float32, device="cuda")
        B = store[1:].view(w.A.shape)                 # 4 bytes past a 16-byte boundary
        B.copy_(A)
        lenia.lenia_rollout(ctx, A, None, 10)
        lenia.lenia_rollout(ctx, B, None, 10)
        lenia.lenia_check(ctx)
        d = float((A - B).abs().max())
    finally:
        lenia.lenia_destroy(ctx)
    print(f"cluster vs cooperative after 10 steps: {d:.2e}")
    assert d <= 1e-4
