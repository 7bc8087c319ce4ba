"""Rollouts of small worlds with global genes on the direct route run as one
cooperative launch (every block keeps an 8 x 8 tile for the whole rollout and
meets the others at a bounded grid barrier after each step).  Against the FP64
oracle's rollout (the 1e-3 gate after 10 steps) and against repeated
lenia_step calls (FP32 rounding).  GPU only."""
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
}


@pytest.mark.parametrize("name", list(WORLDS))
@pytest.mark.parametrize("n", [2, 7, 10])
def test_small_rollout_matches_oracle_and_steps(name, n):
    torch = torch_mod()
    w = WORLDS[name]()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_DIRECT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
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
