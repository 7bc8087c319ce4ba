"""Direct convolution on the tensor cores (LENIA_CONV_DIRECT_BF16 and
_BF16X3: banded Toeplitz products with tcgen05, FP32 accumulation) against
the FP64 oracle.  GPU only.

Error bounds, from the arithmetic: every potential is a sum of non-negative
products K~(d) A(x + d) with sum K~ = 1.  BF16 keeps 8 significant bits, so
rounding one operand moves it by at most 2^-8 relative; both operands
rounded (their product is exact in FP32) move a potential by at most
(2^-7 + 2^-16) U.  With the high/low split x = x_hi + x_lo + e, |e| <= 2^-16
|x|, and the dropped lo x lo product (<= 2^-16), the bound is about
3 2^-16 U (4.6e-5 U), plus FP32 accumulation rounding."""
import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import TOL_STEP, alpha_margin, compare_step, gpu_potentials, gpu_step, torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


def w_c3():
    # 15 kernels of radius 18, five per channel (blocks of four and one)
    return inputs.multi_channel(H=256, W=256, R=18, patch=96, n_geno=3, matched=True, name="c3tc")


def w_c2():
    return inputs.localized_single_channel(H=256, W=512, R=12, patch=64, n_geno=4, live=True, name="c2tc")


def w_narrow():
    # three 32-column tiles, small radius
    return inputs.multi_channel(H=256, W=96, R=5, patch=40, n_geno=2, matched=True, name="narrow")


def w_rings():
    # 3 x 24 ring planes, some of them empty (no lattice point)
    w = inputs.ring_world(H=256, W=256, R=12, n_rings=24, patch=64, n_geno=3, seed_index=9)
    w.alpha_on = 1
    return w


WORLDS = {"c3tc": w_c3, "c2tc": w_c2, "narrow": w_narrow, "rings": w_rings}


def _ref_potentials(w):
    if w.n_rings:
        V = np.stack([oracle.ring_potentials(w.A[c], w.kernels[0].radius, w.n_rings) for c in range(w.n_channels)])
        return V.reshape(-1, w.height, w.width)
    return oracle.step(w, return_u=True)[2]


def _gpu_planes(w, path):
    if not w.n_rings:
        return gpu_potentials(w, path)
    torch = torch_mod()
    cfg, ks = lenia.config_from_world(w, path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A = torch.from_numpy(w.A).cuda()
        V = torch.empty((w.n_channels * w.n_rings, w.height, w.width), dtype=torch.float32, device="cuda")
        lenia.lenia_potentials(ctx, A, V)
        torch.cuda.synchronize()
        return V.cpu().numpy(), lenia.lenia_conv_path(ctx)
    finally:
        lenia.lenia_destroy(ctx)


@pytest.mark.parametrize("name", ["c3tc", "c2tc", "narrow", "rings"])
@pytest.mark.parametrize("path", [lenia.CONV_DIRECT_BF16, lenia.CONV_DIRECT_BF16X3])
def test_tc_potentials_within_bound(name, path):
    w = WORLDS[name]()
    U, used = _gpu_planes(w, path)
    assert used == path
    ref = _ref_potentials(w)
    err = np.abs(U - ref)
    rel = 2.0 ** -7 + 2.0 ** -16 if path == lenia.CONV_DIRECT_BF16 else 3 * 2.0 ** -16 + 2.0 ** -23
    bound = rel * np.abs(ref) + 2e-6
    print(f"{name} path={path}: max|dU| {err.max():.3e}, rms {np.sqrt((err ** 2).mean()):.3e}, "
          f"max |dU| / bound {(err / bound).max():.3f}")
    assert np.all(err <= bound)


def _step_against_oracle(w, path, band):
    """One step on a tensor-core route against the oracle's FP64 step: alpha
    may differ only where the oracle's decision lies within `band` of its
    threshold (the potential error moves the growth test by up to h |g'| |dU|);
    everywhere else the phenospace and the genes are compared."""
    A1, P1, U, al = oracle.step(w, return_u=True, return_alpha=True)
    Ph = np.stack([[oracle.diffuse(w.P[p, k]) for k in range(w.n_kernels)] for p in range(w.n_planes)])
    margin = alpha_margin(w, U, Ph)
    g = gpu_step(w, path)
    H, W = w.height, w.width
    g_alpha = (g["P"].reshape(-1, H, W) != 0).all(axis=0)
    flips = g_alpha != al.astype(bool)
    keep = ~flips
    dA = np.abs(g["A"] - A1)
    dP = np.abs(g["P"].reshape(-1, H, W) - P1.reshape(-1, H, W))
    res = {"alpha1": int(al.sum()), "flips": int(flips.sum()), "flips_outside_band": int((flips & (margin >= band)).sum()),
           "max_dA": float(dA[:, keep].max()), "max_dA_all": float(dA.max()), "max_dP": float(dP[:, keep].max())}
    return res


@pytest.mark.parametrize("name", ["c3tc", "c2tc", "narrow"])
def test_tc_split_step_within_gate(name):
    """The high/low split route: one whole step within 1e-3 of the oracle (the
    gate for the BF16 routes) at every site whose alpha decision agrees; a
    decision may flip only within 2e-4 of its threshold (potential errors up
    to ~4e-6 times |g'| <= 1.2 / sigma with sigma >= 0.03 here)."""
    w = WORLDS[name]()
    res = _step_against_oracle(w, lenia.CONV_DIRECT_BF16X3, 2e-4)
    print(name, "bf16x3", res)
    assert res["alpha1"] > 0 and res["flips_outside_band"] == 0
    assert res["flips"] <= max(2, w.sites // 1000)
    assert res["max_dA"] <= 1e-3 and res["max_dP"] <= 4e-7


@pytest.mark.parametrize("name", ["c3tc", "c2tc", "narrow"])
def test_tc_bf16_step_error_reported(name):
    """The plain BF16 route: the per-step error against the oracle, with the
    sites whose alpha decision differs counted (a potential error of ~1e-4
    may flip decisions near their thresholds).  It is held only where this
    error stays below 1e-3; the test bounds what the arithmetic allows."""
    w = WORLDS[name]()
    res = _step_against_oracle(w, lenia.CONV_DIRECT_BF16, 1.0)
    print(name, "bf16", res)
    assert res["alpha1"] > 0 and res["max_dA"] < 5e-2
