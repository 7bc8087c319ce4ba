"""Ring-wise localized kernel genes (Section 2.4) on the GPU, through the C
ABI, against the FP64 oracle: the ring potentials K_r * A_c, the epilogue
from identical ring potentials, whole steps on both convolution paths, the
evolution step on a ring world, and the paper's own configuration
(512 x 1024, 3 channels, 15 two-bump kernels, R = 12 in 24 rings, all nine
gene types localized) in full.  GPU only.

The ring potentials are unnormalised sums of up to ~50 values in [0, 1]:
FP32 FFTs carry ~1e-6 absolute error there (TOL_V); the recombined,
normalised potentials and the step then meet the usual per-step gates."""
import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import alpha_margin, compare_step, to_dev, torch_mod

pytestmark = pytest.mark.gpu

TOL_V = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


# Under the default alpha reading (alpha_on = 0) the genotypes are matched to
# their patches, so that every kernel's growth test passes in the interiors.
def w_small(alpha_on=1):
    w = inputs.ring_world(H=64, W=128, R=6, n_rings=12, patch=24 if alpha_on else 32, n_geno=3,
                          matched=not alpha_on)
    w.alpha_on = alpha_on
    return w


def w_single(alpha_on=1):
    w = inputs.ring_world(H=128, W=128, R=12, n_rings=24, n_channels=1, patch=40, n_geno=3, seed_index=7)
    w.alpha_on = alpha_on
    return w


def w_ragged(alpha_on=1):
    w = inputs.ring_world(H=72, W=100, R=5, n_rings=10, patch=24 if alpha_on else 32, n_geno=3, seed_index=8,
                          matched=not alpha_on)
    w.alpha_on = alpha_on
    return w


def w_coarse(alpha_on=1):
    # fewer rings than pixels of radius: wide rings
    w = inputs.ring_world(H=64, W=64, R=9, n_rings=4, patch=24 if alpha_on else 32, n_geno=2, seed_index=9,
                          matched=not alpha_on)
    w.alpha_on = alpha_on
    return w


WORLDS = {"small": w_small, "single": w_single, "ragged": w_ragged, "coarse": w_coarse}


def _diffused(world, P):
    out = np.zeros(P.shape, np.float64)
    for p in range(P.shape[0]):
        for k in range(P.shape[1]):
            out[p, k] = oracle.diffuse(P[p, k], world.r_diff, world.eps_p)
    return out


def _gpu(world, conv_path, what="step", V=None):
    torch = torch_mod()
    cfg, ks = lenia.config_from_world(world, conv_path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A = to_dev(world.A)
        P = to_dev(world.P)
        out = {"path": lenia.lenia_conv_path(ctx)}
        if what == "potentials":
            Vg = torch.empty((world.n_channels * world.n_rings, world.height, world.width), dtype=torch.float32,
                             device="cuda")
            lenia.lenia_potentials(ctx, A, Vg)
            torch.cuda.synchronize()
            out["V"] = Vg.cpu().numpy()
            return out
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        al = torch.zeros((world.height, world.width), dtype=torch.uint8, device="cuda")
        if what == "update":
            lenia.lenia_update_from_potentials(ctx, A, P, to_dev(V.astype(np.float32)), A2, P2, al)
        else:
            Vg = torch.empty((world.n_channels * world.n_rings, world.height, world.width), dtype=torch.float32,
                             device="cuda")
            lenia.lenia_potentials(ctx, A, Vg)
            lenia.lenia_update_from_potentials(ctx, A, P, Vg, A2, P2, al)
            A3, P3 = torch.empty_like(A), torch.empty_like(P)
            lenia.lenia_step(ctx, A, P, A3, P3)
            torch.cuda.synchronize()
            assert torch.equal(A2, A3) and torch.equal(P2, P3)     # the step = its two stages
        lenia.lenia_check(ctx)
        out.update(A=A2.cpu().numpy(), P=P2.cpu().numpy(), alpha=al.cpu().numpy())
        return out
    finally:
        lenia.lenia_destroy(ctx)


def _oracle_V(world):
    return np.stack([oracle.ring_potentials(world.A[c], world.kernels[0].radius, world.n_rings)
                     for c in range(world.n_channels)])


@pytest.mark.parametrize("name,path", [("small", 1), ("small", 2), ("single", 1), ("ragged", 2), ("coarse", 1),
                                       ("coarse", 2)])
def test_ring_potentials_parity(name, path):
    w = WORLDS[name]()
    g = _gpu(w, path, "potentials")
    ref = _oracle_V(w).reshape(-1, w.height, w.width)
    err = np.abs(g["V"] - ref).max()
    print(name, path, "max |dV|", err)
    assert err <= TOL_V


@pytest.mark.parametrize("name,alpha_on", [("small", 1), ("small", 0), ("single", 1), ("ragged", 0)])
def test_ring_epilogue_from_identical_potentials(name, alpha_on):
    """The per-site recombination, growth, alpha and update from the oracle's
    ring potentials rounded to FP32 (both sides read the same values)."""
    w = WORLDS[name](alpha_on)
    V32 = _oracle_V(w).astype(np.float32)
    g = _gpu(w, lenia.CONV_AUTO, "update", V=V32.reshape(-1, w.height, w.width))
    A1, P1, al = oracle.ring_update(w, w.A, w.P, V32.astype(np.float64), return_alpha=True)
    _, _, U = oracle.ring_step(w, return_u=True)
    margin = alpha_margin(w, U, _diffused(w, w.P))
    res = compare_step(w, g, A1, P1, al, margin, tol_a=2e-6)
    print(name, alpha_on, res)


@pytest.mark.parametrize("name,path,alpha_on", [("small", 1, 1), ("small", 2, 1), ("small", 1, 0),
                                                ("single", 1, 1), ("ragged", 2, 1), ("coarse", 1, 1)])
def test_ring_step_parity(name, path, alpha_on):
    w = WORLDS[name](alpha_on)
    g = _gpu(w, path)
    A1, P1, U, al = oracle.ring_step(w, return_u=True, return_alpha=True)
    margin = alpha_margin(w, U, _diffused(w, w.P))
    res = compare_step(w, g, A1, P1, al, margin)
    print(name, path, alpha_on, "path", g["path"], "alpha sites", int(al.sum()), res)
    if alpha_on:
        assert al.sum() > 0


def test_ring_evolution_step_matches_oracle():
    """Walls, mutation (of a kernel gene, b1) and penalisation on a ring world,
    compared as in the evolution tests (E_pen exact away from near-threshold
    Delta_sum decisions)."""
    from test_gpu_evolve import _compare
    torch = torch_mod()
    w = w_small()
    walls = inputs.wall_strip(w.height, w.width, 90, 4)
    ev = inputs.evolution_events(w, 2, gamma_mut=3.0, gamma_pen=0.5, mut_half=8, r_oxy=3, eps_pen=0.5)
    _, _, al, _ = oracle.evolve_step(w, ev, walls=walls)
    ys, xs = np.nonzero(al)
    ev["mut_y0"], ev["mut_x0"] = int(ys[len(ys) // 2]), int(xs[len(ys) // 2])
    ev["mut_p"] = 5                                   # b1, a kernel gene
    A1, P1, al, epen, tsum = oracle.evolve_step(w, ev, walls=walls, return_tsum=True)
    keep = (1 - walls).astype(np.float64)
    _, _, U = oracle.ring_step(w, A=w.A * keep, P=w.P * keep, return_u=True)
    margin = alpha_margin(w, U, _diffused(w, w.P * keep))
    cfg, ks = lenia.config_from_world(w)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        lenia.lenia_set_walls(ctx, walls)
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        ga = torch.zeros((w.height, w.width), dtype=torch.uint8, device="cuda")
        ge = torch.zeros((w.height, w.width), dtype=torch.float32, device="cuda")
        lenia.lenia_step_evolve(ctx, A, P, A2, P2, ev, None, ga, ge)
        lenia.lenia_check(ctx)
        g = {"A": A2.cpu().numpy(), "P": P2.cpu().numpy(), "alpha": ga.cpu().numpy(), "epen": ge.cpu().numpy()}
    finally:
        lenia.lenia_destroy(ctx)
    res = _compare(w, ev, walls, g, (A1, P1, al, epen, tsum, margin))
    print(res)
    s = ev["mut_half"]
    sq = np.zeros(al.shape, bool)
    sq[np.ix_(np.arange(ev["mut_y0"] - s, ev["mut_y0"] + s) % w.height,
              np.arange(ev["mut_x0"] - s, ev["mut_x0"] + s) % w.width)] = True
    assert (sq & al.astype(bool)).any()


def test_paper_configuration_full_step():
    """512 x 1024 torus, 3 channels, the 15-kernel topology, two-bump kernels of
    radius 12 cut into 24 rings, m, s, h and r1, w1, b1, r2, w2, b2 localized per
    kernel and site (Section 2.1, 2.4): one whole step against the oracle's."""
    w = inputs.ring_world()
    w.alpha_on = 1
    g = _gpu(w, lenia.CONV_AUTO)
    assert g["path"] == lenia.CONV_FFT
    A1, P1, U, al = oracle.ring_step(w, return_u=True, return_alpha=True)
    margin = alpha_margin(w, U, _diffused(w, w.P))
    res = compare_step(w, g, A1, P1, al, margin)
    print("paper configuration:", "alpha sites", int(al.sum()), res)
    assert al.sum() > 1000
