"""Pins for the oracle's ring decomposition of localized kernels (Section 2.4):
the kernel of kernel k at a site is sum_r k_r K_r, rings K_r of a radius-R
disk cut into n_ring rings, weights k_r = sum_i k(r / n_ring; r_i, w_i, b_i)
from the site's kernel genes, and U = sum_r k_r (K_r * A) / sum_r k_r (K_r * 1).
CPU only.

The checks rest on integer geometry (an isqrt formulation of the ring index,
lattice-point counts), numpy and scipy periodic sums, closed forms (a uniform
field, an impulse's ring-to-ring ratio) and the paper's own identity between
the recombined ring convolutions and one convolution with the recombined
kernel."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import inputs

ndimage = pytest.importorskip("scipy.ndimage")

KGENES = ("r1", "w1", "b1", "r2", "w2", "b2")


def _ring_index(dy, dx, R, n):
    """Ring of an offset: floor(n |d| / R) = isqrt(n^2 |d|^2) // R for |d| < R."""
    q = dy * dy + dx * dx
    if q >= R * R:
        return -1
    return math.isqrt(n * n * q) // R


def _ring_offsets(R, n):
    rings = [[] for _ in range(n)]
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            r = _ring_index(dy, dx, R, n)
            if r >= 0:
                rings[r].append((dy, dx))
    return rings


def _uniform_gene_world(H=40, W=48, R=6, n=12, C=1, genes=None, seed=3):
    """A world whose genes are the same at every site (so the kernel is the
    same everywhere), with random A."""
    genes = genes or dict(mu=0.25, sigma=0.05, h=0.8, r1=0.3, w1=0.12, b1=0.9, r2=0.7, w2=0.1, b2=0.4)
    topo = inputs.paper_topology(C) if C > 1 else [(0, 0)]
    K = len(topo)
    kernels = [inputs.KernelDesc(s, d, R, inputs.KERNEL_BUMPS, (1.0,),
                                 bump=tuple(genes[g] for g in KGENES), h=genes["h"], mu=genes["mu"],
                                 sigma=genes["sigma"]) for (s, d) in topo]
    loc = inputs.LOC_MU | inputs.LOC_SIGMA | inputs.LOC_H | inputs.LOC_KERNEL
    order = ["mu", "sigma", "h"] + list(KGENES)
    P = np.zeros((9, K, H, W), np.float32)
    for p, g in enumerate(order):
        P[p] = genes[g]
    A = inputs.random_field(seed, (C, H, W))
    return inputs.World(H, W, C, kernels, 0.1, localized=loc, maintain_genes=1, A=A, P=P, n_rings=n)


@pytest.mark.parametrize("R,n", [(12, 24), (5, 7), (9, 9), (18, 36), (6, 12)])
def test_rings_partition_the_open_disk(R, n):
    """Section 2.4: the rings dissemble the kernel's disk; every lattice point
    with |d| < R lies in exactly one ring, and ring r holds the points with
    r <= n |d| / R < r + 1."""
    cnt = oracle.ring_counts(R, n)
    ref = [len(o) for o in _ring_offsets(R, n)]
    np.testing.assert_array_equal(cnt, ref)
    inside = sum(1 for dy in range(-R, R + 1) for dx in range(-R, R + 1) if dy * dy + dx * dx < R * R)
    assert cnt.sum() == inside


def test_ring_point_counts_closed_form():
    """R = 12 in 24 rings (the paper's setting): 437 points with |d| < 12 (441
    lattice points with |d| <= 12 minus the 4 on the circle); rings of width
    1/2 pixel with no lattice point are empty, e.g. 1/2 <= |d| < 1."""
    cnt = oracle.ring_counts(12, 24)
    assert cnt.sum() == 441 - 4
    assert cnt[0] == 1 and cnt[1] == 0 and cnt[2] == 4 + 4 and cnt[3] == 0    # |d| = 1 (4) and sqrt(2) (4)


@pytest.mark.parametrize("R,n", [(5, 10), (4, 3)])
def test_ring_potentials_match_numpy_roll_sums(R, n):
    """K_r * A on the torus equals a sum of periodic shifts over the ring's offsets."""
    A = inputs.random_field(11, (20, 24)).astype(np.float64)
    V = oracle.ring_potentials(A, R, n)
    for r, offs in enumerate(_ring_offsets(R, n)):
        ref = np.zeros_like(A)
        for (dy, dx) in offs:
            ref += np.roll(np.roll(A, dy, 0), dx, 1)        # A(y - dy, x - dx)
        np.testing.assert_allclose(V[r], ref, rtol=0, atol=1e-12)


def test_uniform_field_gives_its_value():
    """A uniform field a gives U = a for any positive kernel genes (the
    normalisation by sum_r k_r (K_r * 1))."""
    w = inputs.ring_world(H=48, W=64, R=6, n_rings=12, patch=20, n_geno=3)
    a = np.array([0.3, 0.55, 0.8])
    w.A = np.broadcast_to(a[:, None, None], w.A.shape).astype(np.float32).copy()
    w.P[:] = np.where(w.P > 0, w.P, 0.5)            # positive genes everywhere
    _, _, U = oracle.ring_step(w, return_u=True)
    for k, kd in enumerate(w.kernels):
        np.testing.assert_allclose(U[k], np.float32(a[kd.src]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("R,n", [(6, 12), (7, 5)])
def test_recombined_rings_equal_one_convolution_with_the_recombined_kernel(R, n):
    """Section 2.4's identity: sum_r k_r (K_r * A) / sum_r k_r (K_r * 1) =
    ((sum_r k_r K_r) * A) / ((sum_r k_r K_r) * 1), here with the right side as
    one scipy periodic correlation with the piecewise-constant kernel."""
    g = dict(mu=0.25, sigma=0.05, h=0.8, r1=0.3, w1=0.12, b1=0.9, r2=0.7, w2=0.1, b2=0.4)
    w = _uniform_gene_world(R=R, n=n, genes=g)
    _, _, U = oracle.ring_step(w, return_u=True)
    g = {k: float(np.float32(v)) for k, v in g.items()}     # the genes as stored (FP32)
    kfun = lambda x, r, s, b: b * math.exp(-(x - r) ** 2 / (2 * s * s))
    Kpw = np.zeros((2 * R + 1, 2 * R + 1))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            r = _ring_index(dy, dx, R, n)
            if r >= 0:
                x = r / n
                Kpw[dy + R, dx + R] = kfun(x, g["r1"], g["w1"], g["b1"]) + kfun(x, g["r2"], g["w2"], g["b2"])
    ref = ndimage.correlate(w.A[0].astype(np.float64), Kpw[::-1, ::-1] / Kpw.sum(), mode="wrap")
    np.testing.assert_allclose(U[0], ref, rtol=0, atol=1e-13)


def test_impulse_ring_ratio_is_the_gaussian_kernel_function():
    """An impulse puts 1 in one ring per site, so U at sites in rings r and
    r + 1 differ by k_r / k_{r+1}; with one bump centred on ring r (r_1 = r / n)
    and width w_1 = 1 / n that ratio is exp(1/2), two rings out exp(2)."""
    R, n, r0 = 8, 8, 4          # r0 / n = 1/2 and 1 / n = 1/8 are exact in FP32
    g = dict(mu=0.25, sigma=0.05, h=0.8, r1=r0 / n, w1=1.0 / n, b1=0.9, r2=0.5, w2=0.1, b2=0.0)
    w = _uniform_gene_world(H=32, W=32, R=R, n=n, genes=g)
    w.A[:] = 0.0
    w.A[0, 16, 16] = 1.0
    _, _, U = oracle.ring_step(w, return_u=True)
    # sites at distance 4, 5, 6 from the impulse along x: rings 4, 5, 6
    u4, u5, u6 = U[0, 16, 20], U[0, 16, 21], U[0, 16, 22]
    assert abs(u4 / u5 - math.exp(0.5)) < 1e-12
    assert abs(u4 / u6 - math.exp(2.0)) < 1e-12


def test_flat_kernel_function_gives_the_disk_average():
    """b_2 = 0 and a very wide first bump make every ring weight equal: U is
    the plain average over the open disk |d| < R.  (Without gene maintenance,
    whose diffusion would clip the width to 1.)"""
    R = 5
    g = dict(mu=0.25, sigma=0.05, h=0.8, r1=0.5, w1=1e6, b1=0.7, r2=0.5, w2=0.1, b2=0.0)
    w = _uniform_gene_world(R=R, n=10, genes=g)
    w.maintain_genes = 0
    _, _, U = oracle.ring_step(w, return_u=True)
    d = np.arange(-R, R + 1)
    D = (d[:, None] ** 2 + d[None, :] ** 2 < R * R).astype(np.float64)
    ref = ndimage.correlate(w.A[0].astype(np.float64), D / D.sum(), mode="wrap")
    np.testing.assert_allclose(U[0], ref, rtol=0, atol=1e-12)


def test_kernel_genes_join_the_alpha_mask():
    """Section 2.2: alpha needs every gene plane, the kernel genes included,
    above eps_p; a site whose diffused b_1 is 0 loses alpha and all its genes."""
    w = _uniform_gene_world(H=32, W=40, R=4, n=8)
    w.alpha_on = 1
    w.eps_u = 1e-3
    b1 = 5                                            # plane index of b1 (m, s, h, r1, w1, b1, ...)
    w.P[b1, 0, 10:13, 10:13] = 0.0                    # centre (11, 11) and its 5-point disk stay 0
    A1, P1, al = oracle.ring_step(w, return_alpha=True)
    assert al[11, 11] == 0 and np.all(P1[:, 0, 11, 11] == 0)
    assert al[25, 30] == 1 and np.all(P1[:, 0, 25, 30] > 0)


def test_ring_approximation_of_the_cast_kernel_improves_with_rings():
    """Section 2.4 calls the rings a good approximation of the cast kernel at
    low resolution and reports calibration against it: the potential from
    global bump kernels cast on the grid and the ring-wise potential differ
    less as n_ring grows (the ring weight is the kernel function at the ring's
    inner radius)."""
    R = 12
    g = dict(mu=0.25, sigma=0.05, h=0.8, r1=0.3, w1=0.12, b1=0.9, r2=0.7, w2=0.1, b2=0.4)
    errs = []
    for n in (6, 12, 24, 96):
        w = _uniform_gene_world(H=64, W=64, R=R, n=n, genes=g, seed=5)
        w.A[0] = ndimage.uniform_filter(w.A[0], 5, mode="wrap")      # a smooth field
        _, _, U = oracle.ring_step(w, return_u=True)
        Kc = oracle.kernel(R, inputs.KERNEL_BUMPS, bump=tuple(g[x] for x in KGENES))
        Uc = oracle.potential(w.A[0], Kc)
        errs.append(float(np.max(np.abs(U[0] - Uc))))
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[2] < 0.1 * float(np.max(np.abs(U[0] - U[0].mean()))) + 1e-3, errs


def test_evolution_step_on_a_ring_world_reduces_to_the_ring_step():
    """With gamma = 0 and no walls the evolution step of a ring world is its
    plain ring step."""
    w = inputs.ring_world(H=48, W=64, R=6, n_rings=12, patch=20, n_geno=3)
    w.alpha_on = 1
    ev = inputs.evolution_events(w, 0, gamma_mut=0.0, gamma_pen=0.0)
    assert ev["mut_p"] < w.n_planes == 9
    A1, P1, al, _ = oracle.evolve_step(w, ev)
    A0, P0, al0 = oracle.ring_step(w, return_alpha=True)
    np.testing.assert_array_equal(A1, A0)
    np.testing.assert_array_equal(P1, P0)
    np.testing.assert_array_equal(al, al0)
