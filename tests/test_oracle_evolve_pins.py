"""Pins for the oracle's evolutionary operators: walls (Section 2.7), explosion
penalisation (Section 2.6) and mutation (Section 2.5), in the order of
Algorithm 2.  CPU only.

Each check rests on something other than the oracle's own formulas: lattice
point counts of the disk (Gauss's circle problem), scipy's periodic
correlation, masks built here with numpy, closed forms of the update, and
exact rational values of the two disk averages."""
import math

import numpy as np
import pytest

from paper_2304_05639_gb300 import inputs

ndimage = pytest.importorskip("scipy.ndimage")

# number of lattice points with x^2 + y^2 <= r^2 (Gauss's circle problem, r = 0..8)
GAUSS_CIRCLE = [1, 5, 13, 29, 49, 81, 113, 149, 197]


def _disk(r):
    d = np.arange(-r, r + 1)
    return (d[:, None] ** 2 + d[None, :] ** 2 <= r * r).astype(np.float64)


def _world(H=64, W=80, seed_index=3):
    """One channel, one kernel, mu and sigma maps, gene maintenance on."""
    w = inputs.localized_single_channel(H=H, W=W, R=6, patch=20, n_geno=3, seed_index=seed_index, live=True)
    w.eps_u = 1e-3
    return w


def _events(w, **kw):
    ev = dict(mut_p=0, mut_k=0, mut_x0=10, mut_y0=12, mut_half=4, mut_delta=0.004,
              pen_p=-1, pen_k=0, pen_delta=0.0, gamma_mut=0.0, gamma_pen=0.0, eps_pen=0.5, r_oxy=3)
    ev.update(kw)
    return ev


@pytest.mark.parametrize("r", range(0, 9))
def test_disk_point_counts(oracle, r):
    """Section 2.6: K_oxy is a disk of radius r_oxy; normalised, an impulse
    spreads to the disk's lattice points with weight 1 / N(r)."""
    X = np.zeros((24, 28))
    X[5, 7] = 1.0
    E = oracle.disk_mean(X, r)
    nz = E[E != 0]
    assert nz.size == GAUSS_CIRCLE[r]
    assert np.all(np.abs(nz - 1.0 / GAUSS_CIRCLE[r]) < 1e-16)
    assert abs(E.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("r", [1, 3, 5])
def test_disk_mean_matches_scipy_periodic(oracle, r):
    """A periodic disk average equals scipy's wrap-mode correlation with the
    normalised disk."""
    X = inputs.random_field(77 + r, (40, 56)).astype(np.float64)
    D = _disk(r)
    ref = ndimage.correlate(X, D / D.sum(), mode="wrap")
    np.testing.assert_allclose(oracle.disk_mean(X, r), ref, rtol=0, atol=1e-14)


def test_evolve_without_operators_is_the_plain_step(oracle):
    """With gamma_mut = gamma_pen = 0 and no walls the evolution step is the
    step of Algorithm 2 lines 158-165 (Sections 2.2-2.4) unchanged."""
    w = _world()
    A1, P1, al, _ = oracle.evolve_step(w, _events(w))
    A0, P0, al0 = oracle.step(w, return_alpha=True)
    np.testing.assert_array_equal(A1, A0)
    np.testing.assert_array_equal(P1, P0)
    np.testing.assert_array_equal(al, al0)


@pytest.mark.parametrize("x0,y0,s", [(10, 12, 4), (1, 62, 5), (79, 0, 3)])
def test_mutation_square_and_alpha(oracle, x0, y0, s):
    """Section 2.5: P_{pk} += gamma_mut delta exactly on the periodic square
    x in [x0 - s, x0 + s), y in [y0 - s, y0 + s) intersected with alpha; every
    other gene value is the plain step's."""
    w = _world()
    H, W = w.height, w.width
    gm, dl = 2.5, 0.004
    ev = _events(w, mut_p=1, mut_k=0, mut_x0=x0, mut_y0=y0, mut_half=s, mut_delta=dl, gamma_mut=gm)
    _, P1, al, _ = oracle.evolve_step(w, ev)
    _, P0, al0 = oracle.step(w, return_alpha=True)
    np.testing.assert_array_equal(al, al0)
    sq = np.zeros((H, W), bool)
    sq[np.ix_(np.arange(y0 - s, y0 + s) % H, np.arange(x0 - s, x0 + s) % W)] = True
    expect = (sq & al.astype(bool)) * (gm * dl)
    np.testing.assert_allclose(P1[1, 0] - P0[1, 0], expect, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(P1[0], P0[0])
    # the square must actually touch alpha for the test to say anything
    if (x0, y0) == (10, 12):
        assert (sq & al.astype(bool)).any() or not al.any()


def test_delta_sum_is_the_sum_of_alpha_tests(oracle):
    """Section 2.2: Delta_sum thresholds the sum over kernels of the quantity
    Delta_all tests: h_k g_k (default) or U_k (alpha_on = 1)."""
    w = inputs.multi_channel(H=64, W=64, R=7, patch=24, n_geno=2, seed_index=9, live=True)
    _, _, U = oracle.step(w, return_u=True)
    Ph = np.array([[oracle.diffuse(w.P[p, k], w.r_diff, w.eps_p) for k in range(w.n_kernels)]
                   for p in range(w.n_planes)])
    t = np.zeros((64, 64))
    for k, kd in enumerate(w.kernels):
        mu, sg = Ph[0, k], Ph[1, k]
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(sg > 0, np.exp(-(U[k] - mu) ** 2 / (2 * np.where(sg > 0, sg, 1) ** 2)), 0.0)
        t += kd.h * g
    *_, tsum = oracle.evolve_step(w, _events(w), return_tsum=True)
    np.testing.assert_allclose(tsum, t, rtol=1e-12, atol=1e-14)
    w.alpha_on = 1
    *_, tsum = oracle.evolve_step(w, _events(w), return_tsum=True)
    np.testing.assert_allclose(tsum, U.sum(0), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("r_oxy", [2, 3, 5])
def test_penalising_area_matches_two_library_correlations(oracle, r_oxy):
    """Section 2.6: E_oxy = (1 - Delta_sum(U)) * K_oxy, E_pen = (1 - E_oxy) * K_oxy
    with K_oxy the normalised disk, rebuilt from scipy's periodic correlation.
    Both are averages of averages of 0/1 values, so E_pen N(r)^2 is an integer."""
    w = _world()
    *_, epen, tsum = oracle.evolve_step(w, _events(w, r_oxy=r_oxy), return_tsum=True)
    D = _disk(r_oxy)
    D /= D.sum()
    empty = (~(tsum > w.eps_u)).astype(np.float64)
    e_oxy = ndimage.correlate(empty, D, mode="wrap")
    ref = ndimage.correlate(1.0 - e_oxy, D, mode="wrap")
    np.testing.assert_allclose(epen, ref, rtol=0, atol=1e-13)
    n2 = GAUSS_CIRCLE[r_oxy] ** 2
    assert np.all(np.abs(epen * n2 - np.round(epen * n2)) < 1e-8)


def test_penalising_area_of_a_large_body(oracle):
    """Section 2.6: a body much thicker than 2 r_oxy has E_pen = 1 in its
    interior (no empty site within 2 r_oxy) and nothing far away is penalised."""
    H = W = 96
    k = inputs.KernelDesc(0, 0, 5, inputs.KERNEL_SHELLS, (1.0,), h=1.0, mu=0.3, sigma=0.05)
    A = np.zeros((1, H, W), np.float32)
    A[0, 28:68, 28:68] = 1.0
    P = np.zeros((2, 1, H, W), np.float32)
    P[0, 0, 20:76, 20:76] = 0.3
    P[1, 0, 20:76, 20:76] = 0.05
    w = inputs.World(H, W, 1, [k], 0.1, localized=inputs.LOC_MU | inputs.LOC_SIGMA, maintain_genes=1,
                     alpha_on=1, eps_u=1e-3, A=A, P=P)
    *_, epen, tsum = oracle.evolve_step(w, _events(w, r_oxy=4), return_tsum=True)
    assert epen[48, 48] == 1.0
    assert np.all(epen[:8, :] == 0.0)            # rows 0..7 are > 2 r_oxy from any matter
    # the non-empty region is the body dilated by the kernel's support (R = 5)
    nonempty = tsum > w.eps_u
    assert nonempty[48, 48] and not nonempty[10, 10]


def test_penalisation_acts_on_epen_and_alpha(oracle):
    """Section 2.6: P_{pk} += gamma_pen delta exactly where E_pen > eps_pen and
    alpha hold, after the mutation of the same step (Algorithm 2 order)."""
    w = _world(seed_index=4)
    gp, dl = 0.2, -0.006
    ev = _events(w, pen_p=1, pen_k=0, pen_delta=dl, gamma_pen=gp, eps_pen=0.8, r_oxy=2,
                 mut_p=1, mut_k=0, mut_x0=30, mut_y0=30, mut_half=6, mut_delta=0.003, gamma_mut=1.0)
    _, P1, al, epen = oracle.evolve_step(w, ev)
    _, P0 = oracle.step(w)
    H, W = w.height, w.width
    sq = np.zeros((H, W), bool)
    sq[24:36, 24:36] = True
    a = al.astype(bool)
    expect = (sq & a) * 0.003 + ((epen > 0.8) & a) * (gp * dl)
    np.testing.assert_allclose(P1[1, 0] - P0[1, 0], expect, rtol=0, atol=1e-15)
    assert ((epen > 0.8) & a).any(), "the test world must have a penalised area"
    assert ((epen <= 0.8) & a).any(), "and an unpenalised one"


def test_walls_remove_material_before_the_step(oracle):
    """Section 2.7 and Algorithm 2 (environment first): a step with walls is the
    step from A and P with the wall sites zeroed."""
    w = _world()
    walls = inputs.wall_strip(w.height, w.width, 30, 6)
    A1, P1, al, _ = oracle.evolve_step(w, _events(w), walls=walls)
    keep = (1 - walls).astype(np.float64)
    A0, P0, al0 = oracle.step(w, A=w.A * keep, P=w.P * keep, return_alpha=True)
    np.testing.assert_array_equal(A1, A0)
    np.testing.assert_array_equal(P1, P0)
    np.testing.assert_array_equal(al, al0)


def test_world_filled_with_wall_grows_from_nothing(oracle):
    """A wall over every site leaves A = 0: the signed growth then gives the
    closed form A' = clip(dt sum_k h_k (2 exp(-mu_k^2 / (2 sigma_k^2)) - 1), 0, 1)."""
    w = inputs.global_multi_channel(H=32, W=32, R=5, patch=10)
    for i, kd in enumerate(w.kernels):
        kd.mu = 0.02 * (i % 3)                 # mu = 0 gives G(0) = h
        kd.sigma = 0.03
    walls = np.ones((32, 32), np.uint8)
    A1, *_ = oracle.evolve_step(w, _events(w, mut_p=-1, pen_p=-1), walls=walls)
    for c in range(w.n_channels):
        s = sum(kd.h * (2 * math.exp(-kd.mu ** 2 / (2 * kd.sigma ** 2)) - 1)
                for kd in w.kernels if kd.dst == c)
        assert np.all(np.abs(A1[c] - min(max(w.dt * s, 0.0), 1.0)) < 1e-15)


def test_evolution_events_are_seeded_and_in_range():
    """The random choices of Sections 2.5-2.6 come from the counter-based
    stream: same (seed, step) gives the same events; penalisation raises mu and
    lowers sigma (Figure 3's arrows); a world without gene maps gets none."""
    w = inputs.multi_channel(H=64, W=64, R=6, patch=16, n_geno=2)
    a = [inputs.evolution_events(w, s) for s in range(200)]
    assert a == [inputs.evolution_events(w, s) for s in range(200)]
    for ev in a:
        assert 0 <= ev["mut_p"] < w.n_planes and 0 <= ev["mut_k"] < w.n_kernels
        assert 0 <= ev["mut_x0"] < w.width and 0 <= ev["mut_y0"] < w.height
        assert -0.01 <= ev["mut_delta"] <= 0.01
        assert ev["pen_p"] in (0, 1)
        assert (ev["pen_delta"] >= 0) == (ev["pen_p"] == 0)   # plane 0 is mu, plane 1 is sigma
    assert len({ev["mut_k"] for ev in a}) == w.n_kernels
    g = inputs.global_multi_channel(H=32, W=32, R=5, patch=10)
    ev = inputs.evolution_events(g, 0)
    assert ev["mut_p"] == -1 and ev["pen_p"] == -1
