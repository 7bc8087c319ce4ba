"""Pins for the FP64 oracle: facts fixed by the paper or by mathematics, not
by the oracle's own formulas.  CPU only.

Each test names the passage it rests on (arXiv 2304.05639 sections and
algorithms; the kernel shell and signed growth come from the original Lenia
definitions that the paper cites in Section 1.2)."""
import math
import os

import numpy as np
import pytest

from paper_2304_05639_gb300 import inputs


# ---------------------------------------------------------------- kernels

@pytest.mark.parametrize("R,beta", [(5, (1.0,)), (13, (1.0,)), (18, (0.3, 0.9, 0.5)), (9, (0.2, 1.0))])
def test_kernel_normalised(oracle, R, beta):
    """Algorithm 1 and the note after Algorithm 2: K~ = K / (K * 1), K * 1 = sum K."""
    K = oracle.kernel(R, 0, beta)
    assert K.shape == (2 * R + 1, 2 * R + 1)
    assert abs(K.sum() - 1.0) < 1e-14
    assert (K >= 0).all()


@pytest.mark.parametrize("R,beta", [(7, (1.0,)), (12, (0.4, 1.0, 0.7))])
def test_kernel_d4_symmetric(oracle, R, beta):
    """A kernel that depends on |d| only is invariant under the 8 grid symmetries."""
    K = oracle.kernel(R, 0, beta)
    for t in (K[::-1], K[:, ::-1], K.T, K[::-1, ::-1].T):
        np.testing.assert_array_equal(K, t)


def test_kernel_shell_special_values(oracle):
    """Shell kernel beta[floor(B rho)] core(B rho mod 1), rho = |d| / R:
    core(1/2) = 1 so a pixel at the middle of shell i carries beta_i; shell
    boundaries (B rho integer), the centre and rho = 1 carry 0."""
    R, beta = 8, (0.3, 0.7)                    # B = 2
    K = oracle.kernel(R, 0, beta)
    c = R
    mid0 = K[c, c + 2]                         # rho = 1/4 -> B rho = 1/2
    mid1 = K[c, c + 6]                         # rho = 3/4 -> B rho = 3/2
    assert abs(mid0 / mid1 - 0.3 / 0.7) < 1e-14
    assert K[c, c + 4] == 0.0                  # rho = 1/2, B rho = 1 (boundary)
    assert K[c, c] == 0.0                      # centre
    assert K[c, c + 8] == 0.0                  # rho = 1
    assert K[c + 8, c] == 0.0
    assert mid0 == K[c + 2, c] == K[c - 2, c] == K[c, c - 2]


def test_kernel_core_closed_forms(oracle):
    """One shell: core(q) = exp(4 - 1/(q(1-q))) gives core(1/4) = exp(-4/3),
    core(1/2) = 1, and core(q) = core(1 - q)."""
    R = 8
    K = oracle.kernel(R, 0, (1.0,))
    c = R
    assert abs(K[c, c + 2] / K[c, c + 4] - math.exp(-4.0 / 3.0)) < 1e-14
    assert abs(K[c, c + 3] / K[c, c + 5] - 1.0) < 1e-14
    assert np.argmax(K) in {np.ravel_multi_index(ix, K.shape) for ix in
                            [(c, c + 4), (c, c - 4), (c + 4, c), (c - 4, c)]}


def test_kernel_bump_form(oracle):
    """Section 2.4 kernel function k(x; r, w, b) = b exp(-(x-r)^2 / 2w^2): one
    bump peaks at x = r and falls to exp(-1/2) of the peak at x = r + w."""
    R = 10
    K = oracle.kernel(R, 1, bump=(0.5, 0.1, 2.0, 0.0, 1.0, 0.0))
    c = R
    assert abs(K[c, c + 6] / K[c, c + 5] - math.exp(-0.5)) < 1e-13
    assert K[c, c + 5] == K.max()
    assert K[c, c + 10] == 0.0                 # rho = 1 is outside


@pytest.mark.parametrize("R,form,beta,bump", [(13, 0, (1.0,), None), (18, 0, (0.3, 0.9, 0.5), None),
                                              (16, 0, (1.0, 0.5), None),
                                              (12, 1, (1.0,), (0.3, 0.15, 1.0, 0.8, 0.1, 0.5))])
def test_kernel_support_is_open_disk(oracle, R, form, beta, bump):
    """Algorithm 1: the kernel is defined for d / R < 1 only, so every tap with
    dx^2 + dy^2 >= R^2 is zero (the corners of the (2R+1)^2 square and the
    axis taps at distance R), while taps well inside the disk are not."""
    K = oracle.kernel(R, form, beta) if bump is None else oracle.kernel(R, form, bump=bump)
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    outside = dx * dx + dy * dy >= R * R
    assert (K[outside] == 0.0).all()
    assert K[R, 0] == 0.0 and K[0, R] == 0.0          # |d| = R exactly
    assert (K[~outside] > 0).sum() > 0.5 * (~outside).sum()


# ------------------------------------------------------------ convolution

def _embed(K, H, W):
    """Kernel taps placed at their (wrapped) offsets on an H x W torus."""
    R = (K.shape[0] - 1) // 2
    E = np.zeros((H, W))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            E[dy % H, dx % W] += K[dy + R, dx + R]
    return E


def test_potential_equals_library_fft(oracle):
    """Convolution theorem (note after Algorithm 2): X * Y = F^-1(FX . FY),
    checked against numpy's FFT (a library routine)."""
    H, W, R = 32, 48, 6
    A = inputs.random_field(11, (H, W)).astype(np.float64)
    K = oracle.kernel(R, 0, (0.6, 1.0))
    U = oracle.potential(A, K)
    ref = np.real(np.fft.ifft2(np.fft.fft2(A) * np.fft.fft2(_embed(K, H, W))))
    assert np.max(np.abs(U - ref)) < 1e-13


def test_potential_equals_bruteforce_dft(oracle):
    """Same theorem with an explicit O(N^2) DFT matrix on a tiny torus."""
    H, W, R = 12, 10, 4
    A = inputs.random_field(12, (H, W)).astype(np.float64)
    K = oracle.kernel(R, 0, (1.0,))
    Fy = np.exp(-2j * np.pi * np.outer(np.arange(H), np.arange(H)) / H)
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(W), np.arange(W)) / W)
    dft = lambda X: Fy @ X @ Fx.T
    idft = lambda X: np.conj(Fy) @ X @ np.conj(Fx).T / (H * W)
    ref = np.real(idft(dft(A) * dft(_embed(K, H, W))))
    assert np.max(np.abs(oracle.potential(A, K) - ref)) < 1e-13


def test_potential_uniform_field(oracle):
    """K~ * a = a for a constant field because K~ sums to 1."""
    K = oracle.kernel(13, 0, (1.0,))
    U = oracle.potential(np.full((40, 36), 0.37), K)
    assert np.max(np.abs(U - 0.37)) < 1e-15


def test_potential_translation_equivariant(oracle):
    """The toroidal world (Section 2.1) makes convolution commute with rolls, exactly."""
    A = inputs.random_field(13, (30, 34)).astype(np.float64)
    K = oracle.kernel(7, 0, (0.5, 1.0))
    U = oracle.potential(A, K)
    Ur = oracle.potential(np.roll(A, (5, -9), axis=(0, 1)), K)
    np.testing.assert_array_equal(Ur, np.roll(U, (5, -9), axis=(0, 1)))


def test_potential_delta_wraps(oracle):
    """A unit impulse next to the edge reproduces the kernel, wrapped round the torus."""
    H, W, R = 24, 20, 5
    A = np.zeros((H, W))
    A[1, W - 2] = 1.0
    K = oracle.kernel(R, 0, (1.0,))
    U = oracle.potential(A, K)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            assert U[(1 + dy) % H, (W - 2 + dx) % W] == K[dy + R, dx + R]


def test_potential_extended_precision_gap(oracle):
    """The FP64 sum differs from a long-double sum by far less than 1e-12
    (each potential is <= 1018 terms of size <= 1)."""
    A = inputs.random_field(14, (48, 48)).astype(np.float64)
    K = oracle.kernel(18, 0, (0.3, 1.0, 0.6))
    gap = np.max(np.abs(oracle.potential(A, K) - oracle.potential(A, K, extended=True)))
    assert gap < 1e-13


# -------------------------------------------------------------- diffusion

def test_diffuse_constant_region(oracle):
    """Section 2.3: averaging over non-zero neighbours keeps a constant region."""
    P = np.zeros((20, 20))
    P[5:15, 4:16] = 0.3
    D = oracle.diffuse(P, 1, 0.0)
    assert np.all(D[6:14, 5:15] == 0.3)


def test_diffuse_single_site_spreads_to_disk(oracle):
    """One non-zero site of value v: every site whose disk contains it gets v
    (it is the only non-zero term).  Disk |d| <= r: 5 sites for r = 1, 13 for r = 2."""
    for r, n in ((1, 5), (2, 13)):
        P = np.zeros((16, 16))
        P[8, 8] = 0.42
        D = oracle.diffuse(P, r, 0.0)
        assert np.count_nonzero(D) == n
        assert np.all(D[D != 0] == 0.42)


def test_diffuse_hand_values(oracle):
    """Two neighbours 0.2 (at x=5) and 0.6 (at x=6) on one row, r = 1:
    x=4 sees {0.2} -> 0.2; x=5 sees {0.2, 0.6} -> 0.4; x=6 -> 0.4; x=7 -> 0.6;
    the rows above and below see one value each."""
    P = np.zeros((9, 12))
    P[4, 5], P[4, 6] = 0.2, 0.6
    D = oracle.diffuse(P, 1, 0.0)
    assert D[4, 4] == pytest.approx(0.2, abs=1e-16)
    assert D[4, 5] == pytest.approx(0.4, abs=1e-16)
    assert D[4, 6] == pytest.approx(0.4, abs=1e-16)
    assert D[4, 7] == pytest.approx(0.6, abs=1e-16)
    assert D[3, 5] == 0.2 and D[5, 6] == 0.6 and D[3, 7] == 0.0


def test_diffuse_zero_and_clip(oracle):
    """All-zero genes stay zero; the result is clipped to [0, 1] (Section 2.3)."""
    assert np.all(oracle.diffuse(np.zeros((8, 8)), 1, 0.0) == 0)
    D = oracle.diffuse(np.full((8, 8), 1.5), 1, 0.0)
    assert np.all(D == 1.0)


def test_diffuse_threshold_counts(oracle):
    """Delta_same(P) uses eps: a value at or below eps is summed but not counted."""
    P = np.zeros((8, 8))
    P[3, 3], P[3, 4] = 0.5, 0.01
    D = oracle.diffuse(P, 1, 0.01)
    assert D[3, 3] == pytest.approx(0.51, abs=1e-15)   # (0.5 + 0.01) / 1
    D0 = oracle.diffuse(P, 1, 0.0)
    assert D0[3, 3] == pytest.approx(0.255, abs=1e-15)  # (0.5 + 0.01) / 2


# ------------------------------------------------ growth, update and mask

def _uniform_world(a, mu, sigma, h=1.0, dt=0.1, form=0, H=24, W=24, R=5):
    k = inputs.KernelDesc(0, 0, R, 0, (1.0,), h=h, mu=mu, sigma=sigma)
    A = np.full((1, H, W), a, np.float32)
    return inputs.World(H, W, 1, [k], dt, growth_form=form, A=A)


def test_update_at_growth_peak(oracle):
    """U = mu gives g = 1, so the signed growth is +h: A' = a + dt h."""
    a = 0.25
    w = _uniform_world(a, mu=float(np.float32(a)), sigma=0.02, h=0.8)
    A1, _ = oracle.step(w)
    assert np.max(np.abs(A1 - (float(np.float32(a)) + 0.1 * 0.8))) < 1e-12


def test_update_half_height_is_stationary(oracle):
    """|U - mu| = sigma sqrt(2 ln 2) gives g = 1/2, so 2g - 1 = 0 and A' = A."""
    a, s = 0.3, 0.015
    mu = float(np.float32(a)) - s * math.sqrt(2 * math.log(2))
    A1, _ = oracle.step(_uniform_world(a, mu=mu, sigma=s))
    assert np.max(np.abs(A1 - float(np.float32(a)))) < 1e-12


def test_update_width_is_sigma(oracle):
    """|U - mu| = sigma gives g = exp(-1/2) (the 2 sigma^2 denominator)."""
    a, s, dt = 0.3, 0.02, 0.1
    mu = float(np.float32(a)) - s
    A1, _ = oracle.step(_uniform_world(a, mu=mu, sigma=s, dt=dt))
    assert np.max(np.abs(A1 - (float(np.float32(a)) + dt * (2 * math.exp(-0.5) - 1)))) < 1e-12


def test_update_paper_form(oracle):
    """Section 2.4 form G = h exp(...) >= 0: at U = mu the increment is dt h."""
    a = 0.2
    w = _uniform_world(a, mu=float(np.float32(a)), sigma=0.05, h=0.5, form=1)
    A1, _ = oracle.step(w)
    assert np.max(np.abs(A1 - (float(np.float32(a)) + 0.1 * 0.5))) < 1e-12


def test_update_clips(oracle):
    """[x]_0^1 (note after Algorithm 2): far from mu the signed growth is -1;
    large dt drives A to exactly 0, and at the peak to exactly 1."""
    A1, _ = oracle.step(_uniform_world(0.3, mu=0.9, sigma=0.01, dt=1.0))
    assert np.all(A1 == 0.0)
    A1, _ = oracle.step(_uniform_world(0.9, mu=float(np.float32(0.9)), sigma=0.01, dt=1.0))
    assert np.all(A1 == 1.0)


def test_zero_field_stays_zero(oracle):
    """Empty world with mu = 0.15, sigma = 0.015: g = exp(-50), the growth is
    about -1 and the clip keeps A at 0."""
    A1, _ = oracle.step(_uniform_world(0.0, mu=0.15, sigma=0.015))
    assert np.all(A1 == 0.0)


def _read_golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    d = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            parts = line.split()
            d[" ".join(parts[:-1])] = parts[-1]
    return d


def test_two_channel_routing_golden(oracle):
    """Kernel k reads channel src(k) and writes channel dst(k) (Section 2.1
    topology; Algorithm 1 update A_i += sum_k G_k(K~_k * A_j)).  Hand-derived
    values in tests/golden/two_channel_uniform.txt."""
    g = _read_golden("two_channel_uniform.txt")
    H, W, dt = int(g["H"]), int(g["W"]), float(g["dt"])
    a0, a1, s = float(g["a0"]), float(g["a1"]), float(g["sigma"])
    ks = [inputs.KernelDesc(0, 0, 4, 0, (1.0,), h=0.5, mu=a0, sigma=s),
          inputs.KernelDesc(0, 1, 4, 0, (1.0,), h=0.75, mu=a0 + s * math.sqrt(2 * math.log(2)), sigma=s),
          inputs.KernelDesc(1, 0, 4, 0, (1.0,), h=0.25, mu=a1, sigma=s)]
    A = np.stack([np.full((H, W), a0), np.full((H, W), a1)]).astype(np.float32)
    w = inputs.World(H, W, 2, ks, dt, A=A)
    A1, _ = oracle.step(w)
    assert np.max(np.abs(A1[0] - float(g["expect A0"]))) < 1e-12
    assert np.max(np.abs(A1[1] - float(g["expect A1"]))) < 1e-12


def _gene_world(a, mu, sigma, H=20, W=20, R=4, eps_u=0.01, alpha_on=0, h=1.0):
    k = inputs.KernelDesc(0, 0, R, 0, (1.0,), h=h)
    A = np.full((1, H, W), a, np.float32)
    P = np.zeros((2, 1, H, W), np.float32)
    P[0, 0, 4:16, 4:16] = mu
    P[1, 0, 4:16, 4:16] = sigma
    return inputs.World(H, W, 1, [k], 0.1, localized=3, maintain_genes=1, eps_u=eps_u,
                        alpha_on=alpha_on, A=A, P=P)


def test_mask_keeps_genes_inside_envelope(oracle):
    """Section 2.2: alpha = Delta_all(U) and Delta_all(P).  Uniform A at the
    gene mu gives growth h g = h > eps, so alpha = Delta_all(P_diffused) and
    the genes survive (diffused) exactly there."""
    a = float(np.float32(0.2))
    w = _gene_world(a, a, 0.03)
    A1, P1, alpha = oracle.step(w, return_alpha=True)
    D = np.stack([oracle.diffuse(w.P[p, 0]) for p in range(2)])
    assert np.array_equal(alpha.astype(bool), np.all(D > 0, axis=0))
    np.testing.assert_array_equal(P1[:, 0], D * alpha)
    inside = alpha.astype(bool)
    assert np.max(np.abs(A1[0][inside] - (a + 0.1))) < 1e-12
    # outside alpha the genes are zero and the signed growth is -h (reading R9)
    assert np.max(np.abs(A1[0][~inside] - (a - 0.1))) < 1e-12


def test_mask_kills_genes_without_growth(oracle):
    """Where h g <= eps for some kernel alpha is 0 and every gene is zeroed."""
    w = _gene_world(0.9, 0.1, 0.01)
    _, P1, alpha = oracle.step(w, return_alpha=True)
    assert alpha.sum() == 0 and np.all(P1 == 0)


def test_mask_idempotent_and_subset(oracle):
    """Masking again with the same alpha changes nothing; alpha lies inside Delta_all(P)."""
    w = inputs.localized_single_channel(H=64, W=64, R=6, patch=16, n_geno=4, live=True)
    _, P1, alpha = oracle.step(w, return_alpha=True)
    np.testing.assert_array_equal(P1 * alpha, P1)
    D = np.stack([oracle.diffuse(w.P[p, 0]) for p in range(2)])
    assert np.all(~alpha.astype(bool) | np.all(D > 0, axis=0))


def test_mask_on_potential_switch(oracle):
    """Switch alpha_on = 1: alpha tests U > eps instead of the growth."""
    w = _gene_world(0.005, 0.3, 0.05, alpha_on=1)
    _, _, alpha = oracle.step(w, return_alpha=True)
    assert alpha.sum() == 0                          # U = 0.005 <= 0.01
    w = _gene_world(0.02, 0.3, 0.05, alpha_on=1)
    _, _, alpha = oracle.step(w, return_alpha=True)
    D = oracle.diffuse(w.P[0, 0])
    assert np.array_equal(alpha.astype(bool), D > 0)


def _uniform_gene_world(a, genes, localized=3, H=16, W=16, R=3, dt=0.1, dst=None, C=1, h=None):
    """Uniform phenospace a (per channel) and uniform gene planes over the
    whole torus: every normalised potential is exactly a (K~ * 1 = 1), the
    diffusion of a constant plane returns it (five equal FP32 values sum
    exactly in FP64), so each kernel's growth has a closed form.
    genes[k] = (mu, sigma[, h]) of kernel k; kernel k reads and writes
    channel dst[k] (default 0)."""
    K = len(genes)
    dst = dst or [0] * K
    ks = [inputs.KernelDesc(dst[k], dst[k], R, 0, (1.0,), h=(h[k] if h else 1.0)) for k in range(K)]
    av = [a] * C if np.isscalar(a) else list(a)
    A = np.stack([np.full((H, W), v, np.float32) for v in av])
    n_p = bin(localized).count("1")
    P = np.zeros((n_p, K, H, W), np.float32)
    for k, gk in enumerate(genes):
        for p in range(n_p):
            P[p, k] = np.float32(gk[p])
    return inputs.World(H, W, C, ks, dt, localized=localized, maintain_genes=1, A=A, P=P)


def _g(u, mu, s):
    return math.exp(-(u - mu) ** 2 / (2.0 * s * s))


def test_mask_is_and_over_kernels(oracle):
    """Section 2.2: Delta_all(U) holds only where EVERY kernel's growth test
    passes.  Three kernels on a uniform world: kernels 0 and 2 sit at their
    growth peak (h g = 1 > eps), kernel 1 far from it (g = exp(-112.5)).  The
    AND is false, so alpha = 0, every gene is zeroed, and each kernel's
    masked growth is -h (reading R9): A' = a - 3 dt.  (An OR over kernels, or
    a test of only the first or only the last kernel, would keep the genes.)"""
    a = float(np.float32(0.3))
    w = _uniform_gene_world(a, [(a, 0.02), (a + 0.3, 0.02), (a, 0.05)])
    A1, P1, alpha = oracle.step(w, return_alpha=True)
    assert alpha.sum() == 0 and np.all(P1 == 0)
    assert np.max(np.abs(A1 - (a - 3 * 0.1))) < 1e-12
    # every kernel passing: alpha = 1 everywhere, genes kept, the closed form
    mus = [a, float(np.float32(a - 0.02)), float(np.float32(a + 0.03))]
    sgs = [0.02, 0.03, 0.05]
    w = _uniform_gene_world(a, list(zip(mus, sgs)))
    A1, P1, alpha = oracle.step(w, return_alpha=True)
    assert alpha.all()
    np.testing.assert_array_equal(P1, w.P.astype(np.float64))
    sgs32 = [float(np.float32(s)) for s in sgs]
    inc = sum(2 * _g(a, m, s) - 1 for m, s in zip(mus, sgs32))
    assert np.max(np.abs(A1 - (a + 0.1 * inc))) < 1e-12


def test_mask_and_spans_channels(oracle):
    """alpha is one decision per site over all kernels, whatever channel they
    write: a failing kernel of channel 1 also masks channel 0's kernel, whose
    growth then is -h (not +h)."""
    a0, a1 = float(np.float32(0.2)), float(np.float32(0.6))
    w = _uniform_gene_world([a0, a1], [(a0, 0.02), (a1 + 0.3, 0.02)], dst=[0, 1], C=2, h=[0.5, 0.25])
    A1, P1, alpha = oracle.step(w, return_alpha=True)
    assert alpha.sum() == 0 and np.all(P1 == 0)
    assert np.max(np.abs(A1[0] - (a0 - 0.1 * 0.5))) < 1e-12
    assert np.max(np.abs(A1[1] - (a1 - 0.1 * 0.25))) < 1e-12


def test_localized_h_masked_where_alpha_is_zero(oracle):
    """Reading R9 with a localized h: the update uses the masked genes, so
    where alpha = 0 the gene h is 0 and the growth h (2 g - 1) is 0: A' = a
    exactly (with a global h the same site would get -h).  Where alpha = 1
    the site's own h scales the closed-form growth."""
    a = float(np.float32(0.4))
    hk = float(np.float32(0.7))
    # genes die: mu far from U = a
    w = _uniform_gene_world(a, [(a + 0.3, 0.02, hk)], localized=7)
    A1, P1, alpha = oracle.step(w, return_alpha=True)
    assert alpha.sum() == 0 and np.all(P1 == 0)
    np.testing.assert_array_equal(A1, w.A.astype(np.float64))
    # the same world with a global h = 0.7: A' = a - dt h
    wg = _uniform_gene_world(a, [(a + 0.3, 0.02)], localized=3, h=[hk])
    A1g, _ = oracle.step(wg)
    assert np.max(np.abs(A1g - (a - 0.1 * hk))) < 1e-12
    # genes alive: growth hk (2 g - 1) with the site's h
    mu = float(np.float32(a - 0.01))
    w = _uniform_gene_world(a, [(mu, 0.03, hk)], localized=7)
    A1, P1, alpha = oracle.step(w, return_alpha=True)
    assert alpha.all()
    s32 = float(np.float32(0.03))
    assert np.max(np.abs(A1 - (a + 0.1 * hk * (2 * _g(a, mu, s32) - 1)))) < 1e-12


def test_step_translation_equivariant(oracle):
    """The whole step commutes with torus rolls (all operations are local and periodic)."""
    w = inputs.multi_channel(H=48, W=40, R=5, patch=12, n_geno=3, live=True)
    A1, P1 = oracle.step(w)
    sh = (7, -11)
    A1r, P1r = oracle.step(w, A=np.roll(w.A, sh, axis=(1, 2)), P=np.roll(w.P, sh, axis=(2, 3)))
    np.testing.assert_array_equal(A1r, np.roll(A1, sh, axis=(1, 2)))
    np.testing.assert_array_equal(P1r, np.roll(P1, sh, axis=(2, 3)))


def test_step_bounds(oracle):
    """Clip bounds: 0 <= A' <= 1 and 0 <= P' <= 1 on a random multi-channel world."""
    w = inputs.multi_channel(H=48, W=48, R=6, patch=16, n_geno=4)
    A1, P1 = oracle.step(w)
    assert A1.min() >= 0 and A1.max() <= 1 and P1.min() >= 0 and P1.max() <= 1


# ------------------------------------------------------------------ stats

def test_stats_uniform_mass(oracle):
    st = oracle.stats(np.full((2, 16, 24), 0.5))
    assert np.allclose(st[:, 0], 0.5 * 16 * 24, atol=1e-12)


def test_stats_single_pixel_centroid(oracle):
    A = np.zeros((1, 32, 40))
    A[0, 7, 33] = 0.8
    st = oracle.stats(A)
    assert abs(st[0, 1] - 7) < 1e-9 and abs(st[0, 2] - 33) < 1e-9


def test_stats_roll_shifts_centroid(oracle):
    A = np.zeros((1, 64, 64))
    A[0, 20:30, 10:18] = inputs.random_field(3, (10, 8))
    s0 = oracle.stats(A)
    s1 = oracle.stats(np.roll(A, (5, 50), axis=(1, 2)))
    assert abs(s1[0, 1] - (s0[0, 1] + 5) % 64) < 1e-9
    assert abs(s1[0, 2] - (s0[0, 2] + 50) % 64) < 1e-9


# ----------------------------------------------------------------- inputs

def test_splitmix64_reference_vector():
    """SplitMix64 seeded with 0 starts 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4."""
    z = inputs.splitmix64(0, 2)
    assert int(z[0]) == 0xE220A8397B1DCDAF and int(z[1]) == 0x6E789E6AA1B965F4


def test_inputs_deterministic_and_shaped():
    a = inputs.multi_channel(H=64, W=64, R=6, patch=16, n_geno=4)
    b = inputs.multi_channel(H=64, W=64, R=6, patch=16, n_geno=4)
    np.testing.assert_array_equal(a.A, b.A)
    np.testing.assert_array_equal(a.P, b.P)
    assert a.A.shape == (3, 64, 64) and a.P.shape == (2, 15, 64, 64)
    assert [(k.src, k.dst) for k in a.kernels][:3] == [(0, 0)] * 3
    assert len(a.kernels) == 15


# --------------------------------------------- oracle entry points agree

def test_update_and_sites_agree_with_step(oracle):
    """The update-from-potentials and sampled-site entries reproduce the full
    step exactly (same arithmetic, different drivers)."""
    w = inputs.multi_channel(H=40, W=48, R=5, patch=12, n_geno=3, live=True)
    A1, P1, U, al = oracle.step(w, return_u=True, return_alpha=True)
    A2, P2, al2 = oracle.update(w, w.A, w.P, U, return_alpha=True)
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(P1, P2)
    np.testing.assert_array_equal(al, al2)
    ys = np.array([0, 5, 39, 17, 20]); xs = np.array([0, 47, 3, 22, 30])
    r = oracle.step_sites(w, ys, xs)
    np.testing.assert_array_equal(r["A"], A1[:, ys, xs])
    np.testing.assert_array_equal(r["P"], P1.reshape(-1, 40, 48)[:, ys, xs])
    np.testing.assert_array_equal(r["U"], U[:, ys, xs])
    np.testing.assert_array_equal(r["alpha"], al[ys, xs])
