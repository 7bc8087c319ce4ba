"""Seeded synthetic Lenia worlds.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no kernels, no growth, no convolution).  Both the CUDA
path and the FP64 oracle are fed from it, so it must stay free of either.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style:
draw i of stream s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).  Floats in
[0, 1) take the top 24 bits, so every draw is exactly representable in FP32.

World shapes follow the paper's set-up (Section 2.1: toroidal grid, c channels,
k kernels with 3 self kernels per channel and 2 cross kernels per channel
pair; Section 2.2: per-site gene tensor P[p, k, y, x]).  The paper's seed
creature and runs are not published, so patches of random genotypes stand in
for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
BASE_SEED = 230405639

# Growth form codes and localized-gene bits shared by the C-ABI and the oracle.
GROWTH_SIGNED = 0      # 2*exp(-(u-m)^2/(2 s^2)) - 1, scaled by h
GROWTH_PAPER = 1       # h*exp(-(u-m)^2/(2 s^2))   (Section 2.4 form)
LOC_MU, LOC_SIGMA, LOC_H = 1, 2, 4
LOC_KERNEL = 8         # ring-wise kernel genes r1, w1, b1, r2, w2, b2 (six planes)
KERNEL_SHELLS, KERNEL_BUMPS = 0, 1
HALF_HEIGHT = 1.1774100225154747   # sqrt(2 ln 2): where exp(-z^2 / 2) = 1/2


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64(stream: int, n: int) -> np.ndarray:
    """n uint64 draws of the counter-based SplitMix64 stream `stream`."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream % (1 << 64)) + i * GOLDEN
    return _mix(z)


class Rng:
    """Counter-based stream: every call consumes a fresh, disjoint range."""

    def __init__(self, seed: int):
        self.stream = int(_mix(np.array([seed % (1 << 64)], dtype=np.uint64))[0])
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        i = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.stream) + i * GOLDEN
        return _mix(z)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """float32 draws in [lo, hi); exact FP32 grid values when lo=0, hi=1."""
        u = (self.bits(n) >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
        return (lo + (hi - lo) * u).astype(np.float32)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """int64 draws uniform on {lo, ..., hi} (inclusive)."""
        span = hi - lo + 1
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + np.minimum((u * span).astype(np.int64), span - 1)


@dataclasses.dataclass
class KernelDesc:
    src: int
    dst: int
    radius: int
    form: int = KERNEL_SHELLS
    beta: tuple = (1.0,)
    bump: tuple = (0.0,) * 6
    h: float = 1.0
    mu: float = 0.15
    sigma: float = 0.015


@dataclasses.dataclass
class World:
    """Everything one step needs: configuration, kernels and the state."""
    height: int
    width: int
    n_channels: int
    kernels: list
    dt: float
    growth_form: int = GROWTH_SIGNED
    localized: int = 0
    maintain_genes: int = 0
    eps_u: float = 0.01
    eps_p: float = 0.0
    r_diff: int = 1
    alpha_on: int = 0
    A: np.ndarray | None = None      # float32 [C, H, W]
    P: np.ndarray | None = None      # float32 [n_p, K, H, W] or None
    name: str = ""
    n_rings: int = 0                 # ring decomposition (with LOC_KERNEL)

    @property
    def n_kernels(self) -> int:
        return len(self.kernels)

    @property
    def n_planes(self) -> int:
        return bin(self.localized & 7).count("1") + (6 if self.localized & LOC_KERNEL else 0)

    @property
    def sites(self) -> int:
        return self.height * self.width


def paper_topology(n_channels: int, n_self: int = 3, n_cross: int = 2):
    """(src, dst) pairs: n_self self kernels per channel, then for each channel
    pair (i, j), i < j, alternately i->j and j->i (n_cross per pair)."""
    pairs = []
    for c in range(n_channels):
        pairs += [(c, c)] * n_self
    for i in range(n_channels):
        for j in range(i + 1, n_channels):
            for t in range(n_cross):
                pairs.append((i, j) if t % 2 == 0 else (j, i))
    return pairs


def _place_patches(rng: Rng, H: int, W: int, side: int, n_geno: int, margin: int):
    """Square patches at uniform random centres (toroidal).  Returns, per
    genotype, the (rows, cols) index vectors of the patch and of the patch plus
    `margin`; later genotypes overwrite earlier ones."""
    cy = rng.integers(n_geno, 0, H - 1)
    cx = rng.integers(n_geno, 0, W - 1)
    out = []
    for g in range(n_geno):
        def span(c, n, half):
            return (np.arange(c - half, c - half + 2 * half) % n)
        h0 = side // 2
        out.append((span(cy[g], H, h0), span(cx[g], W, h0),
                    span(cy[g], H, h0 + margin), span(cx[g], W, h0 + margin)))
    return out


def single_kernel_global(H=64, W=64, R=13, patch=20, seed_index=0, dt=0.1,
                         mu=0.15, sigma=0.015, h=1.0, name="c1") -> World:
    """Plain single-channel Lenia: one shell kernel, global genes, a central
    square of U[0,1) noise on an empty torus."""
    rng = Rng(BASE_SEED + seed_index)
    A = np.zeros((1, H, W), np.float32)
    y0, x0 = H // 2 - patch // 2, W // 2 - patch // 2
    A[0, y0:y0 + patch, x0:x0 + patch] = rng.uniform(patch * patch).reshape(patch, patch)
    k = KernelDesc(0, 0, R, KERNEL_SHELLS, (1.0,), h=h, mu=mu, sigma=sigma)
    return World(H, W, 1, [k], dt, A=A, name=name)


def localized_single_channel(H=1024, W=1024, R=12, patch=128, n_geno=16,
                             seed_index=1, dt=0.1, name="c2",
                             mu_range=(0.10, 0.40), sigma_range=(0.01, 0.06),
                             live=False) -> World:
    """One channel, one shell kernel, per-site mu/sigma maps from n_geno random
    genotypes on square patches; gene maintenance on.  With live=True the patch
    noise is scaled to U[0, 2 mu_g) so the initial potential sits near mu."""
    rng = Rng(BASE_SEED + seed_index)
    mus = rng.uniform(n_geno, *mu_range)
    sigmas = rng.uniform(n_geno, *sigma_range)
    A = np.zeros((1, H, W), np.float32)
    P = np.zeros((2, 1, H, W), np.float32)
    for g, (ry, rx, my, mx) in enumerate(_place_patches(rng, H, W, patch, n_geno, R)):
        P[0, 0][np.ix_(my, mx)] = mus[g]
        P[1, 0][np.ix_(my, mx)] = sigmas[g]
        noise = rng.uniform(len(ry) * len(rx)).reshape(len(ry), len(rx))
        if live:
            noise = (noise * np.float32(2.0 * mus[g])).astype(np.float32)
        A[0][np.ix_(ry, rx)] = noise
    k = KernelDesc(0, 0, R, KERNEL_SHELLS, (1.0,), h=1.0,
                   mu=float(np.mean(mus)), sigma=float(np.mean(sigmas)))
    return World(H, W, 1, [k], dt, localized=LOC_MU | LOC_SIGMA, maintain_genes=1,
                 A=A, P=P, name=name)


def multi_channel(H=2048, W=2048, R=18, patch=256, n_geno=16, seed_index=2,
                  dt=0.2, n_channels=3, localized=LOC_MU | LOC_SIGMA,
                  maintain=1, name="c3", mu_range=(0.10, 0.40),
                  sigma_range=(0.01, 0.06), live=False, matched=False) -> World:
    """Multi-channel world with the paper's kernel topology (15 kernels for 3
    channels).  Shells B ~ U{1,2,3}, beta ~ U[0,1), h ~ U[0.1,1).  n_geno
    genotypes, each with per-kernel (mu, sigma), fill square patches; A is
    U[0,1) noise on each patch (U[0, 2 mu) per channel when live=True).

    matched=True (implies live) draws genotypes whose kernels agree with the
    patch they sit on, so that the patch interiors pass every kernel's growth
    test at once: per genotype and channel c a level L ~ U[mu_range); every
    kernel reading c gets sigma ~ U[0.03, 0.06) and mu = L - 1.1774 sigma +
    U[-0.01, 0.01); channel c's noise is U[0, 2 L), whose local mean (the
    potential) is L.  1.1774 = sqrt(2 ln 2) places L near the half-height point
    of each kernel's bump on its upper side, so the patches start close to
    an equilibrium (a larger potential lowers the growth) and stay alive for
    a number of steps.""" 
    rng = Rng(BASE_SEED + seed_index)
    topo = paper_topology(n_channels)
    K = len(topo)
    kernels = []
    for (s, d) in topo:
        B = int(rng.integers(1, 1, 3)[0])
        beta = tuple(float(b) for b in rng.uniform(B))
        h = float(rng.uniform(1, 0.1, 1.0)[0])
        kernels.append(KernelDesc(s, d, R, KERNEL_SHELLS, beta, h=h))
    if matched:
        live = True
        level = rng.uniform(n_geno * n_channels, *mu_range).reshape(n_geno, n_channels)
        jitter = rng.uniform(n_geno * K, -0.01, 0.01).reshape(n_geno, K)
        src = np.array([s for (s, _) in topo])
        sigmas = rng.uniform(n_geno * K, 0.03, 0.06).reshape(n_geno, K)
        mus = (level[:, src] + jitter - np.float32(HALF_HEIGHT) * sigmas).astype(np.float32)
    else:
        mus = rng.uniform(n_geno * K, *mu_range).reshape(n_geno, K)
        sigmas = rng.uniform(n_geno * K, *sigma_range).reshape(n_geno, K)
    for k in range(K):
        kernels[k].mu = float(np.mean(mus[:, k]))
        kernels[k].sigma = float(np.mean(sigmas[:, k]))
    A = np.zeros((n_channels, H, W), np.float32)
    n_p = bin(localized).count("1")
    P = np.zeros((n_p, K, H, W), np.float32) if localized else None
    for g, (ry, rx, my, mx) in enumerate(_place_patches(rng, H, W, patch, n_geno, R)):
        if P is not None:
            planes = []
            if localized & LOC_MU:
                planes.append(mus[g])
            if localized & LOC_SIGMA:
                planes.append(sigmas[g])
            if localized & LOC_H:
                planes.append(np.array([kk.h for kk in kernels], np.float32))
            for p, vals in enumerate(planes):
                for k in range(K):
                    P[p, k][np.ix_(my, mx)] = vals[k]
        for c in range(n_channels):
            noise = rng.uniform(len(ry) * len(rx)).reshape(len(ry), len(rx))
            if matched:
                noise = (noise * np.float32(2.0 * level[g, c])).astype(np.float32)
            elif live:
                m = float(np.mean([mus[g][k] for k, (s, d) in enumerate(topo) if s == c]))
                noise = (noise * np.float32(2.0 * m)).astype(np.float32)
            A[c][np.ix_(ry, rx)] = noise
    return World(H, W, n_channels, kernels, dt, localized=localized,
                 maintain_genes=maintain, A=A, P=P, name=name)


def global_multi_channel(H=256, W=256, R=13, patch=48, seed_index=4, dt=0.2,
                         n_channels=3, name="c5") -> World:
    """Multi-channel world with global per-kernel genes (no gene maps): the
    paper's 15-kernel topology, U[0,1) noise on a central square."""
    rng = Rng(BASE_SEED + seed_index)
    topo = paper_topology(n_channels)
    kernels = []
    for (s, d) in topo:
        B = int(rng.integers(1, 1, 3)[0])
        beta = tuple(float(b) for b in rng.uniform(B))
        h = float(rng.uniform(1, 0.1, 1.0)[0])
        mu = float(rng.uniform(1, 0.10, 0.40)[0])
        sigma = float(rng.uniform(1, 0.01, 0.06)[0])
        kernels.append(KernelDesc(s, d, R, KERNEL_SHELLS, beta, h=h, mu=mu, sigma=sigma))
    A = np.zeros((n_channels, H, W), np.float32)
    y0, x0 = H // 2 - patch // 2, W // 2 - patch // 2
    for c in range(n_channels):
        A[c, y0:y0 + patch, x0:x0 + patch] = rng.uniform(patch * patch).reshape(patch, patch)
    return World(H, W, n_channels, kernels, dt, A=A, name=name)


def batched_worlds(n_worlds=256, sizes=(64, 128, 256, 512), r_range=(8, 16), n_geno=4,
                   seed_index=3, dt=0.1, live=False):
    """n_worlds independent single-channel localized-gene worlds: side drawn
    uniformly from `sizes`, radius uniformly from r_range, n_geno genotypes
    (mu ~ U[0.10, 0.40), sigma ~ U[0.01, 0.06)) on squares of side/8 (at
    least 8) as in the single-world recipe; maintenance on."""
    rng = Rng(BASE_SEED + seed_index)
    side = rng.integers(n_worlds, 0, len(sizes) - 1)
    rad = rng.integers(n_worlds, r_range[0], r_range[1])
    worlds = []
    for w in range(n_worlds):
        S = int(sizes[side[w]])
        R = int(min(rad[w], (S - 1) // 2))
        worlds.append(localized_single_channel(H=S, W=S, R=R, patch=max(8, S // 8), n_geno=n_geno,
                                               seed_index=seed_index * 100000 + w, dt=dt,
                                               name=f"batch{w}", live=live))
    return worlds


# The five workloads, full size.  Parity tests use reduced shapes of the
# same recipes; the benchmark times the 2048^2 multi-channel one.
def workload(name: str) -> World:
    if name == "c1":
        return single_kernel_global()
    if name == "c2":
        return localized_single_channel()
    if name == "c3":
        return multi_channel()
    if name == "c5":
        return global_multi_channel()
    raise KeyError(name)


def ring_world(H=512, W=1024, R=12, n_rings=24, n_channels=3, patch=96, n_geno=8, seed_index=6,
               dt=0.2, localized=LOC_MU | LOC_SIGMA | LOC_H | LOC_KERNEL, live=True, name="rings",
               matched=False) -> World:
    """The paper's configuration (Section 2.1): a 512 x 1024 torus, 3 channels,
    15 kernels in the paper's topology, each kernel two Gaussian bumps cut into
    n_rings rings of a radius-R disk (Section 2.4), every gene localized:
    growth m, s, h and kernel r1, w1, b1, r2, w2, b2 per kernel and site.
    n_geno genotypes fill square patches (as in the other worlds); per kernel
    r1 ~ U[0.1, 0.5), w1 ~ U[0.05, 0.15), b1 ~ U[0.5, 1), r2 ~ U[0.5, 0.9),
    w2 ~ U[0.05, 0.15), b2 ~ U[0.1, 0.6), m ~ U[0.1, 0.4), s ~ U[0.01, 0.06),
    h ~ U[0.1, 1).  A is U[0, 1) noise on each patch (U[0, 2 m) with live).
    matched=True redraws m and s as multi_channel(matched=True) does (a level
    L per genotype and channel, s ~ U[0.03, 0.06), m = L - 1.1774 s + U[-0.01,
    0.01)) and makes channel c's noise U[0, 2 L)."""
    rng = Rng(BASE_SEED + seed_index)
    topo = paper_topology(n_channels)
    K = len(topo)
    ranges = {"mu": (0.10, 0.40), "sigma": (0.01, 0.06), "h": (0.1, 1.0), "r1": (0.1, 0.5), "w1": (0.05, 0.15),
              "b1": (0.5, 1.0), "r2": (0.5, 0.9), "w2": (0.05, 0.15), "b2": (0.1, 0.6)}
    geno = {g: rng.uniform(n_geno * K, *ranges[g]).reshape(n_geno, K) for g in ranges}
    level = None
    if matched:
        level = rng.uniform(n_geno * n_channels, *ranges["mu"]).reshape(n_geno, n_channels)
        jitter = rng.uniform(n_geno * K, -0.01, 0.01).reshape(n_geno, K)
        src = np.array([s_ for (s_, _) in topo])
        geno["sigma"] = rng.uniform(n_geno * K, 0.03, 0.06).reshape(n_geno, K)
        geno["mu"] = (level[:, src] + jitter - np.float32(HALF_HEIGHT) * geno["sigma"]).astype(np.float32)
    kernels = []
    for k, (src, dst) in enumerate(topo):
        bump = tuple(float(np.mean(geno[g][:, k])) for g in ("r1", "w1", "b1", "r2", "w2", "b2"))
        kernels.append(KernelDesc(src, dst, R, KERNEL_BUMPS, (1.0,), bump=bump, h=float(np.mean(geno["h"][:, k])),
                                  mu=float(np.mean(geno["mu"][:, k])), sigma=float(np.mean(geno["sigma"][:, k]))))
    order = [g for g, bit in (("mu", LOC_MU), ("sigma", LOC_SIGMA), ("h", LOC_H)) if localized & bit]
    if localized & LOC_KERNEL:
        order += ["r1", "w1", "b1", "r2", "w2", "b2"]
    A = np.zeros((n_channels, H, W), np.float32)
    P = np.zeros((len(order), K, H, W), np.float32)
    for g, (ry, rx, my, mx) in enumerate(_place_patches(rng, H, W, patch, n_geno, R)):
        for p, name_ in enumerate(order):
            for k in range(K):
                P[p, k][np.ix_(my, mx)] = geno[name_][g, k]
        for c in range(n_channels):
            noise = rng.uniform(len(ry) * len(rx)).reshape(len(ry), len(rx))
            if level is not None:
                noise = (noise * np.float32(2.0 * level[g, c])).astype(np.float32)
            elif live:
                m = float(np.mean([geno["mu"][g, k] for k, (s_, d_) in enumerate(topo) if s_ == c]))
                noise = (noise * np.float32(2.0 * m)).astype(np.float32)
            A[c][np.ix_(ry, rx)] = noise
    return World(H, W, n_channels, kernels, dt, localized=localized, maintain_genes=1, A=A, P=P, name=name,
                 n_rings=n_rings)


def evolution_events(world: World, step: int, seed_index: int = 5, gamma_mut=1.0, gamma_pen=0.2,
                     mut_half=4, r_oxy=3, eps_pen=0.01, delta_scale=0.01) -> dict:
    """The random choices of one step of the evolutionary operators
    (Sections 2.5-2.6), drawn from the counter-based stream (seed, step):
    mutation plane, kernel, delta ~ U[-1, 1) * delta_scale and square centre;
    penalisation plane (mu or sigma), kernel and |delta| ~ U[0, 1) * delta_scale
    with sign +1 for mu (raise mu) and -1 for sigma (lower sigma).  The gamma,
    square half-size, r_oxy and E_pen threshold are carried along."""
    rng = Rng(BASE_SEED * 1000003 + seed_index * 7919 + step)
    n_p = max(1, world.n_planes)
    mut_p = int(rng.integers(1, 0, n_p - 1)[0])
    mut_k = int(rng.integers(1, 0, world.n_kernels - 1)[0])
    mut_delta = float(rng.uniform(1, -1.0, 1.0)[0]) * delta_scale
    y0 = int(rng.integers(1, 0, world.height - 1)[0])
    x0 = int(rng.integers(1, 0, world.width - 1)[0])
    # penalisation acts on a localized mu or sigma plane
    loc_bits = [b for b in (LOC_MU, LOC_SIGMA, LOC_H) if world.localized & b]
    pen_choices = [p for p, bit in enumerate(loc_bits) if bit in (LOC_MU, LOC_SIGMA)]
    pen_p = pen_choices[int(rng.integers(1, 0, len(pen_choices) - 1)[0])] if pen_choices else -1
    pen_k = int(rng.integers(1, 0, world.n_kernels - 1)[0])
    mag = float(rng.uniform(1)[0]) * delta_scale
    sign = 1.0 if (pen_p >= 0 and loc_bits[pen_p] == LOC_MU) else -1.0
    if world.n_planes == 0:
        mut_p = pen_p = -1
    return dict(mut_p=mut_p, mut_k=mut_k, mut_x0=x0, mut_y0=y0, mut_half=mut_half, mut_delta=mut_delta,
                pen_p=pen_p, pen_k=pen_k, pen_delta=sign * mag, gamma_mut=gamma_mut, gamma_pen=gamma_pen,
                eps_pen=eps_pen, r_oxy=r_oxy)


def wall_strip(H: int, W: int, x0: int, width: int) -> np.ndarray:
    """A vertical wall (Section 2.7): columns x0 .. x0 + width - 1, all rows."""
    w = np.zeros((H, W), np.uint8)
    w[:, x0:x0 + width] = 1
    return w


def random_field(seed: int, shape, lo=0.0, hi=1.0) -> np.ndarray:
    """Plain U[lo,hi) float32 array (for unit tests of single stages)."""
    n = int(math.prod(shape))
    return Rng(seed).uniform(n, lo, hi).reshape(shape)
