"""CUDA path (through the C ABI) against the FP64 oracle, element by element,
on seeded synthetic worlds shaped like the paper's runs.  GPU only.

Tolerances (see gpu_util): potentials 2e-6; diffused genes 4e-7; the
phenospace 1e-5 per step; alpha exact except where the oracle puts a
threshold test within 2e-5 of its threshold."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import (TOL_STEP, TOL_U, alpha_margin, compare_step, disk_dilate, gpu_potentials,
                      gpu_step, to_dev, torch_mod)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


def _diffused(world, P=None):
    P = world.P if P is None else P
    if P is None:
        return None
    if not world.maintain_genes:
        return P.astype(np.float64)
    out = np.zeros(P.shape, np.float64)
    for p in range(P.shape[0]):
        for k in range(P.shape[1]):
            out[p, k] = oracle.diffuse(P[p, k], world.r_diff, world.eps_p)
    return out


def _oracle_step(world):
    A1, P1, U, al = oracle.step(world, return_u=True, return_alpha=True)
    margin = alpha_margin(world, U, _diffused(world)) if world.maintain_genes else None
    return A1, P1, U, al, margin


# ------------------------------------------------------------------ worlds

def w_c1():
    return inputs.single_kernel_global()                                   # 64^2, R=13


def w_c2_small():
    return inputs.localized_single_channel(H=128, W=128, R=12, patch=32, n_geno=4, live=True)


# The multi-channel worlds use genotypes matched to their patches
# (inputs.multi_channel(matched=True)): under the default alpha reading the
# AND over 15 kernels then holds in the patch interiors, so the alpha = 1
# arithmetic is compared, not only the masked one.
def w_c3_small():
    return inputs.multi_channel(H=128, W=128, R=18, patch=80, n_geno=2, matched=True)


def w_c3_rect():
    return inputs.multi_channel(H=64, W=256, R=9, patch=48, n_geno=3, matched=True)


def w_c5_small():
    return inputs.global_multi_channel(H=64, W=64, R=13, patch=24)


def w_ragged():
    # not a power of two: direct path; tiles of 32 leave ragged tails in y and x
    return inputs.multi_channel(H=72, W=100, R=5, patch=28, n_geno=3, matched=True)


def w_c3_wide():
    # width a multiple of 256: the streaming epilogue (bands of 1-2 rows here)
    return inputs.multi_channel(H=128, W=512, R=18, patch=96, n_geno=3, matched=True)


def w_c2_wide():
    return inputs.localized_single_channel(H=64, W=768, R=12, patch=32, n_geno=4, live=True)


def w_c5_wide():
    return inputs.global_multi_channel(H=64, W=256, R=13, patch=24)


WORLDS = {"c1": w_c1, "c2s": w_c2_small, "c3s": w_c3_small, "c3rect": w_c3_rect,
          "c5s": w_c5_small, "ragged": w_ragged, "c3w": w_c3_wide, "c2w": w_c2_wide,
          "c5w": w_c5_wide}


# ----------------------------------------------------------------- kernels

@pytest.mark.parametrize("name", ["c1", "c3s", "ragged"])
def test_kernel_weights_match_oracle(name):
    w = WORLDS[name]()
    cfg, ks = lenia.config_from_world(w)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        for k, kd in enumerate(w.kernels):
            got = lenia.lenia_kernel_weights(ctx, k, kd.radius)
            ref = oracle.kernel(kd.radius, kd.form, kd.beta, kd.bump)
            assert np.max(np.abs(got - ref)) <= 1e-15
    finally:
        lenia.lenia_destroy(ctx)


# -------------------------------------------------------------- potentials

@pytest.mark.parametrize("name,path", [("c1", 1), ("c1", 2), ("c3s", 1), ("c3s", 2), ("c3rect", 1),
                                       ("c3rect", 2), ("ragged", 2), ("c2s", 1)])
def test_potentials_parity(name, path):
    w = WORLDS[name]()
    U, used = gpu_potentials(w, path)
    assert used == path
    _, _, Uref = oracle.step(w, return_u=True)
    err = np.max(np.abs(U - Uref))
    print(f"{name} path={path} max|dU|={err:.3e}")
    assert err <= TOL_U


def test_potentials_uniform_and_impulse():
    """K~ * a = a (normalisation) and an impulse reproduces the kernel, wrapped."""
    w = inputs.single_kernel_global(H=128, W=128, R=18)
    w.A = np.full((1, 128, 128), 0.37, np.float32)
    for path in (1, 2):
        U, _ = gpu_potentials(w, path)
        assert np.max(np.abs(U - np.float32(0.37))) <= 1e-6
    A = np.zeros((1, 128, 128), np.float32)
    A[0, 2, 125] = 1.0
    K = oracle.kernel(18, 0, (1.0,))
    ref = np.zeros((128, 128))
    for dy in range(-18, 19):
        for dx in range(-18, 19):
            ref[(2 + dy) % 128, (125 + dx) % 128] = K[dy + 18, dx + 18]
    for path in (1, 2):
        U, _ = gpu_potentials(w, path, A=A)
        assert np.max(np.abs(U[0] - ref)) <= 1e-7


# ------------------------------------------- epilogue from identical inputs

@pytest.mark.parametrize("name", ["c2s", "c3s", "ragged", "c3w", "c2w"])
def test_update_from_identical_potentials(name):
    """Both sides take the same FP32 potentials: alpha and P' agree exactly up
    to rounding; A' differs only by FP32 rounding."""
    torch = torch_mod()
    w = WORLDS[name]()
    _, _, Uref = oracle.step(w, return_u=True)
    U32 = Uref.astype(np.float32)
    A_ref, P_ref, al_ref = oracle.update(w, w.A, w.P, U32.astype(np.float64), return_alpha=True)
    cfg, ks = lenia.config_from_world(w)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A_in, P_in, U_in = to_dev(w.A), to_dev(w.P), to_dev(U32)
        A_out, P_out = torch.empty_like(A_in), torch.empty_like(P_in)
        al = torch.zeros((w.height, w.width), dtype=torch.uint8, device="cuda")
        lenia.lenia_update_from_potentials(ctx, A_in, P_in, U_in, A_out, P_out, al)
        torch.cuda.synchronize()
        g = {"A": A_out.cpu().numpy(), "P": P_out.cpu().numpy(), "alpha": al.cpu().numpy()}
    finally:
        lenia.lenia_destroy(ctx)
    margin = alpha_margin(w, U32.astype(np.float64), _diffused(w))
    res = compare_step(w, g, A_ref, P_ref, al_ref, margin, tol_a=2e-6)
    print(name, res)
    assert res["alpha_flips"] <= max(2, int(1e-4 * w.sites))


# ------------------------------------------------------------ full steps

@pytest.mark.parametrize("name,path", [("c1", 1), ("c1", 2), ("c2s", 1), ("c2s", 2), ("c3s", 1),
                                       ("c3s", 2), ("c3rect", 1), ("c5s", 1), ("c5s", 2),
                                       ("ragged", 2), ("c3w", 1), ("c3w", 2), ("c2w", 2),
                                       ("c5w", 1)])
def test_step_parity(name, path):
    w = WORLDS[name]()
    A1, P1, U, al, margin = _oracle_step(w)
    g = gpu_step(w, path)
    res = compare_step(w, g, A1, P1, al, margin)
    print(name, path, res)


def _variant(**kw):
    w = inputs.multi_channel(H=64, W=64, R=7, patch=32, n_geno=2, matched=True,
                             localized=kw.pop("localized", 3))
    for k, v in kw.items():
        setattr(w, k, v)
    return w


@pytest.mark.parametrize("variant", [
    dict(growth_form=1), dict(alpha_on=1), dict(r_diff=0), dict(r_diff=2), dict(eps_p=0.02),
    dict(localized=7), dict(localized=1), dict(dt=0.0), dict(maintain_genes=0),
])
@pytest.mark.parametrize("path", [1, 2])
def test_step_variants(variant, path):
    w = _variant(**variant)
    A1, P1, U, al, margin = _oracle_step(w)
    g = gpu_step(w, path)
    res = compare_step(w, g, A1, P1, al, margin)
    print(variant, path, res)
    if variant == dict(dt=0.0):
        np.testing.assert_array_equal(g["A"], w.A)


def test_bump_kernels():
    """Section 2.4 two-bump kernels, global genes."""
    w = inputs.global_multi_channel(H=64, W=64, R=10, patch=24)
    for i, kd in enumerate(w.kernels):
        kd.form = 1
        kd.bump = (0.3 + 0.02 * i, 0.1, 1.0, 0.7, 0.08, 0.5)
    A1, P1, U, al, margin = _oracle_step(w)
    for path in (1, 2):
        compare_step(w, gpu_step(w, path), A1, P1, al, margin)


def test_empty_world_stays_empty():
    w = w_c3_small()
    w.A = np.zeros_like(w.A)
    for path in (1, 2):
        g = gpu_step(w, path)
        assert np.all(g["A"] == 0)


# ------------------------------------------------------------------ stats

def test_stats_parity():
    w = w_c3_small()
    g = gpu_step(w, 1, stats=True)
    ref = oracle.stats(g["A"])
    st = g["stats"]
    assert np.allclose(st[:, 0], ref[:, 0], rtol=2e-6, atol=1e-4)
    d = np.abs(st[:, 1:] - ref[:, 1:])
    d = np.minimum(d, np.array([w.height, w.width]) - d)        # circular distance
    assert d.max() <= 1e-3


# -------------------------------------------------------------- rollouts

@pytest.mark.parametrize("name,path", [("c1", 1), ("c1", 2), ("c5s", 1)])
def test_rollout_10_steps_global_genes(name, path):
    """10 steps within 1e-3 of the oracle (global genes: no alpha decisions)."""
    torch = torch_mod()
    w = WORLDS[name]()
    A_ref, _, st_ref = oracle.rollout(w, 10)
    cfg, ks = lenia.config_from_world(w, path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A = to_dev(w.A)
        st = torch.zeros((10, w.n_channels, 3), dtype=torch.float32, device="cuda")
        lenia.lenia_rollout(ctx, A, None, 10, st)
        torch.cuda.synchronize()
        err = np.max(np.abs(A.cpu().numpy() - A_ref))
        print(name, path, "10-step max|dA|", err)
        assert err <= 1e-3
        assert np.allclose(st.cpu().numpy()[:, :, 0], st_ref[:, :, 0], rtol=1e-4, atol=1e-2)
    finally:
        lenia.lenia_destroy(ctx)


@pytest.mark.parametrize("name,path", [("c2s", 1), ("c2s", 2), ("c2w", 2)])
def test_rollout_30_steps_localized_statistics(name, path):
    """Localized genes over 30 steps: alpha decisions near a threshold may go
    either way in FP32 and FP64, so trajectories drift apart; compared are the
    per-channel mass and circular-mean centre (the statistics the rollout
    reports), whose gap is printed against the step and bounded."""
    torch = torch_mod()
    w = WORLDS[name]()
    n = 30
    _, _, st_ref = oracle.rollout(w, n)
    cfg, ks = lenia.config_from_world(w, path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        st = torch.zeros((n, w.n_channels, 3), dtype=torch.float32, device="cuda")
        lenia.lenia_rollout(ctx, A, P, n, st)
        lenia.lenia_check(ctx)
        g = st.cpu().numpy().astype(np.float64)
    finally:
        lenia.lenia_destroy(ctx)
    mass_ref = np.maximum(st_ref[:, :, 0], 1.0)
    rel_mass = np.abs(g[:, :, 0] - st_ref[:, :, 0]) / mass_ref
    H, W = w.height, w.width
    dy = np.abs((g[:, :, 1] - st_ref[:, :, 1] + H / 2) % H - H / 2)
    dx = np.abs((g[:, :, 2] - st_ref[:, :, 2] + W / 2) % W - W / 2)
    for t in (0, 4, 9, 19, 29):
        print(f"{name} step {t + 1}: mass rel gap {rel_mass[t].max():.2e}, centre gap "
              f"{max(dy[t].max(), dx[t].max()):.2e} px")
    assert rel_mass[:10].max() <= 1e-4 and rel_mass.max() <= 1e-2, rel_mass.max(axis=1)
    assert max(dy[:10].max(), dx[:10].max()) <= 1e-2 and max(dy.max(), dx.max()) <= 0.5


def _w_c3_live_256():
    # streaming epilogue (width 256), paper topology, localized mu/sigma
    return inputs.multi_channel(H=128, W=256, R=9, patch=64, n_geno=3, matched=True, name="c3live")


@pytest.mark.parametrize("name,path", [("c2s", 1), ("c2s", 2), ("c2w", 2), ("c3live", 1)])
def test_rollout_10_steps_localized_pointwise(name, path):
    """Ten steps of a localized-gene world, compared site by site with the
    oracle's own ten steps at 1e-3 (the rollout gate), after every step.  An
    alpha decision that flips between FP32 and FP64 at step t (allowed only
    within 2e-5 of a threshold) changes that site, and its influence spreads
    by at most the kernel radius per later step; only the sites inside that
    footprint (each flip dilated by R per later step) are excluded, and their
    number is bounded.  Alpha = 1 sites are counted at every step."""
    torch = torch_mod()
    w = _w_c3_live_256() if name == "c3live" else WORLDS[name]()
    n = 10
    R = max(k.radius for k in w.kernels)
    H, W = w.height, w.width
    cfg, ks = lenia.config_from_world(w, path)
    ctx = lenia.lenia_init(cfg, ks)
    states = []
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        for _ in range(n):
            lenia.lenia_step(ctx, A, P, A2, P2)
            A, A2, P, P2 = A2, A, P2, P
            states.append((A.cpu().numpy(), P.cpu().numpy()))
        lenia.lenia_check(ctx)
    finally:
        lenia.lenia_destroy(ctx)
    rA, rP = w.A, w.P
    foot = np.zeros((H, W), bool)
    alive, flips, dA, dP = [], [], 0.0, 0.0
    for t in range(n):
        rA, rP, ral = oracle.step(w, A=rA, P=rP, return_alpha=True)
        gA, gP = states[t]
        g_alpha = (gP != 0).all(axis=0).all(axis=0)
        # footprint of earlier flips, grown by one radius per step
        foot = disk_dilate(foot, max(R, w.r_diff)) if t else foot
        f = (g_alpha != ral.astype(bool)) & ~foot
        foot |= f
        alive.append(int(ral.sum()))
        flips.append(int(f.sum()))
        keep = ~foot
        dA = max(dA, float(np.abs(gA - rA)[:, keep].max()))
        dP = max(dP, float(np.abs(gP - rP)[:, :, keep].max()))
    print(f"{name} path={path} alpha=1 per step {alive} new flips {flips} excluded {int(foot.sum())} "
          f"of {H * W}: max over steps |dA| {dA:.2e} |dP| {dP:.2e}")
    assert alive[0] >= 100
    assert foot.sum() <= H * W // 10
    assert dA <= 1e-3 and dP <= 1e-3


def test_rollout_equals_repeated_steps_and_is_deterministic():
    torch = torch_mod()
    w = w_c3_small()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        for _ in range(3):
            lenia.lenia_step(ctx, A, P, A2, P2)
            A, A2, P, P2 = A2, A, P2, P
        Ar, Pr = to_dev(w.A), to_dev(w.P)
        lenia.lenia_rollout(ctx, Ar, Pr, 3)
        torch.cuda.synchronize()
        assert torch.equal(A, Ar) and torch.equal(P, Pr)
        Ar2, Pr2 = to_dev(w.A), to_dev(w.P)
        lenia.lenia_rollout(ctx, Ar2, Pr2, 3)
        torch.cuda.synchronize()
        assert torch.equal(Ar, Ar2) and torch.equal(Pr, Pr2)
    finally:
        lenia.lenia_destroy(ctx)


def test_check_reports_ok_after_steps():
    torch = torch_mod()
    w = w_c3_wide()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        lenia.lenia_rollout(ctx, A, P, 4)
        lenia.lenia_check(ctx)                    # raises on a device-side timeout
    finally:
        lenia.lenia_destroy(ctx)


def test_bounded_wait_timeout_is_reported_and_context_survives():
    """A device wait that nothing completes gives up after its clock bound and
    surfaces as LENIA_ETIMEOUT on the host; the status clears and the context
    keeps working (no fault, no trap)."""
    torch = torch_mod()
    w = w_c3_wide()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        lenia.lenia_selftest_wait_timeout(ctx, 200)       # about 0.1 s of SM clock
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_check(ctx)
        assert e.value.status == lenia.LENIA_ETIMEOUT
        lenia.lenia_check(ctx)                            # cleared
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        lenia.lenia_step(ctx, A, P, A2, P2)
        lenia.lenia_check(ctx)
    finally:
        lenia.lenia_destroy(ctx)


def test_step_host_matches_step():
    torch = torch_mod()
    w = w_c2_small()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A_out = np.zeros_like(w.A)
        P_out = np.zeros_like(w.P)
        st = np.zeros((1, 3), np.float32)
        lenia.lenia_step_host(ctx, w.A, w.P, A_out, P_out, st)
        A_in, P_in = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A_in), torch.empty_like(P_in)
        lenia.lenia_step(ctx, A_in, P_in, A2, P2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(A_out, A2.cpu().numpy())
        np.testing.assert_array_equal(P_out, P2.cpu().numpy())
        assert st[0, 0] > 0
    finally:
        lenia.lenia_destroy(ctx)


def test_step_host_async_pipeline_matches_step():
    """Several independent host worlds enqueued back to back (uploads of one
    overlapping downloads of the previous): each output equals lenia_step of
    its own input, stats included."""
    torch = torch_mod()
    worlds = [w_c3_small(), inputs.multi_channel(H=128, W=128, R=18, patch=40, n_geno=4, seed_index=12, live=True),
              inputs.multi_channel(H=128, W=128, R=18, patch=40, n_geno=4, seed_index=13, live=True)]
    cfg, ks = lenia.config_from_world(worlds[0], lenia.CONV_FFT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        ins = [(pin(w.A), pin(w.P)) for w in worlds] * 2              # six calls, inputs reused
        outs = [(torch.empty_like(a).pin_memory(), torch.empty_like(p).pin_memory(),
                 torch.zeros((3, 3), dtype=torch.float32).pin_memory()) for (a, p) in ins]
        for (a, p), (ao, po, so) in zip(ins, outs):
            lenia.lenia_step_host_async(ctx, a, p, ao, po, so)
        lenia.lenia_host_wait(ctx)
        for j, ((a, p), (ao, po, so)) in enumerate(zip(ins, outs)):
            A_in, P_in = a.cuda(), p.cuda()
            A2, P2 = torch.empty_like(A_in), torch.empty_like(P_in)
            st = torch.zeros((3, 3), dtype=torch.float32, device="cuda")
            lenia.lenia_step(ctx, A_in, P_in, A2, P2, st)
            torch.cuda.synchronize()
            assert torch.equal(ao, A2.cpu()) and torch.equal(po, P2.cpu()), j
            assert torch.equal(so, st.cpu()), j
    finally:
        lenia.lenia_destroy(ctx)


# ------------------------------------------------------- errors and edges

def test_argument_errors():
    torch = torch_mod()
    w = w_c2_small()
    cfg, ks = lenia.config_from_world(w, 1)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_step(ctx, A, P, A, P2)                     # A_in == A_out
        assert e.value.status == lenia.LENIA_EINVAL
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_step(ctx, A, None, A2, P2)                 # genes required
        assert e.value.status == lenia.LENIA_EINVAL
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_rollout(ctx, A, P, -1)
        assert e.value.status == lenia.LENIA_EINVAL
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_backward(ctx, A, P, 4, A2, A2)
        assert e.value.status == lenia.LENIA_ENOTSUP
        lenia.lenia_rollout(ctx, A, P, 0)                          # zero steps is a no-op
    finally:
        lenia.lenia_destroy(ctx)


# ------------------------------------------------- full size, sampled sites

def _sample_sites(H, W, n, seed):
    r = inputs.Rng(seed)
    ys = list(r.integers(n, 0, H - 1)) + [0, H - 1, 0, H - 1, H // 2, 1]
    xs = list(r.integers(n, 0, W - 1)) + [0, W - 1, W - 1, 0, 0, W // 2]
    return np.array(ys), np.array(xs)


def _sampled_compare(w, path, n=400, seed=7, min_alpha1=None):
    g = gpu_step(w, path)
    ys, xs = _sample_sites(w.height, w.width, n, seed)
    # also sample inside patches (where genes live)
    if w.P is not None:
        nz = np.argwhere(w.P[0, 0] != 0)
        if len(nz):
            pick = nz[inputs.Rng(seed + 1).integers(min(n, len(nz)), 0, len(nz) - 1)]
            ys = np.concatenate([ys, pick[:, 0]])
            xs = np.concatenate([xs, pick[:, 1]])
    r = oracle.step_sites(w, ys, xs)
    sub = {"A": g["A"][:, ys, xs][:, None, :], "P": g["P"][:, :, ys, xs][:, :, None, :] if g["P"] is not None else None}
    sw = inputs.World(1, len(ys), w.n_channels, w.kernels, w.dt, w.growth_form, w.localized,
                      w.maintain_genes, w.eps_u, w.eps_p, w.r_diff, w.alpha_on,
                      A=w.A[:, ys, xs][:, None, :])
    margin = None
    refP = None
    if w.maintain_genes:
        Ph = r["Ph"].reshape(w.n_planes, w.n_kernels, 1, -1)
        margin = alpha_margin(sw, r["U"][:, None, :], Ph)
        refP = r["P"].reshape(w.n_planes, w.n_kernels, 1, -1)
    elif r["P"] is not None:
        refP = r["P"].reshape(w.n_planes, w.n_kernels, 1, -1)
    res = compare_step(sw, sub, r["A"][:, None, :], refP, r["alpha"][None, :], margin, min_alpha1=min_alpha1)
    print(w.name, path, res)
    return res


@pytest.mark.slow
def test_full_size_headline_sampled():
    """2048^2, 3 channels, 15 kernels R=18, localized mu/sigma with genotypes
    matched to their patches: the benchmark's workload and launch
    configuration (FFT path, streaming epilogue), checked at sampled sites,
    at least 100 of them with alpha = 1 (the patch interiors)."""
    w = inputs.multi_channel(matched=True)
    res = _sampled_compare(w, 1)
    assert res["alpha1"] >= 100, res


@pytest.mark.slow
def test_full_size_headline_unmatched_sampled():
    """The same shapes with independently drawn genotypes (most sites fail
    some kernel's growth test: the masked branch at full size)."""
    w = inputs.multi_channel()
    _sampled_compare(w, 1, min_alpha1=0)


@pytest.mark.slow
def test_full_size_localized_1024_sampled():
    _sampled_compare(inputs.localized_single_channel(), 1)


@pytest.mark.slow
def test_max_fft_size_4096_sampled():
    w = inputs.localized_single_channel(H=4096, W=4096, R=12, patch=256, n_geno=8)
    _sampled_compare(w, 1, n=200)


@pytest.mark.slow
def test_tall_multichannel_4096_columns_sampled():
    """4096 x 256, 3 channels, 15 kernels: 4096-point column transforms with five
    kernels per channel (eight warps per column block, two TMEM column ranges),
    checked at sampled sites, plus a 4-step rollout equal to repeated steps."""
    torch = torch_mod()
    w = inputs.multi_channel(H=4096, W=256, R=18, patch=96, n_geno=4, seed_index=14, matched=True, name="tall")
    _sampled_compare(w, 1, n=300)
    cfg, ks = lenia.config_from_world(w, lenia.CONV_FFT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        a, p = A.clone(), P.clone()
        lenia.lenia_rollout(ctx, a, p, 4)
        for _ in range(4):
            A2, P2 = torch.empty_like(A), torch.empty_like(P)
            lenia.lenia_step(ctx, A, P, A2, P2)
            A, P = A2, P2
        torch.cuda.synchronize()
        assert torch.equal(a, A) and torch.equal(p, P)
    finally:
        lenia.lenia_destroy(ctx)

