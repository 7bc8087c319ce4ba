"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle on the same seeded inputs."""
import numpy as np

from paper_2304_05639_gb300 import lenia

# Per-step gate on the phenospace from identical inputs (FP32 vs FP64).
TOL_STEP = 1e-5
# Potentials U = K~ * A: FP32 sums (direct) or FP32 FFTs vs FP64 direct sums.
TOL_U = 2e-6
# Diffused genes: an FP32 mean of at most (2 r + 1)^2 values in [0, 1].
TOL_P = 4e-7
# Alpha decisions closer than this to a threshold may legitimately differ
# between FP32 and FP64 (they are reported, not compared).
ALPHA_BAND = 2e-5


def torch_mod():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def to_dev(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_step(world, conv_path=lenia.CONV_AUTO, A=None, P=None, stats=False, alpha=False):
    """One step through lenia_step (or lenia_update_from_potentials for alpha)."""
    torch = torch_mod()
    cfg, ks = lenia.config_from_world(world, conv_path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A_in = to_dev(world.A if A is None else A)
        Pn = world.P if P is None else P
        P_in = to_dev(Pn) if world.n_planes else None
        A_out = torch.empty_like(A_in)
        P_out = torch.empty_like(P_in) if P_in is not None else None
        st = torch.zeros((world.n_channels, 3), dtype=torch.float32, device="cuda") if stats else None
        al = None
        if alpha:
            U = torch.empty((world.n_kernels, world.height, world.width), dtype=torch.float32, device="cuda")
            lenia.lenia_potentials(ctx, A_in, U)
            al = torch.zeros((world.height, world.width), dtype=torch.uint8, device="cuda")
            lenia.lenia_update_from_potentials(ctx, A_in, P_in, U, A_out, P_out, al)
        else:
            lenia.lenia_step(ctx, A_in, P_in, A_out, P_out, st)
        torch.cuda.synchronize()
        out = {"A": A_out.cpu().numpy(), "P": P_out.cpu().numpy() if P_out is not None else None,
               "path": lenia.lenia_conv_path(ctx)}
        if stats:
            out["stats"] = st.cpu().numpy()
        if alpha:
            out["alpha"] = al.cpu().numpy()
            out["U"] = U.cpu().numpy()
        return out
    finally:
        lenia.lenia_destroy(ctx)


def gpu_potentials(world, conv_path=lenia.CONV_AUTO, A=None):
    torch = torch_mod()
    cfg, ks = lenia.config_from_world(world, conv_path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A_in = to_dev(world.A if A is None else A)
        U = torch.empty((world.n_kernels, world.height, world.width), dtype=torch.float32, device="cuda")
        lenia.lenia_potentials(ctx, A_in, U)
        torch.cuda.synchronize()
        return U.cpu().numpy(), lenia.lenia_conv_path(ctx)
    finally:
        lenia.lenia_destroy(ctx)


def alpha_margin(world, U, Ph):
    """Smallest distance of any alpha test to its threshold at each site,
    from oracle potentials U[K, ...] and diffused genes Ph[n_p, K, ...]."""
    K = world.n_kernels
    loc = world.localized
    planes = {}
    i = 0
    for bit, name in ((1, "mu"), (2, "sigma"), (4, "h")):
        if loc & bit:
            planes[name] = Ph[i]
            i += 1
    m = np.full(U.shape[1:], np.inf)
    for k in range(K):
        kd = world.kernels[k]
        mu = planes["mu"][k] if "mu" in planes else kd.mu
        sg = planes["sigma"][k] if "sigma" in planes else kd.sigma
        h = planes["h"][k] if "h" in planes else kd.h
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            g = np.where(sg > 0, np.exp(-0.5 * ((U[k] - mu) / np.where(sg > 0, sg, 1.0)) ** 2), 0.0)
        t = U[k] if world.alpha_on else h * g
        m = np.minimum(m, np.abs(t - world.eps_u))
    return m


def compare_step(world, gpu, ref_A, ref_P, ref_alpha, margin, tol_a=TOL_STEP, min_alpha1=None):
    """Compare a GPU step with the oracle's.  Alpha must agree exactly except
    at sites whose decision lies within ALPHA_BAND of a threshold (counted;
    their number is bounded); every site where the two alphas agree is
    compared, P' within TOL_P and A' within tol_a.  With gene maintenance the
    oracle must have at least min_alpha1 sites with alpha = 1 (default 1), so
    that the alpha = 1 arithmetic is exercised, not only the masked one.
    Returns a dict of measured errors and counts."""
    C, H, W = world.A.shape
    res = {}
    if world.maintain_genes:
        amb = margin < ALPHA_BAND
        # with eps_p >= 0, alpha = 1 leaves every gene plane > 0 and alpha = 0 zeroes them all
        g_alpha = (gpu["P"].reshape(-1, H, W) != 0).all(axis=0) if gpu.get("alpha") is None \
            else gpu["alpha"].astype(bool)
        r_alpha = ref_alpha.astype(bool)
        res["alpha1"] = int(r_alpha.sum())
        need = 1 if min_alpha1 is None else min_alpha1
        assert res["alpha1"] >= need, f"only {res['alpha1']} alpha = 1 sites (need {need})"
        mism = (g_alpha != r_alpha) & ~amb
        assert mism.sum() == 0, f"alpha differs at {int(mism.sum())} unambiguous sites"
        keep = g_alpha == r_alpha
        res["ambiguous_sites"] = int(amb.sum())
        res["alpha_flips"] = int((~keep).sum())
        assert res["ambiguous_sites"] <= max(20, H * W // 100), res
        dP = np.abs(gpu["P"].reshape(-1, H, W) - ref_P.reshape(-1, H, W))[:, keep]
        res["max_dP"] = float(dP.max()) if dP.size else 0.0
        assert res["max_dP"] <= TOL_P, res
    else:
        keep = np.ones((H, W), bool)
        if ref_P is not None:
            np.testing.assert_array_equal(gpu["P"], ref_P.astype(np.float32))
    dA = np.abs(gpu["A"] - ref_A)[:, keep]
    res["max_dA"] = float(dA.max())
    assert res["max_dA"] <= tol_a, res
    return res


def disk_dilate(mask, r):
    """Sites within Euclidean distance r of a True site, on the torus."""
    out = mask.copy()
    if r <= 0 or not mask.any():
        return out
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            if dy * dy + dx * dx <= r * r:
                out |= np.roll(mask, (dy, dx), axis=(0, 1))
    return out
