"""The evolutionary lines of Algorithm 2 on the GPU (lenia_set_walls,
lenia_step_evolve) against the FP64 oracle's evolve_step: walls (Section
2.7), the penalising area E_pen (Section 2.6), mutation (Section 2.5) and
penalisation (Section 2.6).  GPU only.

E_pen is an average of averages of 0/1 values, so both sides get it exactly
(the GPU from integer counts) wherever the Delta_sum decisions it depends on
agree.  A Delta_sum decision within TSUM_BAND of eps_u may differ between
FP32 and FP64; sites within 2 r_oxy (Chebyshev) of such a decision are set
aside, like sites whose alpha test lies within ALPHA_BAND of its threshold."""
import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import ALPHA_BAND, TOL_P, TOL_STEP, alpha_margin, to_dev, torch_mod

pytestmark = pytest.mark.gpu

TSUM_BAND = 5e-5
GAUSS_CIRCLE = {1: 5, 2: 13, 3: 29, 4: 49, 5: 81, 8: 197, 10: 317, 32: 3209}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


def w_loc1():
    w = inputs.localized_single_channel(H=64, W=80, R=6, patch=20, n_geno=3, seed_index=3, live=True)
    w.eps_u = 1e-3
    return w


def _potential_alpha(w):
    # with 15 kernels the growth test of every kernel rarely passes at once on
    # noise; the potential test (alpha_on) gives the bodies an alpha mask
    w.alpha_on = 1
    return w


def w_c3s():
    return _potential_alpha(inputs.multi_channel(H=128, W=128, R=12, patch=40, n_geno=4, live=True))


def w_c3w():
    # width a multiple of 256: the streaming epilogue writes alpha and Delta_sum
    return _potential_alpha(inputs.multi_channel(H=128, W=512, R=18, patch=40, n_geno=4, live=True))


def w_c2w():
    return inputs.localized_single_channel(H=64, W=768, R=12, patch=32, n_geno=4, live=True)


def w_ragged():
    return _potential_alpha(inputs.multi_channel(H=72, W=100, R=5, patch=20, n_geno=3, live=True))


WORLDS = {"loc1": w_loc1, "c3s": w_c3s, "c3w": w_c3w, "c2w": w_c2w, "ragged": w_ragged}


def _diffused(world, P):
    out = np.zeros(P.shape, np.float64)
    for p in range(P.shape[0]):
        for k in range(P.shape[1]):
            out[p, k] = oracle.diffuse(P[p, k], world.r_diff, world.eps_p)
    return out


def _dilate(mask, d):
    """Chebyshev dilation by d on the torus."""
    out = mask.copy()
    for dy in range(-d, d + 1):
        for dx in range(-d, d + 1):
            out |= np.roll(np.roll(mask, dy, 0), dx, 1)
    return out


def gpu_evolve(world, ev, walls=None, conv_path=lenia.CONV_AUTO, stats=False):
    torch = torch_mod()
    cfg, ks = lenia.config_from_world(world, conv_path)
    ctx = lenia.lenia_init(cfg, ks)
    H, W = world.height, world.width
    try:
        if walls is not None:
            lenia.lenia_set_walls(ctx, walls)
        A = to_dev(world.A)
        P = to_dev(world.P) if world.n_planes else None
        A2 = torch.empty_like(A)
        P2 = torch.empty_like(P) if P is not None else None
        al = torch.full((H, W), 7, dtype=torch.uint8, device="cuda")
        ep = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
        st = torch.zeros((world.n_channels, 3), dtype=torch.float32, device="cuda") if stats else None
        lenia.lenia_step_evolve(ctx, A, P, A2, P2, ev, st, al, ep)
        lenia.lenia_check(ctx)
        out = {"A": A2.cpu().numpy(), "P": P2.cpu().numpy() if P2 is not None else None,
               "alpha": al.cpu().numpy(), "epen": ep.cpu().numpy(), "A_in": A.cpu().numpy(),
               "P_in": P.cpu().numpy() if P is not None else None, "path": lenia.lenia_conv_path(ctx)}
        if stats:
            out["stats"] = st.cpu().numpy()
        return out
    finally:
        lenia.lenia_destroy(ctx)


def _events_for(world, walls, r_oxy, seed_step=0):
    """Seeded events with the mutation square centred on an alpha site and a
    penalising threshold that splits the alpha sites (and is no multiple of
    1 / n^2, so no E_pen value sits on it)."""
    ev = inputs.evolution_events(world, seed_step, gamma_mut=2.0, gamma_pen=0.5, mut_half=6, r_oxy=r_oxy)
    _, _, al, epen = oracle.evolve_step(world, ev, walls=walls)
    ys, xs = np.nonzero(al)
    if len(ys):
        j = len(ys) // 2
        ev["mut_y0"], ev["mut_x0"] = int(ys[j]), int(xs[j])
        n2 = GAUSS_CIRCLE[r_oxy] ** 2
        vals = np.unique(epen[al.astype(bool)])
        lo = float(np.median(epen[al.astype(bool)]))
        if len(vals) > 1 and lo >= vals[-1]:
            lo = float(vals[-2])
        ev["eps_pen"] = (np.floor(lo * n2 + 1e-6) + 0.5) / n2
    return ev


def _oracle_reference(world, ev, walls):
    A1, P1, al, epen, tsum = oracle.evolve_step(world, ev, walls=walls, return_tsum=True)
    keep = 1.0 if walls is None else (1 - walls).astype(np.float64)
    Aw = world.A * keep
    Pw = world.P * keep if world.n_planes else None
    _, _, U = oracle.step(world, A=Aw, P=Pw, return_u=True)
    margin = alpha_margin(world, U, _diffused(world, Pw)) if world.maintain_genes else None
    return A1, P1, al, epen, tsum, margin


def _compare(world, ev, walls, g, ref):
    A1, P1, al, epen, tsum, margin = ref
    H, W = world.height, world.width
    r = ev["r_oxy"]
    amb_a = margin < ALPHA_BAND if margin is not None else np.zeros((H, W), bool)
    amb_t = np.abs(tsum - world.eps_u) < TSUM_BAND
    unsure = _dilate(amb_t, 2 * r)
    # alpha: exact where unambiguous
    ga = g["alpha"].astype(bool)
    assert set(np.unique(g["alpha"])) <= {0, 1}
    assert ((ga != al.astype(bool)) & ~amb_a).sum() == 0
    keep = ~amb_a & (ga == al.astype(bool))
    # E_pen: exact rational values wherever the empty decisions agree
    n2 = GAUSS_CIRCLE[r] ** 2
    ge = g["epen"].astype(np.float64)
    tol = n2 * 2.0 ** -23                    # an FP32 value <= 1 times n^2
    if tol < 0.2:
        assert np.all(np.abs(ge * n2 - np.round(ge * n2)) < tol)
    dE = np.abs(ge - epen)[~unsure]
    assert dE.max() <= 1e-7, dE.max()
    # phenospace
    dA = np.abs(g["A"] - A1)[:, keep]
    assert dA.max() <= TOL_STEP, dA.max()
    res = {"ambiguous_alpha": int(amb_a.sum()), "unsure_epen": int(unsure.sum()), "max_dA": float(dA.max()),
           "max_dE": float(dE.max())}
    if world.n_planes:
        K = world.n_kernels
        Pg = g["P"].reshape(-1, H, W)
        Pr = P1.reshape(-1, H, W)
        ok = np.broadcast_to(keep, Pg.shape).copy()
        if ev["pen_p"] >= 0:
            ok[ev["pen_p"] * K + ev["pen_k"]] &= ~unsure
        dP = np.abs(Pg - Pr)[ok]
        res["max_dP"] = float(dP.max())
        assert res["max_dP"] <= TOL_P + 1e-7, res
    return res


@pytest.mark.parametrize("name,r_oxy,with_walls", [("loc1", 3, True), ("loc1", 1, False), ("c3s", 4, True),
                                                   ("c3w", 10, True), ("c2w", 8, False), ("ragged", 2, True),
                                                   ("c3w", 32, False)])
def test_evolve_step_matches_oracle(name, r_oxy, with_walls):
    w = WORLDS[name]()
    walls = inputs.wall_strip(w.height, w.width, w.width // 3, 5) if with_walls else None
    ev = _events_for(w, walls, r_oxy)
    ref = _oracle_reference(w, ev, walls)
    A1, P1, al, epen, tsum, margin = ref
    a = al.astype(bool)
    K = w.n_kernels
    # the operators must act somewhere for the comparison to mean anything
    s = ev["mut_half"]
    sq = np.zeros(a.shape, bool)
    sq[np.ix_(np.arange(ev["mut_y0"] - s, ev["mut_y0"] + s) % w.height,
              np.arange(ev["mut_x0"] - s, ev["mut_x0"] + s) % w.width)] = True
    assert (sq & a).any() and ((epen > ev["eps_pen"]) & a).any() and ((epen <= ev["eps_pen"]) & a).any()
    g = gpu_evolve(w, ev, walls)
    res = _compare(w, ev, walls, g, ref)
    print(name, r_oxy, with_walls, "path", g["path"], res)
    # the walls were removed from the caller's state, in place, and nothing else changed
    if walls is not None:
        wb = walls.astype(bool)
        assert np.all(g["A_in"][:, wb] == 0) and np.all(g["P_in"][..., wb] == 0)
        np.testing.assert_array_equal(g["A_in"][:, ~wb], w.A[:, ~wb])
        np.testing.assert_array_equal(g["P_in"][..., ~wb], w.P[..., ~wb])


def test_evolve_global_genes_walls_only():
    """Without gene maps the operators are off; walls and E_pen still apply."""
    w = inputs.global_multi_channel(H=64, W=64, R=13, patch=24)
    walls = inputs.wall_strip(64, 64, 40, 4)
    ev = inputs.evolution_events(w, 0, r_oxy=3)
    assert ev["mut_p"] == -1 and ev["pen_p"] == -1
    ref = _oracle_reference(w, ev, walls)
    g = gpu_evolve(w, ev, walls)
    res = _compare(w, ev, walls, g, ref)
    assert np.all(g["alpha"] == 1)
    print(res)


def test_evolve_without_operators_is_lenia_step_bit_for_bit():
    """gamma = 0 and no walls: the same launches as lenia_step plus the two
    disk passes, so A' and P' are identical to lenia_step's."""
    torch = torch_mod()
    for w in (w_c3w(), w_loc1()):
        ev = inputs.evolution_events(w, 3, gamma_mut=0.0, gamma_pen=0.0)
        g = gpu_evolve(w, ev)
        cfg, ks = lenia.config_from_world(w, lenia.CONV_AUTO)
        ctx = lenia.lenia_init(cfg, ks)
        try:
            A = to_dev(w.A)
            P = to_dev(w.P)
            A2, P2 = torch.empty_like(A), torch.empty_like(P)
            lenia.lenia_step(ctx, A, P, A2, P2)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(g["A"], A2.cpu().numpy())
            np.testing.assert_array_equal(g["P"], P2.cpu().numpy())
        finally:
            lenia.lenia_destroy(ctx)


def test_evolve_rollout_is_deterministic_and_keeps_walls_clear():
    """Eight seeded evolution steps twice: identical results; after every step
    the state the next step reads has no material inside the walls."""
    torch = torch_mod()
    w = w_c3w()
    walls = inputs.wall_strip(w.height, w.width, 200, 8)
    wb = torch.from_numpy(walls.astype(bool)).cuda()
    finals = []
    for _ in range(2):
        cfg, ks = lenia.config_from_world(w, lenia.CONV_AUTO)
        ctx = lenia.lenia_init(cfg, ks)
        try:
            lenia.lenia_set_walls(ctx, walls)
            A, P = to_dev(w.A), to_dev(w.P)
            A2, P2 = torch.empty_like(A), torch.empty_like(P)
            st = torch.zeros((8, w.n_channels, 3), dtype=torch.float32, device="cuda")
            for s in range(8):
                ev = inputs.evolution_events(w, s, gamma_mut=5.0, gamma_pen=0.2, r_oxy=4)
                lenia.lenia_step_evolve(ctx, A, P, A2, P2, ev, st[s])
                assert bool((A[:, wb] == 0).all()) and bool((P[..., wb] == 0).all())
                A, A2, P, P2 = A2, A, P2, P
            lenia.lenia_check(ctx)
            finals.append((A.cpu().numpy(), P.cpu().numpy(), st.cpu().numpy()))
        finally:
            lenia.lenia_destroy(ctx)
    for a, b in zip(finals[0], finals[1]):
        np.testing.assert_array_equal(a, b)
    assert np.all(np.isfinite(finals[0][0])) and np.all(np.isfinite(finals[0][2]))
    assert finals[0][2][0, :, 0].min() > 0          # mass after the first step


def test_evolve_argument_errors():
    torch = torch_mod()
    w = w_loc1()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_AUTO)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        base = inputs.evolution_events(w, 0)
        for bad in ({"r_oxy": 0}, {"r_oxy": 33}, {"mut_p": 2}, {"pen_p": -2}, {"mut_k": 1},
                    {"mut_half": 33}, {"mut_x0": 80}, {"mut_y0": -1}, {"eps_pen": float("nan")},
                    {"gamma_mut": float("inf")}):
            ev = dict(base, **bad)
            with pytest.raises(lenia.LeniaError) as e:
                lenia.lenia_step_evolve(ctx, A, P, A2, P2, ev)
            assert e.value.status == lenia.LENIA_EINVAL, bad
        with pytest.raises(lenia.LeniaError):
            lenia.lenia_step_evolve(ctx, A, P, A, P2, base)          # A and A_out overlap
        lenia.lenia_set_walls(ctx, np.zeros((64, 80), np.uint8))   # no wall sites: fine
        lenia.lenia_set_walls(ctx, None)
        lenia.lenia_step_evolve(ctx, A, P, A2, P2, base)
        lenia.lenia_check(ctx)
    finally:
        lenia.lenia_destroy(ctx)
    g = inputs.global_multi_channel(H=64, W=64, R=13, patch=24)
    cfg, ks = lenia.config_from_world(g, lenia.CONV_AUTO)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A = to_dev(g.A)
        A2 = torch.empty_like(A)
        ev = dict(inputs.evolution_events(w, 0), mut_p=0)
        with pytest.raises(lenia.LeniaError) as e:
            lenia.lenia_step_evolve(ctx, A, None, A2, None, ev)         # no gene planes to mutate
        assert e.value.status == lenia.LENIA_EINVAL
    finally:
        lenia.lenia_destroy(ctx)


@pytest.mark.parametrize("r", [4, 10])
def test_full_size_evolve_properties_and_sampled_epen(r):
    """The 2048 x 2048, 3-channel, 15-kernel world: the evolution step adds
    exactly gamma delta on (square AND alpha) and on (E_pen > eps_pen AND
    alpha) to lenia_step's genes, leaves A' unchanged, and E_pen at sampled
    sites equals the value rebuilt from the oracle's per-site potentials over
    the sites' 2 r_oxy neighbourhoods."""
    torch = torch_mod()
    w = _potential_alpha(inputs.multi_channel(live=True))
    H, W, K = w.height, w.width, w.n_kernels
    # r = 4 runs the compile-time-radius disk kernel (with tiles of one value
    # inside the bodies and in the empty background), r = 10 the general one
    # the first site (stride 16) whose 200 x 200 window is all matter, and the
    # left ends of the matter on rows through it (a body's edge)
    S = (w.A[0] > 0).astype(np.int64).cumsum(0).cumsum(1)
    h = 100
    centre = next((y, x) for y in range(h, H - h, 16) for x in range(h, W - h, 16)
                  if S[y + h - 1, x + h - 1] - S[y - h - 1, x + h - 1] - S[y + h - 1, x - h - 1]
                  + S[y - h - 1, x - h - 1] == (2 * h) ** 2)
    edges = [(y, int(np.nonzero(w.A[0][y])[0].min())) for y in (centre[0] - 60, centre[0], centre[0] + 37)]
    # alpha (the potential test) covers the bodies' interiors, which lie deep in
    # the non-empty area: a threshold just below 1 leaves the sites within
    # 2 r_oxy of empty space unpenalised
    ev = inputs.evolution_events(w, 11, gamma_mut=5.0, gamma_pen=0.2, mut_half=16, r_oxy=r, eps_pen=0.999)
    ev["mut_y0"], ev["mut_x0"] = centre
    cfg, ks = lenia.config_from_world(w, lenia.CONV_AUTO)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        A3, P3 = torch.empty_like(A), torch.empty_like(P)
        al = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        ep = torch.empty((H, W), dtype=torch.float32, device="cuda")
        lenia.lenia_step(ctx, A, P, A3, P3)
        lenia.lenia_step_evolve(ctx, A, P, A2, P2, ev, None, al, ep)
        lenia.lenia_check(ctx)
        assert torch.equal(A2, A3)
        a = al.bool()
        yy = torch.arange(H, device="cuda")[:, None]
        xx = torch.arange(W, device="cuda")[None, :]
        s = ev["mut_half"]
        sq = (((yy - ev["mut_y0"] + s) % H) < 2 * s) & (((xx - ev["mut_x0"] + s) % W) < 2 * s)
        mut_add = float(np.float32(ev["gamma_mut"] * ev["mut_delta"]))
        pen_add = float(np.float32(ev["gamma_pen"] * ev["pen_delta"]))
        n2 = GAUSS_CIRCLE[r] ** 2
        pen = ep.double() * n2 > np.floor(ev["eps_pen"] * n2) + 0.5
        diff = (P2 - P3).reshape(-1, H, W)
        mp = ev["mut_p"] * K + ev["mut_k"]
        pp = ev["pen_p"] * K + ev["pen_k"]
        expect = torch.zeros_like(diff)
        expect[mp] += torch.where(sq & a, mut_add, 0.0)
        expect[pp] += torch.where(pen & a, pen_add, 0.0)
        assert float((diff - expect).abs().max()) <= 2e-7
        counts = (int((sq & a).sum()), int((pen & a).sum()), int((~pen & a).sum()))
        print("mutated, penalised, unpenalised alpha sites:", counts)
        assert min(counts) > 0, counts
        epen = ep.cpu().numpy()
    finally:
        lenia.lenia_destroy(ctx)
    # sampled E_pen: oracle potentials on each site's (4r+1)^2 neighbourhood
    rng = inputs.Rng(4242)
    centres = [centre] + [(y, (x + k) % W) for (y, x) in edges for k in (-10, -4)] + \
        [tuple(int(v) for v in rng.integers(2, 0, 2047))]
    d = np.arange(-2 * r, 2 * r + 1)
    D = (d[:, None] ** 2 + d[None, :] ** 2 <= r * r)[r:3 * r + 1, r:3 * r + 1]
    n = int(D.sum())
    checked, partial = 0, 0
    for (cy, cx) in centres:
        yy = (cy + d[:, None] + 0 * d[None, :]) % H
        xx = (cx + 0 * d[:, None] + d[None, :]) % W
        out = oracle.step_sites(w, yy.ravel(), xx.ravel())
        t = out["U"].sum(0).reshape(len(d), len(d))   # alpha_on: the tests are the potentials
        empty = (~(t > w.eps_u)).astype(np.float64)
        # a decision within TSUM_BAND of eps_u may go either way in FP32: the
        # GPU value must be one of the values its possible outcomes give
        amb = np.argwhere(np.abs(t - w.eps_u) < TSUM_BAND)
        if len(amb) > 4:
            continue
        refs = []
        for bits in range(1 << len(amb)):
            e = empty.copy()
            for j, (y, x) in enumerate(amb):
                if bits >> j & 1:
                    e[y, x] = 1.0 - e[y, x]
            e_oxy = np.zeros((2 * r + 1, 2 * r + 1))
            for y in range(2 * r + 1):
                for x in range(2 * r + 1):
                    e_oxy[y, x] = (e[y:y + 2 * r + 1, x:x + 2 * r + 1] * D).sum() / n
            refs.append(((1 - e_oxy) * D).sum() / n)
        refs = np.array(refs)
        assert np.min(np.abs(epen[cy, cx] - refs)) <= 1e-7, (cy, cx, epen[cy, cx], refs)
        checked += 1
        partial += bool(np.all((refs > 0) & (refs < 1)))
    print("sampled E_pen sites checked:", checked, "with 0 < E_pen < 1:", partial)
    assert checked >= 3 and partial >= 1
