"""Batched worlds (lenia_batch_*): a batch rollout equals per-world rollouts
on the same convolution paths (bit for bit, except that a grouped world of
width 256 k runs the tiled epilogue where a single world would run the
streaming one: those agree to rounding), and one batch step matches the FP64
oracle per world.  GPU only."""
import numpy as np
import pytest

import oracle
from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import compare_step, alpha_margin, to_dev, torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    oracle.build()
    torch_mod()


def _worlds():
    ws = inputs.batched_worlds(n_worlds=9, sizes=(64, 128, 256), r_range=(6, 12), live=True)
    # worlds sharing a shape and kernel (different genotypes and states): groups
    ws += inputs.batched_worlds(n_worlds=6, sizes=(64, 256), r_range=(9, 9), seed_index=7, live=True)
    # one non-power-of-two world (direct path only) and one multi-channel world
    ws.append(inputs.localized_single_channel(H=96, W=80, R=7, patch=16, n_geno=2, live=True, name="odd"))
    ws.append(inputs.multi_channel(H=64, W=128, R=9, patch=20, n_geno=3, live=True, name="mc"))
    return ws


@pytest.mark.parametrize("n_steps", [3, 4])
def test_batch_rollout_equals_single_world_rollouts(n_steps):
    torch = torch_mod()
    ws = _worlds()
    batch = lenia.lenia_batch_init(ws, autotune=True)
    try:
        A = [to_dev(w.A) for w in ws]
        P = [to_dev(w.P) if w.P is not None else None for w in ws]
        lenia.lenia_batch_rollout(batch, A, P, n_steps)
        lenia.lenia_batch_check(batch)
        paths = [lenia.lenia_batch_conv_path(batch, i) for i in range(len(ws))]
        assert set(paths) <= {lenia.CONV_FFT, lenia.CONV_DIRECT}
        assert paths[-2] == lenia.CONV_DIRECT        # 96 x 80 has no FFT path
        groups = [lenia.lenia_batch_group_of(batch, i) for i in range(len(ws))]
        assert max(groups) >= 1, groups             # shared shapes form groups
        for i, w in enumerate(ws):
            cfg, ks = lenia.config_from_world(w, paths[i])
            ctx = lenia.lenia_init(cfg, ks)
            try:
                a, p = to_dev(w.A), (to_dev(w.P) if w.P is not None else None)
                lenia.lenia_rollout(ctx, a, p, n_steps)
                torch.cuda.synchronize()
                if lenia.lenia_batch_group_of(batch, i) >= 0 and w.width % 256 == 0:
                    assert float((a - A[i]).abs().max()) <= 1e-5 * n_steps, w.name
                    if p is not None:
                        assert float((p - P[i]).abs().max()) <= 1e-6 * n_steps, w.name
                else:
                    assert torch.equal(a, A[i]), w.name
                    if p is not None:
                        assert torch.equal(p, P[i]), w.name
            finally:
                lenia.lenia_destroy(ctx)
        # the captured graphs are reused for the same buffers
        lenia.lenia_batch_rollout(batch, A, P, 2)
        lenia.lenia_batch_check(batch)
    finally:
        lenia.lenia_batch_destroy(batch)


def test_batch_step_matches_oracle():
    torch = torch_mod()
    ws = _worlds()[:4] + _worlds()[9:15] + _worlds()[-2:]
    batch = lenia.lenia_batch_init(ws, autotune=True)
    try:
        A = [to_dev(w.A) for w in ws]
        P = [to_dev(w.P) if w.P is not None else None for w in ws]
        lenia.lenia_batch_rollout(batch, A, P, 1)
        lenia.lenia_batch_check(batch)
        alive = 0
        for i, w in enumerate(ws):
            A1, P1, U, al = oracle.step(w, return_u=True, return_alpha=True)
            Ph = np.stack([[oracle.diffuse(w.P[p, k]) for k in range(w.n_kernels)] for p in range(w.n_planes)])
            g = {"A": A[i].cpu().numpy(), "P": P[i].cpu().numpy()}
            alive += compare_step(w, g, A1, P1, al, alpha_margin(w, U, Ph), min_alpha1=0)["alpha1"]
        print("alpha = 1 sites over the batch:", alive)
        assert alive >= 1000
    finally:
        lenia.lenia_batch_destroy(batch)


def test_grouped_worlds_match_oracle_and_single_worlds():
    """Twelve worlds of three shapes (FFT path, one radius, different
    genotypes and states) form three groups, each stepping in one launch per
    stage: one step matches the oracle per world, and three steps match
    single-world rollouts (bit for bit at widths 64 and 128)."""
    torch = torch_mod()
    ws = inputs.batched_worlds(n_worlds=12, sizes=(64, 128, 256), r_range=(9, 9), seed_index=11, live=True)
    batch = lenia.lenia_batch_init(ws, autotune=False)
    try:
        groups = [lenia.lenia_batch_group_of(batch, i) for i in range(len(ws))]
        assert all(g >= 0 for g in groups) and len(set(groups)) == len({w.height for w in ws}), groups
        A = [to_dev(w.A) for w in ws]
        P = [to_dev(w.P) for w in ws]
        lenia.lenia_batch_rollout(batch, A, P, 1)
        lenia.lenia_batch_check(batch)
        alive = 0
        for i, w in enumerate(ws):
            A1, P1, U, al = oracle.step(w, return_u=True, return_alpha=True)
            Ph = np.stack([[oracle.diffuse(w.P[p, k]) for k in range(w.n_kernels)] for p in range(w.n_planes)])
            alive += compare_step(w, {"A": A[i].cpu().numpy(), "P": P[i].cpu().numpy()}, A1, P1, al,
                                  alpha_margin(w, U, Ph), min_alpha1=0)["alpha1"]
        print("alpha = 1 sites over the batch:", alive)
        assert alive >= 1000
        lenia.lenia_batch_rollout(batch, A, P, 2)          # three steps in all
        lenia.lenia_batch_check(batch)
        for i, w in enumerate(ws):
            cfg, ks = lenia.config_from_world(w, lenia.CONV_FFT)
            ctx = lenia.lenia_init(cfg, ks)
            try:
                a, p = to_dev(w.A), to_dev(w.P)
                lenia.lenia_rollout(ctx, a, p, 3)
                torch.cuda.synchronize()
                if w.width % 256 == 0:
                    assert float((a - A[i]).abs().max()) <= 3e-5 and float((p - P[i]).abs().max()) <= 3e-6
                else:
                    assert torch.equal(a, A[i]) and torch.equal(p, P[i]), w.name
            finally:
                lenia.lenia_destroy(ctx)
    finally:
        lenia.lenia_batch_destroy(batch)


def test_full_batched_workload_sampled_worlds_match_oracle():
    """The benchmark's batched workload in its launch configuration: 256
    single-channel localized worlds, sides drawn from {64, 128, 256, 512}, radii
    8..16, autotuned paths, grouped launches.  After one batch step, a sample
    of worlds of every side - four of side 512, whose group carries most of the
    sites and runs the 512-wide grouped kernels - is compared with the oracle
    element by element."""
    ws = inputs.batched_worlds(live=True)
    batch = lenia.lenia_batch_init(ws, autotune=True)
    try:
        A = [to_dev(w.A) for w in ws]
        P = [to_dev(w.P) for w in ws]
        lenia.lenia_batch_rollout(batch, A, P, 1)
        lenia.lenia_batch_check(batch)
        by_side = {}
        for i, w in enumerate(ws):
            by_side.setdefault(w.height, []).append(i)
        assert sorted(by_side) == [64, 128, 256, 512]
        groups512 = {lenia.lenia_batch_group_of(batch, i) for i in by_side[512]}
        assert len(groups512) == 1 and -1 not in groups512, groups512      # one group of 512-side worlds
        pick = by_side[512][:4] + by_side[256][:3] + by_side[128][:2] + by_side[64][:2]
        alive = 0
        for i in pick:
            w = ws[i]
            A1, P1, U, al = oracle.step(w, return_u=True, return_alpha=True)
            Ph = np.stack([[oracle.diffuse(w.P[p, k]) for k in range(w.n_kernels)] for p in range(w.n_planes)])
            res = compare_step(w, {"A": A[i].cpu().numpy(), "P": P[i].cpu().numpy()}, A1, P1, al,
                               alpha_margin(w, U, Ph), min_alpha1=0)
            alive += res["alpha1"]
            print(w.name, w.height, "R", w.kernels[0].radius, "path", lenia.lenia_batch_conv_path(batch, i),
                  "group", lenia.lenia_batch_group_of(batch, i), res)
        assert alive >= 1000
    finally:
        lenia.lenia_batch_destroy(batch)


@pytest.mark.parametrize("kind,param", [(1, 1), (1, 3), (1, 8), (0, 1), (0, 4), (2, 1), (2, 2)])
def test_epilogue_shapes_match_oracle(kind, param):
    """Every epilogue shape the autotuner chooses from, forced on two groups
    (256- and 512-side worlds, one radius): the queued streaming kernel (one
    persistent launch over a device work queue, per-world tensor maps in
    device memory) with 1, 3 or 8 bands per world, the tiled kernel with 1 or 4
    rows per thread, and its four-columns-per-thread form with 1 or 2 rows.  One batch step against the oracle per world, and
    two steps against the tiled kernel's two steps."""
    torch = torch_mod()
    ws = inputs.batched_worlds(n_worlds=7, sizes=(256, 512), r_range=(9, 9), seed_index=21, live=True)
    sides = sorted({w.height for w in ws})
    assert sides == [256, 512]

    def run(k, prm, n):
        batch = lenia.lenia_batch_init(ws, autotune=False)
        try:
            for side in sides:
                first = next(i for i, w in enumerate(ws) if w.height == side)
                lenia.lenia_batch_set_epilogue_shape(batch, first, k, prm)
                assert lenia.lenia_batch_epilogue_shape(batch, first) == (k, prm)
            A = [to_dev(w.A) for w in ws]
            P = [to_dev(w.P) for w in ws]
            lenia.lenia_batch_rollout(batch, A, P, n)
            lenia.lenia_batch_check(batch)
            return [a.cpu().numpy() for a in A], [p.cpu().numpy() for p in P]
        finally:
            lenia.lenia_batch_destroy(batch)

    A1, P1 = run(kind, param, 1)
    alive = 0
    for i, w in enumerate(ws):
        Ar, Pr, U, al = oracle.step(w, return_u=True, return_alpha=True)
        Ph = np.stack([[oracle.diffuse(w.P[p, k]) for k in range(w.n_kernels)] for p in range(w.n_planes)])
        alive += compare_step(w, {"A": A1[i], "P": P1[i]}, Ar, Pr, al, alpha_margin(w, U, Ph), min_alpha1=0)["alpha1"]
    assert alive >= 1000
    A2, P2 = run(kind, param, 2)
    B2, Q2 = run(0, 2, 2)
    for i in range(len(ws)):
        assert np.abs(A2[i] - B2[i]).max() <= 2e-5 and np.abs(P2[i] - Q2[i]).max() <= 2e-6, i
