"""Error paths without a GPU fault: the library's failure-injection hook
(lenia_debug_fail_after) makes one checked CUDA call report a failure after
it has run.  The entry point in progress must return LENIA_ECUDA (the
message says it was injected), and the same context must keep working:
the next calls reproduce the results of an untouched run.  GPU only (the
entry points need a device), but nothing on the device fails."""
import numpy as np
import pytest

from paper_2304_05639_gb300 import build, inputs, lenia
from gpu_util import to_dev, torch_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    torch_mod()
    yield
    lenia.lenia_debug_fail_after(-1)


def _world():
    return inputs.multi_channel(H=64, W=256, R=9, patch=48, n_geno=3, matched=True)


def _expect_injected(fn):
    with pytest.raises(lenia.LeniaError) as e:
        fn()
    assert e.value.status == lenia.LENIA_ECUDA
    assert "injected" in str(e.value)


@pytest.mark.parametrize("path", [lenia.CONV_FFT, lenia.CONV_DIRECT])
def test_step_reports_injected_failure_and_recovers(path):
    torch = torch_mod()
    w = _world()
    cfg, ks = lenia.config_from_world(w, path)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        A2, P2 = torch.empty_like(A), torch.empty_like(P)
        lenia.lenia_step(ctx, A, P, A2, P2)
        torch.cuda.synchronize()
        ref_A, ref_P = A2.clone(), P2.clone()
        n_calls = lenia.lenia_launches_per_step(ctx)
        for k in range(n_calls):                       # fail at every launch of the step in turn
            lenia.lenia_debug_fail_after(k)
            _expect_injected(lambda: lenia.lenia_step(ctx, A, P, A2, P2))
            lenia.lenia_check(ctx)                      # nothing failed on the device
            A2.zero_(), P2.zero_()
            lenia.lenia_step(ctx, A, P, A2, P2)
            torch.cuda.synchronize()
            assert torch.equal(A2, ref_A) and torch.equal(P2, ref_P), k
    finally:
        lenia.lenia_debug_fail_after(-1)
        lenia.lenia_destroy(ctx)


def test_rollout_reports_injected_failure_and_recovers():
    torch = torch_mod()
    w = _world()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_FFT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A, P = to_dev(w.A), to_dev(w.P)
        st = torch.zeros((5, 3, 3), device="cuda")
        lenia.lenia_rollout(ctx, A, P, 5, st)
        torch.cuda.synchronize()
        ref = (A.clone(), P.clone(), st.clone())
        # with per-step statistics every step launches directly: the error surfaces
        lenia.lenia_debug_fail_after(7)
        A, P = to_dev(w.A), to_dev(w.P)
        _expect_injected(lambda: lenia.lenia_rollout(ctx, A, P, 5, st))
        lenia.lenia_check(ctx)
        A, P = to_dev(w.A), to_dev(w.P)
        lenia.lenia_rollout(ctx, A, P, 5, st)
        torch.cuda.synchronize()
        assert torch.equal(A, ref[0]) and torch.equal(P, ref[1]) and torch.equal(st, ref[2])
        # without statistics pairs of steps replay a captured graph; a failure
        # during the capture falls back to direct launches, which succeed
        A, P = to_dev(w.A), to_dev(w.P)
        lenia.lenia_rollout(ctx, A, P, 6)
        torch.cuda.synchronize()
        ref6 = (A.clone(), P.clone())
        ctx2 = lenia.lenia_init(cfg, ks)
        try:
            lenia.lenia_debug_fail_after(1)
            A, P = to_dev(w.A), to_dev(w.P)
            lenia.lenia_rollout(ctx2, A, P, 6)
            torch.cuda.synchronize()
            assert torch.equal(A, ref6[0]) and torch.equal(P, ref6[1])
        finally:
            lenia.lenia_destroy(ctx2)
    finally:
        lenia.lenia_debug_fail_after(-1)
        lenia.lenia_destroy(ctx)


def test_host_step_reports_injected_failure_and_recovers():
    w = _world()
    cfg, ks = lenia.config_from_world(w, lenia.CONV_FFT)
    ctx = lenia.lenia_init(cfg, ks)
    try:
        A_ref, P_ref = np.zeros_like(w.A), np.zeros_like(w.P)
        st_ref = np.zeros((3, 3), np.float32)
        lenia.lenia_step_host(ctx, w.A, w.P, A_ref, P_ref, st_ref)
        for k in range(12):                 # uploads, the step's launches, downloads, waits
            lenia.lenia_debug_fail_after(k)
            A_out, P_out = np.zeros_like(w.A), np.zeros_like(w.P)
            st = np.zeros((3, 3), np.float32)
            try:
                lenia.lenia_step_host(ctx, w.A, w.P, A_out, P_out, st)
                injected = False
            except lenia.LeniaError as e:
                assert e.status == lenia.LENIA_ECUDA and "injected" in str(e)
                injected = True
            lenia.lenia_debug_fail_after(-1)
            lenia.lenia_step_host(ctx, w.A, w.P, A_out, P_out, st)
            np.testing.assert_array_equal(A_out, A_ref)
            np.testing.assert_array_equal(P_out, P_ref)
            np.testing.assert_array_equal(st, st_ref)
            if k == 0:
                assert injected
    finally:
        lenia.lenia_debug_fail_after(-1)
        lenia.lenia_destroy(ctx)
