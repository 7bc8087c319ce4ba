"""Python binding of liblenia's C ABI (include/lenia.h).

Argument marshalling only: every step of the Lenia update runs in the CUDA
library.  Functions keep the C names; device pointers may be given as ints
or as CUDA tensors (their ``data_ptr()``), and ``stream`` defaults to the
current torch stream.  A non-OK status raises LeniaError with the library's
description.  If liblenia.so has not been built this module raises on use:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from . import inputs as _inputs

LENIA_OK, LENIA_EINVAL, LENIA_ENOMEM, LENIA_ECUDA, LENIA_ETIMEOUT, LENIA_ENOTSUP = range(6)
CONV_AUTO, CONV_FFT, CONV_DIRECT, CONV_DIRECT_BF16, CONV_DIRECT_BF16X3 = 0, 1, 2, 3, 4
ROUTE_STEPS, ROUTE_COOPERATIVE, ROUTE_CLUSTER = 0, 1, 2

# Every function the header declares (checked by the tests).
EXPORTS = ("lenia_init", "lenia_step", "lenia_rollout", "lenia_backward", "lenia_stats",
           "lenia_potentials", "lenia_update_from_potentials", "lenia_step_host",
           "lenia_kernel_weights", "lenia_conv_path", "lenia_rollout_route", "lenia_launches_per_step",
           "lenia_last_error", "lenia_status_string", "lenia_destroy", "lenia_profile_start",
           "lenia_profile_stop", "lenia_profile_kind_name", "lenia_stats_noalloc", "lenia_check", "lenia_set_genes", "lenia_batch_init",
           "lenia_batch_rollout", "lenia_batch_conv_path", "lenia_batch_check", "lenia_batch_destroy",
           "lenia_selftest_wait_timeout", "lenia_set_walls", "lenia_step_evolve",
           "lenia_step_host_async", "lenia_host_wait", "lenia_batch_group_of", "lenia_measure_fp32_peak",
           "lenia_debug_fail_after", "lenia_batch_epilogue_shape", "lenia_batch_set_epilogue_shape")
PROFILE_KINDS = 9


class LeniaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class LeniaConfig(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("n_channels", ctypes.c_int32), ("n_kernels", ctypes.c_int32),
                ("dt", ctypes.c_float), ("growth_form", ctypes.c_int32),
                ("localized", ctypes.c_int32), ("maintain_genes", ctypes.c_int32),
                ("eps_u", ctypes.c_float), ("eps_p", ctypes.c_float),
                ("r_diff", ctypes.c_int32), ("alpha_on", ctypes.c_int32),
                ("conv_path", ctypes.c_int32), ("max_rollout_steps", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32), ("n_rings", ctypes.c_int32)]


class LeniaKernelDesc(ctypes.Structure):
    _fields_ = [("src_channel", ctypes.c_int32), ("dst_channel", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("form", ctypes.c_int32),
                ("n_shells", ctypes.c_int32), ("beta", ctypes.c_double * 4),
                ("bump", ctypes.c_double * 6), ("h", ctypes.c_float),
                ("mu", ctypes.c_float), ("sigma", ctypes.c_float)]


class LeniaEvents(ctypes.Structure):
    _fields_ = [("mut_plane", ctypes.c_int32), ("mut_kernel", ctypes.c_int32),
                ("mut_x0", ctypes.c_int32), ("mut_y0", ctypes.c_int32), ("mut_half", ctypes.c_int32),
                ("mut_delta", ctypes.c_double), ("gamma_mut", ctypes.c_double),
                ("pen_plane", ctypes.c_int32), ("pen_kernel", ctypes.c_int32),
                ("pen_delta", ctypes.c_double), ("gamma_pen", ctypes.c_double),
                ("eps_pen", ctypes.c_double), ("r_oxy", ctypes.c_int32)]


def events_struct(ev: dict) -> LeniaEvents:
    """LeniaEvents from a dict of one step's random choices (the keys of
    inputs.evolution_events)."""
    return LeniaEvents(ev["mut_p"], ev["mut_k"], ev["mut_x0"], ev["mut_y0"], ev["mut_half"],
                       ev["mut_delta"], ev["gamma_mut"], ev["pen_p"], ev["pen_k"], ev["pen_delta"],
                       ev["gamma_pen"], ev["eps_pen"], ev["r_oxy"])


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblenia.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"liblenia.so not found at {p}: run paper_2304_05639_gb300.build.build() "
                           "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    st = ctypes.c_int
    lib.lenia_init.argtypes = [ctypes.POINTER(LeniaConfig), ctypes.POINTER(LeniaKernelDesc), vp,
                               ctypes.POINTER(vp)]
    lib.lenia_init.restype = st
    lib.lenia_step.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.lenia_step.restype = st
    lib.lenia_rollout.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp]
    lib.lenia_rollout.restype = st
    lib.lenia_backward.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp]
    lib.lenia_backward.restype = st
    lib.lenia_stats.argtypes = [vp, vp, vp, vp]
    lib.lenia_stats.restype = st
    lib.lenia_potentials.argtypes = [vp, vp, vp, vp]
    lib.lenia_potentials.restype = st
    lib.lenia_update_from_potentials.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.lenia_update_from_potentials.restype = st
    lib.lenia_step_host.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.lenia_step_host.restype = st
    lib.lenia_step_host_async.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.lenia_step_host_async.restype = st
    lib.lenia_host_wait.argtypes = [vp, vp]
    lib.lenia_host_wait.restype = st
    lib.lenia_debug_fail_after.argtypes = [ctypes.c_int32]
    lib.lenia_debug_fail_after.restype = st
    lib.lenia_kernel_weights.argtypes = [vp, ctypes.c_int32, vp]
    lib.lenia_kernel_weights.restype = st
    lib.lenia_conv_path.argtypes = [vp]
    lib.lenia_conv_path.restype = ctypes.c_int32
    lib.lenia_rollout_route.argtypes = [vp]
    lib.lenia_rollout_route.restype = ctypes.c_int32
    lib.lenia_launches_per_step.argtypes = [vp]
    lib.lenia_launches_per_step.restype = ctypes.c_int32
    lib.lenia_last_error.argtypes = [vp]
    lib.lenia_last_error.restype = ctypes.c_char_p
    lib.lenia_status_string.argtypes = [ctypes.c_int]
    lib.lenia_status_string.restype = ctypes.c_char_p
    lib.lenia_profile_start.argtypes = [vp, ctypes.c_int32]
    lib.lenia_profile_start.restype = st
    lib.lenia_profile_stop.argtypes = [vp, vp, vp]
    lib.lenia_profile_stop.restype = st
    lib.lenia_profile_kind_name.argtypes = [ctypes.c_int32]
    lib.lenia_profile_kind_name.restype = ctypes.c_char_p
    lib.lenia_stats_noalloc.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, vp]
    lib.lenia_stats_noalloc.restype = st
    lib.lenia_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.lenia_measure_fp32_peak.restype = st
    lib.lenia_batch_init.argtypes = [ctypes.c_int32, ctypes.POINTER(LeniaConfig), ctypes.POINTER(LeniaKernelDesc),
                                     ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.lenia_batch_init.restype = st
    lib.lenia_batch_rollout.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int32, vp]
    lib.lenia_batch_rollout.restype = st
    lib.lenia_batch_group_of.argtypes = [vp, ctypes.c_int32]
    lib.lenia_batch_group_of.restype = ctypes.c_int32
    lib.lenia_batch_epilogue_shape.argtypes = [vp, ctypes.c_int32, vp]
    lib.lenia_batch_epilogue_shape.restype = ctypes.c_int32
    lib.lenia_batch_set_epilogue_shape.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.lenia_batch_set_epilogue_shape.restype = st
    lib.lenia_batch_conv_path.argtypes = [vp, ctypes.c_int32]
    lib.lenia_batch_conv_path.restype = ctypes.c_int32
    lib.lenia_batch_check.argtypes = [vp, vp]
    lib.lenia_batch_check.restype = st
    lib.lenia_batch_destroy.argtypes = [vp]
    lib.lenia_batch_destroy.restype = None
    lib.lenia_selftest_wait_timeout.argtypes = [vp, ctypes.c_int32, vp]
    lib.lenia_selftest_wait_timeout.restype = st
    lib.lenia_set_genes.argtypes = [vp, vp]
    lib.lenia_set_genes.restype = st
    lib.lenia_set_walls.argtypes = [vp, vp]
    lib.lenia_set_walls.restype = st
    lib.lenia_step_evolve.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(LeniaEvents), vp, vp, vp, vp]
    lib.lenia_step_evolve.restype = st
    lib.lenia_check.argtypes = [vp, vp]
    lib.lenia_check.restype = st
    lib.lenia_destroy.argtypes = [vp]
    lib.lenia_destroy.restype = None
    if path is None:
        _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _check(ctx, status):
    if status != LENIA_OK:
        lib = load()
        msg = lib.lenia_last_error(ctx).decode() if ctx else lib.lenia_status_string(status).decode()
        raise LeniaError(status, msg or lib.lenia_status_string(status).decode())


# ------------------------------------------------------------ C-ABI mirror

def lenia_init(cfg: LeniaConfig, kernels, stream=None):
    lib = load()
    arr = (LeniaKernelDesc * len(kernels))(*kernels)
    out = ctypes.c_void_p()
    st = lib.lenia_init(ctypes.byref(cfg), arr, _stream(stream), ctypes.byref(out))
    if st != LENIA_OK:
        raise LeniaError(st, f"lenia_init: {lib.lenia_status_string(st).decode()}")
    return out.value


def lenia_step(ctx, A_in, P_in, A_out, P_out, stats_out=None, stream=None):
    _check(ctx, load().lenia_step(ctx, _ptr(A_in), _ptr(P_in), _ptr(A_out), _ptr(P_out),
                                  _ptr(stats_out), _stream(stream)))


def lenia_rollout(ctx, A, P, n_steps, stats_out=None, stream=None):
    _check(ctx, load().lenia_rollout(ctx, _ptr(A), _ptr(P), int(n_steps), _ptr(stats_out),
                                     _stream(stream)))


def lenia_backward(ctx, A0, P0, n_steps, gA_T, gA0=None, g_genes=None, stream=None):
    _check(ctx, load().lenia_backward(ctx, _ptr(A0), _ptr(P0), int(n_steps), _ptr(gA_T), _ptr(gA0),
                                      _ptr(g_genes), _stream(stream)))


def lenia_stats(ctx, A, out, stream=None):
    _check(ctx, load().lenia_stats(ctx, _ptr(A), _ptr(out), _stream(stream)))


def lenia_stats_noalloc(A, n_channels, height, width, out, stream=None):
    """lenia_stats for callers that cannot allocate device memory (static scratch)."""
    st = load().lenia_stats_noalloc(_ptr(A), int(n_channels), int(height), int(width), _ptr(out),
                                    _stream(stream))
    if st != LENIA_OK:
        raise LeniaError(st, f"lenia_stats_noalloc: {load().lenia_status_string(st).decode()}")


def lenia_measure_fp32_peak(stream=None):
    """(scalar, packed-pair) FP32 FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().lenia_measure_fp32_peak(ctypes.byref(a), ctypes.byref(b), _stream(stream))
    if st != LENIA_OK:
        raise LeniaError(st, f"lenia_measure_fp32_peak: {load().lenia_status_string(st).decode()}")
    return a.value, b.value


def lenia_batch_init(worlds, autotune: bool = True, conv_path: int = CONV_AUTO, stream=None):
    """One batch over inputs.World objects; returns the batch handle."""
    lib = load()
    cfgs, kds = [], []
    for w in worlds:
        cfg, ks = config_from_world(w, conv_path)
        cfgs.append(cfg)
        kds.extend(ks)
    ca = (LeniaConfig * len(cfgs))(*cfgs)
    ka = (LeniaKernelDesc * len(kds))(*kds)
    out = ctypes.c_void_p()
    st = lib.lenia_batch_init(len(cfgs), ca, ka, int(bool(autotune)), _stream(stream), ctypes.byref(out))
    if st != LENIA_OK:
        raise LeniaError(st, f"lenia_batch_init: {lib.lenia_status_string(st).decode()}")
    return out.value


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def lenia_batch_rollout(batch, A_list, P_list, n_steps, stream=None):
    lib = load()
    pa = _ptr_array(A_list)
    pp = _ptr_array(P_list) if P_list is not None else None
    st = lib.lenia_batch_rollout(batch, pa, pp, int(n_steps), _stream(stream))
    if st != LENIA_OK:
        raise LeniaError(st, f"lenia_batch_rollout: {lib.lenia_status_string(st).decode()}")


def lenia_batch_conv_path(batch, world: int) -> int:
    return load().lenia_batch_conv_path(batch, int(world))


def lenia_batch_group_of(batch, world: int) -> int:
    return load().lenia_batch_group_of(batch, int(world))


def lenia_batch_epilogue_shape(batch, world: int):
    """(kind, param) of world's group: (0, rows per thread) tiled, (2, rows per
    thread) tiled with four columns per thread, (1, bands per world) queued
    streaming; (-1, 0) without a group."""
    v = ctypes.c_int32(0)
    kind = load().lenia_batch_epilogue_shape(batch, int(world), ctypes.byref(v))
    return kind, v.value


def lenia_batch_set_epilogue_shape(batch, world: int, kind: int, param: int):
    st_ = load().lenia_batch_set_epilogue_shape(batch, int(world), int(kind), int(param))
    if st_ != 0:
        raise LeniaError(st_, "lenia_batch_set_epilogue_shape")


def lenia_batch_check(batch, stream=None):
    st = load().lenia_batch_check(batch, _stream(stream))
    if st != LENIA_OK:
        raise LeniaError(st, "lenia_batch_check")


def lenia_batch_destroy(batch):
    if batch:
        load().lenia_batch_destroy(batch)


def lenia_set_genes(ctx, genes):
    """genes: host array-like [K][3] of (mu, sigma, h)."""
    g = np.ascontiguousarray(np.asarray(genes, dtype=np.float32))
    _check(ctx, load().lenia_set_genes(ctx, g.ctypes.data))


def lenia_selftest_wait_timeout(ctx, limit_mcycles: int = 200, stream=None):
    _check(ctx, load().lenia_selftest_wait_timeout(ctx, int(limit_mcycles), _stream(stream)))


def lenia_debug_fail_after(n_calls: int):
    """Test hook: report the checked CUDA call after n_calls successful ones as
    failed (n_calls < 0 disarms)."""
    load().lenia_debug_fail_after(int(n_calls))


def lenia_check(ctx, stream=None):
    _check(ctx, load().lenia_check(ctx, _stream(stream)))


def lenia_potentials(ctx, A_in, U_out, stream=None):
    _check(ctx, load().lenia_potentials(ctx, _ptr(A_in), _ptr(U_out), _stream(stream)))


def lenia_update_from_potentials(ctx, A_in, P_in, U_in, A_out, P_out, alpha_out=None, stream=None):
    _check(ctx, load().lenia_update_from_potentials(ctx, _ptr(A_in), _ptr(P_in), _ptr(U_in),
                                                    _ptr(A_out), _ptr(P_out), _ptr(alpha_out),
                                                    _stream(stream)))


def lenia_set_walls(ctx, mask):
    """mask: host [H, W] array (non-zero = wall) or None to remove the walls."""
    if mask is None:
        _check(ctx, load().lenia_set_walls(ctx, None))
        return
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    _check(ctx, load().lenia_set_walls(ctx, m.ctypes.data))


def lenia_step_evolve(ctx, A, P, A_out, P_out, events, stats_out=None, alpha_out=None, epen_out=None,
                      stream=None):
    """events: a LeniaEvents or a dict with the keys of inputs.evolution_events."""
    ev = events if isinstance(events, LeniaEvents) else events_struct(events)
    _check(ctx, load().lenia_step_evolve(ctx, _ptr(A), _ptr(P), _ptr(A_out), _ptr(P_out), ctypes.byref(ev),
                                         _ptr(stats_out), _ptr(alpha_out), _ptr(epen_out), _stream(stream)))


def lenia_step_host_async(ctx, A_in, P_in, A_out, P_out, stats_out=None, stream=None):
    _check(ctx, load().lenia_step_host_async(ctx, _ptr(A_in), _ptr(P_in), _ptr(A_out), _ptr(P_out),
                                             _ptr(stats_out), _stream(stream)))


def lenia_host_wait(ctx, stream=None):
    _check(ctx, load().lenia_host_wait(ctx, _stream(stream)))


def lenia_step_host(ctx, A_in, P_in, A_out, P_out, stats_out=None, stream=None):
    _check(ctx, load().lenia_step_host(ctx, _ptr(A_in), _ptr(P_in), _ptr(A_out), _ptr(P_out),
                                       _ptr(stats_out), _stream(stream)))


def lenia_kernel_weights(ctx, k: int, radius: int) -> np.ndarray:
    out = np.zeros((2 * radius + 1, 2 * radius + 1), np.float64)
    _check(ctx, load().lenia_kernel_weights(ctx, int(k), out.ctypes.data))
    return out


def lenia_conv_path(ctx) -> int:
    return load().lenia_conv_path(ctx)


def lenia_rollout_route(ctx) -> int:
    """ROUTE_STEPS, ROUTE_COOPERATIVE or ROUTE_CLUSTER: the form of lenia_rollout."""
    return load().lenia_rollout_route(ctx)


def lenia_launches_per_step(ctx) -> int:
    return load().lenia_launches_per_step(ctx)


def lenia_profile_start(ctx, max_launches: int):
    _check(ctx, load().lenia_profile_start(ctx, int(max_launches)))


def lenia_profile_stop(ctx) -> dict:
    """{kind name: (total ms, launches)} for the kinds that launched."""
    tot = np.zeros(PROFILE_KINDS, np.float32)
    cnt = np.zeros(PROFILE_KINDS, np.int32)
    _check(ctx, load().lenia_profile_stop(ctx, tot.ctypes.data, cnt.ctypes.data))
    lib = load()
    return {lib.lenia_profile_kind_name(k).decode(): (float(tot[k]), int(cnt[k]))
            for k in range(PROFILE_KINDS) if cnt[k]}


def lenia_profile_kind_name(kind: int):
    r = load().lenia_profile_kind_name(int(kind))
    return r.decode() if r else None


def lenia_destroy(ctx):
    if ctx:
        load().lenia_destroy(ctx)


# ------------------------------------------------------ world helpers

def config_from_world(world: "_inputs.World", conv_path: int = CONV_AUTO, max_rollout_steps: int = 0,
                      ckpt_every: int = 0):
    cfg = LeniaConfig(world.height, world.width, world.n_channels, world.n_kernels,
                      float(world.dt), world.growth_form, world.localized, world.maintain_genes,
                      float(world.eps_u), float(world.eps_p), world.r_diff, world.alpha_on,
                      conv_path, max_rollout_steps, ckpt_every, int(getattr(world, "n_rings", 0)))
    ks = []
    for k in world.kernels:
        d = LeniaKernelDesc()
        d.src_channel, d.dst_channel, d.radius, d.form = k.src, k.dst, k.radius, k.form
        d.n_shells = len(k.beta)
        for i, b in enumerate(k.beta):
            d.beta[i] = b
        for i, b in enumerate(k.bump):
            d.bump[i] = b
        d.h, d.mu, d.sigma = k.h, k.mu, k.sigma
        ks.append(d)
    return cfg, ks


class Simulation:
    """A context plus device state for one world (torch tensors on cuda)."""

    def __init__(self, world, conv_path: int = CONV_AUTO, device="cuda"):
        import torch
        self.world = world
        cfg, ks = config_from_world(world, conv_path)
        self.ctx = lenia_init(cfg, ks)
        self.device = device
        self.A = torch.from_numpy(np.ascontiguousarray(world.A)).to(device)
        self.P = (torch.from_numpy(np.ascontiguousarray(world.P)).to(device)
                  if world.n_planes else None)
        self.A2 = torch.empty_like(self.A)
        self.P2 = torch.empty_like(self.P) if self.P is not None else None
        self.stats = torch.zeros((world.n_channels, 3), dtype=torch.float32, device=device)

    @property
    def conv_path(self):
        return lenia_conv_path(self.ctx)

    def step(self, with_stats=True):
        lenia_step(self.ctx, self.A, self.P, self.A2, self.P2, self.stats if with_stats else None)
        self.A, self.A2 = self.A2, self.A
        if self.P is not None:
            self.P, self.P2 = self.P2, self.P

    def potentials(self, A=None):
        import torch
        A = self.A if A is None else A
        U = torch.empty((self.world.n_kernels, self.world.height, self.world.width),
                        dtype=torch.float32, device=self.device)
        lenia_potentials(self.ctx, A, U)
        return U

    def close(self):
        if self.ctx:
            lenia_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def genes_of(world) -> np.ndarray:
    """[K][3] float32 (mu, sigma, h) of a world's kernels."""
    return np.array([[k.mu, k.sigma, k.h] for k in world.kernels], np.float32)


class LeniaRollout:
    """Differentiable n-step rollout of a world with global genes.

    ``rollout(A0, genes)`` returns A_T; gradients flow to A0 and to the
    per-kernel genes [K][3] (mu, sigma, h) through lenia_backward (the
    hand-written adjoint with checkpointed recompute)."""

    def __init__(self, world, n_steps: int, ckpt_every: int = 8, conv_path: int = CONV_AUTO):
        import torch

        cfg, ks = config_from_world(world, conv_path, max_rollout_steps=n_steps, ckpt_every=ckpt_every)
        self.ctx = lenia_init(cfg, ks)
        self.n_steps = n_steps
        self.K = world.n_kernels
        outer = self

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(fctx, A0, genes):
                lenia_set_genes(outer.ctx, genes.detach().float().cpu().numpy())
                A = A0.detach().contiguous().clone()
                lenia_rollout(outer.ctx, A, None, outer.n_steps)
                fctx.save_for_backward(A0, genes)
                return A

            @staticmethod
            def backward(fctx, gA_T):
                A0, genes = fctx.saved_tensors
                lenia_set_genes(outer.ctx, genes.detach().float().cpu().numpy())
                gA0 = torch.empty_like(A0)
                gg = torch.empty((outer.K, 3), dtype=torch.float32, device=A0.device)
                lenia_backward(outer.ctx, A0.detach().contiguous(), None, outer.n_steps,
                               gA_T.detach().float().contiguous(), gA0, gg)
                return gA0, gg.to(genes.dtype)

        self._fn = _Fn

    def __call__(self, A0, genes):
        return self._fn.apply(A0, genes)

    def close(self):
        if self.ctx:
            lenia_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
