"""FP64 CPU oracle for the Lenia step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It is independent of the CUDA library: the C
source next to this file is compiled with gcc into its own shared library and
shares no code with the product.

Functions take numpy arrays, promote them to float64 and return float64.
Each one follows a passage of arXiv 2304.05639 (see the C source for the
formulas and the readings taken where the paper is silent).

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, special values and a
library FFT).  Multi-step chaotic rollouts beyond a few steps are only
comparable statistically.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lenia_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblenia_oracle.so")
_lock = threading.Lock()
_lib = None

LOC_MU, LOC_SIGMA, LOC_H, LOC_KERNEL = 1, 2, 4, 8


class OracleCfg(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
                ("K", ctypes.c_int), ("dt", ctypes.c_double),
                ("growth_form", ctypes.c_int), ("localized", ctypes.c_int),
                ("maintain", ctypes.c_int), ("r_diff", ctypes.c_int),
                ("alpha_on", ctypes.c_int), ("eps_u", ctypes.c_double),
                ("eps_p", ctypes.c_double), ("n_rings", ctypes.c_int)]


class OracleEvo(ctypes.Structure):
    _fields_ = [("mut_p", ctypes.c_int), ("mut_k", ctypes.c_int), ("mut_x0", ctypes.c_int),
                ("mut_y0", ctypes.c_int), ("mut_half", ctypes.c_int), ("mut_delta", ctypes.c_double),
                ("pen_p", ctypes.c_int), ("pen_k", ctypes.c_int), ("pen_delta", ctypes.c_double),
                ("gamma_mut", ctypes.c_double), ("gamma_pen", ctypes.c_double), ("eps_pen", ctypes.c_double),
                ("r_oxy", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP across output rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_kernel.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.oracle_kernel.restype = ctypes.c_int
            lib.oracle_potential.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_diffuse.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_step.argtypes = [ctypes.POINTER(OracleCfg), ip, ip, ip, dp, dp, dp, dp,
                                        ctypes.POINTER(ctypes.c_long), dp, dp, dp, dp, dp,
                                        ctypes.POINTER(ctypes.c_ubyte)]
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_update.argtypes = [ctypes.POINTER(OracleCfg), ip, dp, dp, dp, dp, dp, dp, dp, dp,
                                          ctypes.POINTER(ctypes.c_ubyte), dp]
            lib.oracle_disk_mean.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
            lib.oracle_evolve_step.argtypes = [ctypes.POINTER(OracleCfg), ip, ip, ip, dp, dp, dp, dp,
                                               ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_ubyte),
                                               ctypes.POINTER(OracleEvo), dp, dp, dp, dp,
                                               ctypes.POINTER(ctypes.c_ubyte), dp, dp]
            lib.oracle_evolve_step.restype = ctypes.c_int
            lib.oracle_update.restype = ctypes.c_int
            fp = ctypes.POINTER(ctypes.c_float)
            lib.oracle_step_sites.argtypes = [ctypes.POINTER(OracleCfg), ip, ip, ip, dp, dp, dp, dp,
                                              ctypes.POINTER(ctypes.c_long), fp, fp, ctypes.c_long,
                                              ip, ip, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_ubyte)]
            lib.oracle_step_sites.restype = ctypes.c_int
            lib.oracle_stats.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            lib.oracle_ring_counts.argtypes = [ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_ring_potentials.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
            ub = ctypes.POINTER(ctypes.c_ubyte)
            lib.oracle_ring_step.argtypes = [ctypes.POINTER(OracleCfg), ip, ip, ctypes.c_int, dp, dp, dp, dp, dp,
                                             dp, dp, dp, ub]
            lib.oracle_ring_step.restype = ctypes.c_int
            lib.oracle_ring_update.argtypes = [ctypes.POINTER(OracleCfg), ip, ip, ctypes.c_int, dp, dp, dp, dp, dp,
                                               dp, dp, dp, dp, ub, dp]
            lib.oracle_ring_update.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return _load().oracle_num_threads()


def kernel(radius: int, form: int = 0, beta=(1.0,), bump=(0.0,) * 6) -> np.ndarray:
    """Normalised kernel K~ on offsets -R..R (shape (2R+1, 2R+1))."""
    lib = _load()
    n = 2 * radius + 1
    out = np.zeros((n, n), np.float64)
    b = _f64(list(beta) + [0.0] * (4 - len(beta)))
    bu = _f64(list(bump) + [0.0] * (6 - len(bump)))
    rc = lib.oracle_kernel(radius, form, len(beta), _dp(b), _dp(bu), _dp(out))
    if rc != 0:
        raise ValueError("kernel sums to zero")
    return out


def potential(A: np.ndarray, K: np.ndarray, extended: bool = False) -> np.ndarray:
    """Periodic convolution of one plane A[H, W] with K~[(2R+1), (2R+1)]."""
    lib = _load()
    A = _f64(A)
    K = _f64(K)
    H, W = A.shape
    R = (K.shape[0] - 1) // 2
    U = np.zeros((H, W), np.float64)
    lib.oracle_potential(H, W, _dp(A), R, _dp(K), _dp(U), int(extended))
    return U


def diffuse(P: np.ndarray, r_diff: int = 1, eps_p: float = 0.0) -> np.ndarray:
    lib = _load()
    P = _f64(P)
    H, W = P.shape
    out = np.zeros((H, W), np.float64)
    lib.oracle_diffuse(H, W, _dp(P), r_diff, float(eps_p), _dp(out))
    return out


def stats(A: np.ndarray) -> np.ndarray:
    """[C, 3]: mass, circular-mean centre y, centre x of each channel."""
    lib = _load()
    A = _f64(A)
    C, H, W = A.shape
    out = np.zeros((C, 3), np.float64)
    lib.oracle_stats(C, H, W, _dp(A), _dp(out))
    return out


def world_kernels(world) -> list:
    return [kernel(k.radius, k.form, k.beta, k.bump) for k in world.kernels]


class _Args:
    """ctypes views of a world's configuration and kernels."""

    def __init__(self, world, kernels=None):
        K = world.n_kernels
        if K > 64:
            raise ValueError("oracle supports at most 64 kernels")
        ks = world_kernels(world) if kernels is None else kernels
        self.off = np.zeros(K, np.int64)
        o = 0
        for i, k in enumerate(ks):
            self.off[i] = o
            o += k.size
        self.Kw = _f64(np.concatenate([k.ravel() for k in ks]))
        self.cfg = OracleCfg(world.height, world.width, world.n_channels, K, float(world.dt),
                             world.growth_form, world.localized, world.maintain_genes, world.r_diff,
                             world.alpha_on, float(world.eps_u), float(world.eps_p),
                             int(getattr(world, "n_rings", 0)))
        ia = lambda v: np.ascontiguousarray(np.asarray(v, np.int32))
        self.src = ia([k.src for k in world.kernels])
        self.dst = ia([k.dst for k in world.kernels])
        self.rad = ia([k.radius for k in world.kernels])
        self.h = _f64([k.h for k in world.kernels])
        self.mu = _f64([k.mu for k in world.kernels])
        self.sg = _f64([k.sigma for k in world.kernels])

    def ip(self, a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))

    def kernel_args(self):
        return (ctypes.byref(self.cfg), self.ip(self.src), self.ip(self.dst), self.ip(self.rad),
                _dp(self.h), _dp(self.mu), _dp(self.sg), _dp(self.Kw),
                self.off.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))


_NULL_D = ctypes.POINTER(ctypes.c_double)()
_NULL_B = ctypes.POINTER(ctypes.c_ubyte)()


def _bp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)) if a is not None else _NULL_B


def _opt(a):
    return _dp(a) if a is not None else _NULL_D


def step(world, A=None, P=None, kernels=None, return_u=False, return_alpha=False):
    """One step of ``world`` (an inputs.World) from state (A, P), FP64.

    Returns (A_out, P_out) and, on request, U[K, H, W] and alpha[H, W]."""
    lib = _load()
    args = _Args(world, kernels)
    A = _f64(world.A if A is None else A)
    P = world.P if P is None else P
    K = world.n_kernels
    C, H, W = A.shape
    A_out = np.zeros_like(A)
    Pp = _f64(P) if (world.n_planes and P is not None) else None
    P_out = np.zeros_like(Pp) if Pp is not None else None
    U = np.zeros((K, H, W), np.float64) if return_u else None
    alpha = np.zeros((H, W), np.uint8) if return_alpha else None
    rc = lib.oracle_step(*args.kernel_args(), _dp(A), _opt(Pp), _dp(A_out), _opt(P_out), _opt(U),
                         _bp(alpha))
    if rc != 0:
        raise RuntimeError("oracle_step failed")
    out = [A_out, P_out]
    if return_u:
        out.append(U)
    if return_alpha:
        out.append(alpha)
    return tuple(out)


def update(world, A, P, U, return_alpha=False):
    """The step after the convolution from given potentials U[K, H, W]."""
    lib = _load()
    args = _Args(world)
    A = _f64(A)
    U = _f64(U)
    Pp = _f64(P) if (world.n_planes and P is not None) else None
    A_out = np.zeros_like(A)
    P_out = np.zeros_like(Pp) if Pp is not None else None
    alpha = np.zeros(A.shape[1:], np.uint8)
    rc = lib.oracle_update(ctypes.byref(args.cfg), args.ip(args.dst), _dp(args.h), _dp(args.mu),
                           _dp(args.sg), _dp(A), _opt(Pp), _dp(U), _dp(A_out), _opt(P_out), _bp(alpha),
                           _NULL_D)
    if rc != 0:
        raise RuntimeError("oracle_update failed")
    return (A_out, P_out, alpha) if return_alpha else (A_out, P_out)


def disk_mean(X, r):
    """Periodic average over the disk |d| <= r."""
    lib = _load()
    X = _f64(X)
    H, W = X.shape
    out = np.zeros((H, W))
    lib.oracle_disk_mean(H, W, _dp(X), int(r), _dp(out))
    return out


def evolve_step(world, events, walls=None, A=None, P=None, return_tsum=False):
    """One step with walls, explosion penalisation and mutation (Algorithm 2,
    Sections 2.5-2.7).  `events` holds the step's random choices (see
    inputs.evolution_events); walls is a [H, W] 0/1 array or None.
    Returns (A', P', alpha, E_pen) and, on request, sum_k t_k (the quantity
    Delta_sum(U) thresholds)."""
    lib = _load()
    args = _Args(world)
    A = _f64(world.A if A is None else A)
    P = world.P if P is None else P
    Pp = _f64(P) if (world.n_planes and P is not None) else None
    A_out = np.zeros_like(A)
    P_out = np.zeros_like(Pp) if Pp is not None else None
    H, W = A.shape[1:]
    alpha = np.zeros((H, W), np.uint8)
    epen = np.zeros((H, W))
    tsum = np.zeros((H, W))
    wl = np.ascontiguousarray(walls, np.uint8) if walls is not None else None
    ev = OracleEvo(events["mut_p"], events["mut_k"], events["mut_x0"], events["mut_y0"], events["mut_half"],
                   events["mut_delta"], events["pen_p"], events["pen_k"], events["pen_delta"],
                   events["gamma_mut"], events["gamma_pen"], events["eps_pen"], events["r_oxy"])
    rc = lib.oracle_evolve_step(*args.kernel_args(), _bp(wl), ctypes.byref(ev), _dp(A), _opt(Pp),
                                _dp(A_out), _opt(P_out), _bp(alpha), _dp(epen), _dp(tsum))
    if rc != 0:
        raise RuntimeError("oracle_evolve_step failed")
    out = (A_out, P_out, alpha, epen)
    return out + (tsum,) if return_tsum else out


def ring_counts(R: int, n: int) -> np.ndarray:
    """Pixel count of each of the n rings of a radius-R disk (Section 2.4)."""
    out = np.zeros(n)
    _load().oracle_ring_counts(int(R), int(n), _dp(out))
    return out


def ring_potentials(X, R: int, n: int) -> np.ndarray:
    """K_r * X for the n rings of a radius-R disk: [n, H, W] (Section 2.4)."""
    X = _f64(X)
    H, W = X.shape
    out = np.zeros((n, H, W))
    _load().oracle_ring_potentials(H, W, _dp(X), int(R), int(n), _dp(out))
    return out


def _ring_radius(world):
    radii = {k.radius for k in world.kernels}
    if len(radii) != 1:
        raise ValueError("ring decomposition needs one kernel radius")
    return radii.pop()


def ring_step(world, A=None, P=None, return_u=False, return_alpha=False):
    """One step of a world with ring-wise localized kernel genes (Algorithm 2
    with Section 2.4's ring decomposition).  Returns (A', P') and, on request,
    the recombined potentials U[K, H, W] and alpha[H, W]."""
    lib = _load()
    args = _Args(world)
    A = _f64(world.A if A is None else A)
    Pp = _f64(world.P if P is None else P)
    A_out, P_out = np.zeros_like(A), np.zeros_like(Pp)
    H, W = A.shape[1:]
    U = np.zeros((world.n_kernels, H, W))
    alpha = np.zeros((H, W), np.uint8)
    rc = lib.oracle_ring_step(ctypes.byref(args.cfg), args.ip(args.src), args.ip(args.dst), _ring_radius(world),
                              _dp(args.h), _dp(args.mu), _dp(args.sg), _dp(A), _dp(Pp), _dp(A_out), _dp(P_out),
                              _dp(U), _bp(alpha))
    if rc != 0:
        raise RuntimeError("oracle_ring_step failed")
    out = [A_out, P_out]
    if return_u:
        out.append(U)
    if return_alpha:
        out.append(alpha)
    return tuple(out)


def ring_update(world, A, P, V, return_alpha=False):
    """The ring step after the ring convolutions, from given ring potentials
    V[C, n_rings, H, W]."""
    lib = _load()
    args = _Args(world)
    A, Pp, V = _f64(A), _f64(P), _f64(V)
    A_out, P_out = np.zeros_like(A), np.zeros_like(Pp)
    alpha = np.zeros(A.shape[1:], np.uint8)
    rc = lib.oracle_ring_update(ctypes.byref(args.cfg), args.ip(args.src), args.ip(args.dst), _ring_radius(world),
                                _dp(args.h), _dp(args.mu), _dp(args.sg), _dp(A), _dp(Pp), _dp(V), _dp(A_out),
                                _dp(P_out), _NULL_D, _bp(alpha), _NULL_D)
    if rc != 0:
        raise RuntimeError("oracle_ring_update failed")
    return (A_out, P_out, alpha) if return_alpha else (A_out, P_out)


def step_sites(world, ys, xs, A=None, P=None):
    """The step at listed sites only (direct sums), for worlds too large for a
    full oracle step.  A and P are float32 arrays of the world's shape.
    Returns dict with A [C, n], P [n_p K, n] (or None), U [K, n], the diffused
    unmasked genes Ph [n_p K, n] (or None) and alpha [n]."""
    lib = _load()
    args = _Args(world)
    A = np.ascontiguousarray(world.A if A is None else A, dtype=np.float32)
    P = world.P if P is None else P
    ys = np.ascontiguousarray(ys, np.int32)
    xs = np.ascontiguousarray(xs, np.int32)
    n = len(ys)
    C, K = world.n_channels, world.n_kernels
    npk = world.n_planes * K
    Pf = np.ascontiguousarray(P, dtype=np.float32) if npk else None
    A_out = np.zeros((C, n))
    P_out = np.zeros((npk, n)) if npk else None
    U = np.zeros((K, n))
    Ph = np.zeros((npk, n)) if npk else None
    alpha = np.zeros(n, np.uint8)
    fptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if a is not None \
        else ctypes.POINTER(ctypes.c_float)()
    rc = lib.oracle_step_sites(*args.kernel_args(), fptr(A), fptr(Pf), n, args.ip(ys), args.ip(xs),
                               _dp(A_out), _opt(P_out), _dp(U), _opt(Ph), _bp(alpha))
    if rc != 0:
        raise RuntimeError("oracle_step_sites failed")
    return {"A": A_out, "P": P_out, "U": U, "Ph": Ph, "alpha": alpha}


def rollout(world, n_steps: int, A=None, P=None):
    """n_steps oracle steps; returns final (A, P) and per-step stats [n, C, 3]."""
    A = _f64(world.A if A is None else A)
    P = None if world.P is None and P is None else _f64(world.P if P is None else P)
    ks = world_kernels(world)
    st = []
    for _ in range(n_steps):
        A, P = step(world, A, P, kernels=ks)
        st.append(stats(A))
    return A, P, np.stack(st) if st else np.zeros((0, A.shape[0], 3))
