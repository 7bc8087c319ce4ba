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

LOC_MU, LOC_SIGMA, LOC_H = 1, 2, 4


class OracleCfg(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
                ("K", ctypes.c_int), ("dt", ctypes.c_double),
                ("growth_form", ctypes.c_int), ("localized", ctypes.c_int),
                ("maintain", ctypes.c_int), ("r_diff", ctypes.c_int),
                ("alpha_on", ctypes.c_int), ("eps_u", ctypes.c_double),
                ("eps_p", ctypes.c_double)]


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
            lib.oracle_stats.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
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


def step(world, A=None, P=None, kernels=None, return_u=False, return_alpha=False):
    """One step of ``world`` (an inputs.World) from state (A, P), FP64.

    Returns (A_out, P_out) and, on request, U[K, H, W] and alpha[H, W]."""
    lib = _load()
    A = _f64(world.A if A is None else A)
    P = world.P if P is None else P
    K = world.n_kernels
    if K > 64:
        raise ValueError("oracle supports at most 64 kernels")
    C, H, W = A.shape
    ks = world_kernels(world) if kernels is None else kernels
    off = np.zeros(K, np.int64)
    o = 0
    for i, k in enumerate(ks):
        off[i] = o
        o += k.size
    Kw = _f64(np.concatenate([k.ravel() for k in ks]))
    cfg = OracleCfg(H, W, C, K, float(world.dt), world.growth_form, world.localized,
                    world.maintain_genes, world.r_diff, world.alpha_on,
                    float(world.eps_u), float(world.eps_p))
    ia = lambda v: np.ascontiguousarray(np.asarray(v, np.int32))
    src = ia([k.src for k in world.kernels])
    dst = ia([k.dst for k in world.kernels])
    rad = ia([k.radius for k in world.kernels])
    h = _f64([k.h for k in world.kernels])
    mu = _f64([k.mu for k in world.kernels])
    sg = _f64([k.sigma for k in world.kernels])
    A_out = np.zeros_like(A)
    n_p = world.n_planes
    Pp = _f64(P) if (n_p and P is not None) else None
    P_out = np.zeros_like(Pp) if Pp is not None else None
    U = np.zeros((K, H, W), np.float64) if return_u else None
    alpha = np.zeros((H, W), np.uint8) if return_alpha else None
    ipp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    null = ctypes.POINTER(ctypes.c_double)()
    lib.oracle_step(ctypes.byref(cfg), ipp(src), ipp(dst), ipp(rad), _dp(h), _dp(mu), _dp(sg),
                    _dp(Kw), off.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                    _dp(A), _dp(Pp) if Pp is not None else null, _dp(A_out),
                    _dp(P_out) if P_out is not None else null,
                    _dp(U) if U is not None else null,
                    alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)) if alpha is not None
                    else ctypes.POINTER(ctypes.c_ubyte)())
    out = [A_out, P_out]
    if return_u:
        out.append(U)
    if return_alpha:
        out.append(alpha)
    return tuple(out)


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
