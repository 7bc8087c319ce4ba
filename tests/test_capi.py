"""The C-ABI library builds, loads, and exports every entry point that
include/lenia.h declares; argument validation runs on the host before any
CUDA call (so it is testable without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2304_05639_gb300 import build, inputs, lenia

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lenia.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "lenia.h")).read()
    return sorted(set(re.findall(r"LENIA_API[^;(]*?\b(lenia_\w+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = _declared()
    for must in ("lenia_init", "lenia_step", "lenia_rollout", "lenia_backward", "lenia_stats",
                 "lenia_destroy", "lenia_last_error"):
        assert must in names
    assert sorted(lenia.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def _init_status(lib, world, **over):
    cfg, ks = lenia.config_from_world(world)
    for k, v in over.items():
        if k.startswith("k0_"):
            setattr(ks[0], k[3:], v)
        else:
            setattr(cfg, k, v)
    arr = (lenia.LeniaKernelDesc * len(ks))(*ks)
    out = ctypes.c_void_p(123)
    st = lib.lenia_init(ctypes.byref(cfg), arr, None, ctypes.byref(out))
    return st, out.value


@pytest.mark.parametrize("over", [
    dict(width=30),                       # not a multiple of 4
    dict(height=4),
    dict(n_channels=0),
    dict(n_kernels=65),
    dict(dt=-1.0),
    dict(growth_form=7),
    dict(localized=8),
    dict(maintain_genes=1, localized=0),
    dict(r_diff=9),
    dict(conv_path=1, height=100),        # FFT path needs powers of two
    dict(k0_radius=0),
    dict(k0_radius=40),                   # 2R + 1 > 64
    dict(k0_src_channel=3),
    dict(k0_n_shells=5),
    dict(k0_sigma=0.0),                   # global sigma must be > 0
    dict(k0_form=3),
])
def test_init_rejects_invalid_config(lib, over):
    w = inputs.single_kernel_global()
    st, out = _init_status(lib, w, **over)
    assert st == lenia.LENIA_EINVAL
    assert out is None


@pytest.mark.parametrize("over", [
    dict(n_rings=0),                      # kernel genes need the ring decomposition
    dict(n_rings=65),
    dict(localized=7),                    # rings without kernel genes
    dict(n_channels=8, n_rings=40),       # 320 ring planes > 256
    dict(k0_radius=5),                    # one radius for every kernel
])
def test_init_rejects_invalid_ring_config(lib, over):
    w = inputs.ring_world(H=64, W=64, R=6, n_rings=12, patch=16, n_geno=2)
    st, out = _init_status(lib, w, **over)
    assert st == lenia.LENIA_EINVAL
    assert out is None


def test_status_strings(lib):
    assert lib.lenia_status_string(0) == b"ok"
    assert lib.lenia_status_string(1) == b"invalid argument"
    assert lib.lenia_last_error(None) == b"null context"
    lib.lenia_destroy(None)               # no-op


def test_context_free_entry_points_validate_on_the_host(lib):
    """Null outputs and null contexts are rejected before any CUDA call."""
    d = ctypes.c_double(0.0)
    assert lib.lenia_measure_fp32_peak(None, ctypes.byref(d), None) == lenia.LENIA_EINVAL
    assert lib.lenia_measure_fp32_peak(ctypes.byref(d), None, None) == lenia.LENIA_EINVAL
    assert lib.lenia_rollout(None, None, None, 1, None, None) == lenia.LENIA_EINVAL
    assert lib.lenia_backward(None, None, None, 1, None, None, None, None) == lenia.LENIA_EINVAL
    assert lib.lenia_step_host_async(None, None, None, None, None, None, None) == lenia.LENIA_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of lenia_config, lenia_kernel_desc and lenia_events
    have the C compiler's sizes and field offsets."""
    structs = {"lenia_config": lenia.LeniaConfig, "lenia_kernel_desc": lenia.LeniaKernelDesc,
               "lenia_events": lenia.LeniaEvents}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lenia.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, v = line.split()
        got[(cname, field)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
