"""Host logic of the multi-GPU replica path of bench.py (independent worlds,
no data-path collective): the slowest rank's time sets the job time, and the
job value counts every rank's site-steps.  Two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [10.0 + 5.0 * rank, 3.0 - rank]          # rank 1 slower on the first
        got = bench.max_over_ranks(local_ms, torch)
        value = bench.job_value(world, 1000, 20, got[0])
        dist.barrier()
        out[rank] = (got, value)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_two_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        got, value = out[r]
        assert got == [15.0, 3.0]
        assert value == pytest.approx(2 * 1000 * 20 / 0.015)


def test_single_rank_is_identity():
    assert bench.max_over_ranks([1.5, 2.5], torch) == [1.5, 2.5]
    assert bench.job_value(1, 4096, 10, 2.0) == pytest.approx(4096 * 10 / 0.002)


def test_gpus_flag_spawns_ranks():
    """`bench.py --gpus 2` outside torchrun starts two ranks itself (gloo on
    CPU here): rank 0 reports n_gpus = 2 and the slower rank's time."""
    import json
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"),
                          "--gpus", "2", "--rank-check"], capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["ms_max"] == 11.0
    assert d["value"] == pytest.approx(2 * 1000 / 0.011)
