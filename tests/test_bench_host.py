"""Host-side logic of bench.py, on CPU: the reference arm's JSON line and the
multi-rank reduction (two gloo ranks)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "pr1", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == bench.UNIT and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1


def test_job_throughput_is_weak_scaling():
    assert bench.job_throughput(1000, 1, 1.0) == pytest.approx(1e6)
    assert bench.job_throughput(1000, 4, 2.0) == pytest.approx(2e6)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 15.0, 1: 15.0}


def test_oracle_process_pool_driver_equals_the_oracle():
    """The all-cores CPU baseline runs the oracle's own functions on a process
    pool; its results must be the oracle's, bit for bit."""
    import multiprocessing as mp

    import oracle
    import oracle.parallel as op
    import synth

    inst = synth.make_config("pr1")
    with mp.get_context("spawn").Pool(2) as pool:
        a = op.varlingam_pool(inst.X, inst.p, pool, 2)
    b = oracle.varlingam(inst.X, inst.p)
    assert np.array_equal(a["D"], b["D"])
    assert list(a["order"]) == list(b["order"])
    assert np.array_equal(a["B0"], b["B0"])
    assert np.array_equal(a["Btau"], b["Btau"])
