"""Host-side logic of bench.py on CPU: the replica aggregation across ranks
(world size 2 over gloo, as torchrun launches it), the environment parsing,
and the reference arm (the FP64 oracle timed on the host cores), which only
rank 0 runs."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, loc = bench.dist_env()
        # rank 1 is the slower one: the step time is the max over ranks
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, torch.device("cpu"))
        value = bench.replica_rate(1e6, ms * 1e-3, w)
        q.put((rank, w, r, loc, ms, value))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world_size_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    assert all(p.exitcode == 0 for p in ps)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, w, r, loc, ms, value in got:
        assert w == 2 and r == rank and loc == rank
        assert ms == 15.0                       # the slower rank's time
        assert value == pytest.approx(2 * 1e6 / 15e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.replica_rate(10.0, 2.0, 1) == 5.0


def test_reference_arm_only_rank0_prints(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py", "--impl", "reference", "--n", "4096", "--steps", "1",
                    "--warmup", "0"]
        args = bench.parse()
    finally:
        sys.argv = sys_argv
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_cpu():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "4096",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "interactions/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
