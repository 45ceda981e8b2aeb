"""The multi-GPU host logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

Records are independent, so the copy path shards with no collective; the
only cross-rank steps are the barrier and the max over ranks of the timed
region.  Weak scaling: the job's throughput is every rank's bytes over the
slowest rank's time.  The reference arm runs on rank 0 alone.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        dist.barrier()
        # rank k's timed region lasted 10 (k + 1) ms
        slowest = bench.max_over_ranks(10.0 * (rank + 1), w)
        out.put((r, w, local, slowest, bench.job_throughput(1e9, w, slowest)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time_and_the_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert [g[2] for g in got] == [0, 1]
    for _, _, _, slowest, gbs in got:
        assert slowest == 20.0
        assert gbs == pytest.approx(2 * 1e9 / 0.020 / 1e9)


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(2e9, 1, 1.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
