"""The N > 1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank simulates its own environments (weak scaling, no collective on the data path);
the only exchange is the job's timing: the longest rank's time and the sum of the ranks'
units.  The reference arm runs on rank 0 alone."""
import argparse
import multiprocessing as mp
import os
import socket

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r took 10 + 2r ms for its own 8000 env-substeps
        q.put((rank,) + bench.job_rate(10.0 + 2.0 * rank, 8000, ws))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, job_ms, units in got:
        assert job_ms == 12.0 and units == 16000, (rank, job_ms, units)
        assert abs(value - 16000 / 0.012) < 1e-6 * value


def test_job_rate_single_rank_needs_no_process_group():
    assert bench.job_rate(5.0, 1000, 1) == (1000 / 0.005, 5.0, 1000)


def test_every_rank_gets_its_own_scene_seed():
    seeds = {bench.env_seed(7, r) for r in range(8)}
    assert len(seeds) == 8 and bench.env_seed(7, 0) == 7


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(ref_envs=1, seed=0, warmup=0, steps=1)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
