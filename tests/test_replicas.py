"""The multi-GPU path is replicas only (every rank projects its own field; nothing is exchanged):
its host logic, the slowest-rank timing and the whole-job throughput, on two gloo ranks on the
CPU, and the reference arm's ranks other than 0, which must exit without work."""
import os
import socket
import sys
import time

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, ms_by_rank, out_dir: str):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_total, value = bench.job_timing(ms_by_rank[rank], 1000, 5, world)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{ms_total!r} {value!r}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_timing_takes_the_slowest_of_two_gloo_ranks(tmp_path):
    ms_by_rank = [10.0, 12.5]
    mp.spawn(_rank_main, args=(2, _free_port(), ms_by_rank, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        ms_total, value = map(float, (tmp_path / f"rank{rank}.txt").read_text().split())
        assert ms_total == 12.5                      # every rank reports the job's time
        assert value == pytest.approx(2 * 1000 * 5 / 0.0125)


def test_job_timing_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    ms_total, value = bench.job_timing(8.0, 512 ** 3, 10, 1)
    assert ms_total == 8.0
    assert value == pytest.approx(512 ** 3 * 10 / 0.008)


def test_reference_arm_ranks_other_than_0_do_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 3, 3, 2

    monkeypatch.setenv("RANK", "1")
    t0 = time.perf_counter()
    assert bench.run_reference(Args()) is None
    assert time.perf_counter() - t0 < 1.0            # no oracle sample was taken
    assert capsys.readouterr().out == ""
