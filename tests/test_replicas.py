"""Host side of the multi-GPU path (replicas only: the path has no exchange step).

bench.py under torchrun runs one independent replica per rank and reports the
whole job as every rank's frames over the slowest rank's time.  Here two gloo
ranks on the CPU exercise that aggregation (the same helpers bench.py calls).
"""
import json
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow replica
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        fps = bench.replica_throughput(2, 100, world, ms)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "fps": fps}, f)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_every_rank_frames(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for g in got:
        assert g["ms"] == pytest.approx(15.0)
        assert g["fps"] == pytest.approx(2 * 100 * 2 / 0.015)


def test_single_rank_passes_values_through():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.replica_throughput(1, 10, 1, 2.0) == pytest.approx(5000.0)
