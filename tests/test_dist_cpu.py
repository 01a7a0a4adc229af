"""The N > 1 path of bench.py on the CPU: two gloo ranks (one process each, rendezvous on
127.0.0.1) check that the whole-job figure is the sum of the ranks' units over the
slowest rank's time, that the barrier returns on both ranks, and that the reference arm
does no work on ranks other than 0. No GPU, no collective on the data path."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    ws, r, local = bench.dist_init("gloo")
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier()
    units, secs = bench.aggregate(100.0 * (rank + 1), 0.5 + rank)
    bench.barrier()
    # the reference arm returns at once on rank != 0 (rank 0 alone times the oracle)
    if rank != 0:
        bench.run_reference(bench.parse_args(["--impl", "reference", "--scale", "4", "--steps", "1", "--warmup", "3"]))
    out[rank] = (units, secs)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_aggregate_max_time_and_sum_units():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        units, secs = res[r]
        assert units == 300.0  # 100 + 200
        assert secs == 1.5     # the slower rank's 0.5 + 1
