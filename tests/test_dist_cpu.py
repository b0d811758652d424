"""Host side of the multi-GPU path on CPU: two gloo ranks run bench.py's
distributed helpers (max over ranks of the step time, per-rank workloads) as
the GPU run does under torchrun, without a GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    step_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    mx = bench.max_over_ranks(step_ms, w, device="cpu")
    seeds = bench.rank_seeds(r)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{r} {w} {mx} {seeds['pencil']} {seeds['batch']}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_own_workloads(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = free_port()
    mp.spawn(worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    for r, row in enumerate(rows):
        rank, world, mx, ps, bs = int(row[0]), int(row[1]), float(row[2]), int(row[3]), int(row[4])
        assert (rank, world) == (r, 2)
        assert mx == 15.0  # the slowest rank's time, seen by every rank
    assert rows[0][3] != rows[1][3] and rows[0][4] != rows[1][4]  # independent pencils per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
