"""Host side of the shift-partitioned filter (Sec. 6: each process owns a
range of the linear systems) on the CPU: the choice of ranges, the summation
tree they must align with, and the all-gather of the partial blocks over two
gloo ranks.  The GPU part (partial filters and their combination on the
device, bit for bit against one handle) is in test_gpu_partition.py."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1404_2891_gb300 import dist as pdist  # noqa: E402


@pytest.mark.parametrize("q", [8, 16, 21, 32, 33, 256])
@pytest.mark.parametrize("world", [1, 2, 4, 8])
def test_ranges_partition_the_shifts_along_the_leaves(q, world):
    r = pdist.shift_ranges(q, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == q
    for (a, b), (c, d) in zip(r, r[1:]):
        assert b == c and a < b
    leaves = pdist.leaf_bounds(q)
    L = 8 // world
    for k, (a, b) in enumerate(r):
        assert (a, b) == (leaves[k * L], leaves[(k + 1) * L])


def test_too_few_shifts_for_the_ranks():
    with pytest.raises(ValueError):
        pdist.shift_ranges(5, 8)
    with pytest.raises(ValueError):
        pdist.shift_ranges(32, 3)


def tree_sum(terms, bounds):
    """The documented tree: leaves summed in order, then pairwise level by level."""
    leaves = []
    for j in range(len(bounds) - 1):
        acc = 0j
        for t in terms[bounds[j]:bounds[j + 1]]:
            acc = acc + t
        leaves.append(acc)
    w = 1
    while w < len(leaves):
        for j in range(0, len(leaves) - w, 2 * w):
            leaves[j] = leaves[j] + leaves[j + w]
        w *= 2
    return leaves[0]


@pytest.mark.parametrize("q", [16, 21, 32])
@pytest.mark.parametrize("world", [2, 4, 8])
def test_partial_subtrees_combine_to_the_same_bits(q, world):
    """With the ranges of shift_ranges, adding the ranks' subtree sums along the
    top of the tree reproduces the one-rank sum exactly (same association)."""
    rng = np.random.default_rng(q * 10 + world)
    terms = rng.standard_normal(q) * 10.0 ** rng.uniform(-8, 8, q) + 1j * rng.standard_normal(q)
    full = tree_sum(list(terms), pdist.leaf_bounds(q))
    leaves = pdist.leaf_bounds(q)
    L = 8 // world
    parts = []
    for r, (a, b) in enumerate(pdist.shift_ranges(q, world)):
        local = [x - a for x in leaves[r * L:(r + 1) * L + 1]]
        parts.append(tree_sum(list(terms[a:b]), local))
    comb = tree_sum(parts, list(range(world + 1)))
    assert comb == full
    # the naive order (left to right over all terms) generally differs: the tree matters
    naive = 0j
    for t in terms:
        naive = naive + t
    assert abs(naive - full) <= 1e-9 * np.abs(terms).sum()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def gather_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1404_2891_gb300 import dist as pd
    rng = np.random.default_rng(100 + rank)
    block = rng.standard_normal((33, 5)) + 1j * rng.standard_normal((33, 5))
    got = pd.gather_blocks(block)
    np.save(os.path.join(out_dir, f"mine{rank}.npy"), block)
    np.save(os.path.join(out_dir, f"got{rank}.npy"), np.stack(got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_partials_in_rank_order(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(gather_worker, args=(2, free_port(), str(tmp_path)), nprocs=2, join=True)
    mine = [np.load(tmp_path / f"mine{r}.npy") for r in range(2)]
    for r in range(2):
        got = np.load(tmp_path / f"got{r}.npy")
        assert got.shape == (2, 33, 5)
        for j in range(2):
            assert np.array_equal(got[j], mine[j])  # bit for bit, rank order
