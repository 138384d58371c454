"""Energy sharding over two ranks with the gloo backend on CPU.

The GPU solve is replaced by a host function of the energy (the multi-rank
logic under test is partitioning, the max-over-ranks timing reduction and
the host-side gather, none of which touches a GPU)."""

import os
import socket

import numpy as np
import pytest

from paper_1104_0623_gb300 import shard


def fake_solve(E):
    E = np.asarray(E)
    return np.stack([E * (k + 1) + 1j * k for k in range(3)], axis=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nE, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    E = np.linspace(0.1, 7.9, nE) + 1e-6j
    got = shard.solve_sharded(fake_solve, E, rank, world)
    t = shard.max_over_ranks(1.0 + rank)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), got)
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("nE", [7, 8, 512])
def test_two_ranks_gather_the_whole_grid(tmp_path, nE):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, nE, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    E = np.linspace(0.1, 7.9, nE) + 1e-6j
    ref = fake_solve(E)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"r{r}.npy"), ref)
        assert np.load(tmp_path / f"t{r}.npy")[0] == 2.0


def test_shard_bounds_partition():
    for nE in (0, 1, 5, 512, 513):
        for world in (1, 2, 3, 8):
            blocks = [shard.shard_bounds(nE, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == nE
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_step_energies_are_disjoint_across_ranks():
    E = np.linspace(0.1, 7.9, 512) + 1e-6j
    seen = []
    for step in range(4):
        for rank in range(4):
            seen.append(shard.step_energies(E, step, rank, 4, 8))
    allE = np.concatenate(seen)
    assert len(np.unique(allE)) == len(allE) == 128
