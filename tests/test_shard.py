"""Multi-rank logic of the shift and instance splits, on CPU ranks (gloo)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import pfgen
from paper_2311_11833_gb300 import shard


def test_partition_instances_balanced_and_complete():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(size=257)
    for world in (1, 2, 3, 8):
        parts = shard.partition_instances(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(257))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: the heaviest bin exceeds the mean by at most the largest item
        assert max(loads) <= np.mean(loads) + max(costs) + 1e-12
    assert shard.partition_instances(costs, 2) == shard.partition_instances(costs, 2)


def test_shift_subsets_cover_once():
    for K in (1, 4, 6, 8):
        for world in (1, 2, 3, 5):
            got = sorted(k for r in range(world) for k in shard.shift_subset(K, r, world))
            assert got == list(range(K))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = pfgen.make_instance("plain")
    A = oracle.to_scipy(inst)
    t = pfgen.symmetric_shifts(4)
    beta = oracle.weights_float(list(t))
    b = pfgen.rhs(inst.n, 2, 3)

    def partial(t_sub, w_sub):
        if len(t_sub) == 0:
            return torch.zeros(b.shape, dtype=torch.float64)
        X = oracle.perturbed_solutions(A, inst.D, t_sub, b)
        return torch.tensor(oracle.combine(X, w_sub))

    x = shard.solve_shift_split(partial, t, beta)
    if rank == 0:
        np.save(out_path, x.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shift_split_allreduce_equals_full_combine(tmp_path, world):
    out = str(tmp_path / "x.npy")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    inst = pfgen.make_instance("plain")
    t = pfgen.symmetric_shifts(4)
    ref = oracle.x_hat(oracle.to_scipy(inst), inst.D, t, pfgen.rhs(inst.n, 2, 3))
    np.testing.assert_allclose(np.load(out), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
