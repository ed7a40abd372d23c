"""The N > 1 path on the CPU: two gloo ranks share a ragged ensemble (no exchange while stepping) and
gather the per-instance observables; the result equals one process stepping every instance."""
import os
import socket

import numpy as np
import pytest

from paper_1805_00007_gb300 import shard
from paper_1805_00007_gb300 import workloads as wl

torch = pytest.importorskip("torch")


def _ensemble():
    ens = wl.shear_ensemble(n_inst=7, sides=(8, 12, 16), seed=21)
    return [(dict(p, shear=p["shear"] * 50.0, Ustar=p["Ustar"] * 50.0), f) for p, f in ens]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nsteps, out_path):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ens = _ensemble()
    idx, params, fields = shard.shard(ens, rank, world)
    vals = []
    for p, f in zip(params, fields):
        phi, _ = oracle.simulate(p, f, nsteps)
        ob = oracle.observe(phi, f)
        vals.append((ob["mass"], ob["err_l2"]))
    allv = shard.gather(vals, idx, len(ens))
    if rank == 0:
        np.save(out_path, np.array(allv))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_balanced_and_complete():
    sizes = [64 * 64, 512 * 512, 128 * 128, 256 * 256, 512 * 512, 64 * 64, 256 * 256]
    for world in (1, 2, 3, 4):
        parts = shard.partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert shard.partition(sizes, 2) == shard.partition(list(sizes), 2)  # deterministic


def test_two_gloo_ranks_equal_one_process(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    nsteps = 12
    out = tmp_path / "gathered.npy"
    mp.start_processes(_rank_main, args=(2, _free_port(), nsteps, str(out)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    for k, (p, f) in enumerate(_ensemble()):
        phi, _ = oracle.simulate(p, f, nsteps)
        ob = oracle.observe(phi, f)
        assert got[k][0] == ob["mass"] and got[k][1] == ob["err_l2"]
