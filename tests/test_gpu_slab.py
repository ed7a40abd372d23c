"""Domain decomposition on the GPU: one periodic grid stepped as several slab handles of the library on one
device, the halos moved by the library's own lb_ch_halo_export / lb_ch_halo_import before every step
(paper_1805_00007_gb300.shard.SlabStack).  The slabs together give the single handle's result bit for bit
(the per-node arithmetic is unchanged, only where its inputs come from), and the FP64 oracle to 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import shard
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _whole(p, phi0, nsteps, prec, tile=False):
    with abi.Simulation(p, phi0, prec=prec) as sim:
        if tile:
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 1)
        sim.step(nsteps)
        return sim.phi()


def _slabs(p, phi0, nsteps, prec, n_slabs, tile=False):
    with shard.SlabStack(p, phi0, prec=prec, n_slabs=n_slabs) as st:
        for h in st.handles:
            abi.lb_ch_test_hook(h, abi.LBCH_HOOK_TILE_KERNEL, 1 if tile else 0)
        st.step(nsteps)
        return st.phi()


CASES = {
    "zalesak": lambda: wl.zalesak(n=64)[:2],                       # rotation: the flow jumps across y = 0
    "zalesak_tau08": lambda: wl.zalesak(n=64, tau=0.8)[:2],        # with the populations
    "vortex": lambda: wl.single_vortex(n=48, T=40)[:2],            # time-dependent, sin(2 pi y / ny) of the grid
}


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n_slabs", [2, 3])
def test_slabs_equal_the_whole_grid_bitwise(prec, case, n_slabs):
    p, phi0 = CASES[case]()
    p = dict(p, ny=p["ny"] - 5)          # a ragged split (59 rows: 30 + 29, or 20 + 20 + 19)
    phi0 = phi0[:p["ny"]]
    nsteps = 23
    whole = _whole(p, phi0, nsteps, prec)
    assert np.array_equal(_slabs(p, phi0, nsteps, prec, n_slabs), whole)
    if prec == "f64":
        ref, _ = oracle.simulate(p, phi0, nsteps)
        assert float(np.max(np.abs(whole - ref))) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_slabs_on_the_tile_kernel(prec):
    p, phi0 = CASES["zalesak_tau08"]()
    assert np.array_equal(_slabs(p, phi0, 17, prec, 4, tile=True), _whole(p, phi0, 17, prec))


def test_one_slab_is_the_whole_grid():
    """A single slab exchanges with itself: its halos are its own periodic images."""
    p, phi0 = CASES["vortex"]()
    assert np.array_equal(_slabs(p, phi0, 11, "f32", 1), _whole(p, phi0, 11, "f32"))


def test_slab_rejections():
    p, phi0 = CASES["zalesak"]()
    halo = shard.halo_field(phi0, 0, 32)
    with pytest.raises(abi.LbchError) as ei:   # walls
        abi.lb_ch_init_slab(dict(p, walls=1, vel=wl.VEL_SHEAR, shear=1e-3), 0, 32, halo)
    assert ei.value.status == abi.LBCH_EINVAL
    with pytest.raises(abi.LbchError):         # Model III
        abi.lb_ch_init_slab(dict(p, model=3), 0, 32, halo)
    with pytest.raises(abi.LbchError):         # rows outside the grid
        abi.lb_ch_init_slab(p, 40, 32, halo)
    h = abi.lb_ch_init_slab(p, 0, 32, halo)
    try:
        with pytest.raises(abi.LbchError) as ei:  # several steps without the exchange in between
            abi.lb_ch_step(h, 2)
        assert ei.value.status == abi.LBCH_EINVAL and "one step per call" in str(ei.value)
        dev = torch.device("cuda")
        g = torch.zeros(64 * 64, dtype=torch.float64, device=dev)
        with pytest.raises(abi.LbchError):         # the adjoint is for whole grids
            abi.lb_ch_adjoint_begin(h, g.data_ptr())
    finally:
        abi.lb_ch_free(h)
    with abi.Simulation(p, phi0, prec="f64") as sim:  # halos belong to slab handles
        with pytest.raises(abi.LbchError):
            abi.lb_ch_halo_bytes(sim.h)


def _rank_main(rank, world, port, prec, nsteps, out_path):
    """One process per slab, both on the one GPU here (the kernels of one rank never wait on another's: the
    halos move between steps through the host, by gloo)."""
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    p, phi0 = CASES["vortex"]()
    sl = shard.SlabRank(p, phi0, prec=prec, rank=rank, world=world)
    sl.step(nsteps)
    parts = [None] * world
    dist.all_gather_object(parts, (sl.y0, sl.phi()))
    sl.close()
    if rank == 0:
        np.save(out_path, np.concatenate([ph for _, ph in sorted(parts, key=lambda t: t[0])], axis=0))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_equal_the_whole_grid(tmp_path, world):
    """shard.SlabRank, the one-slab-per-rank driver, in separate processes exchanging through a gloo process
    group: the gathered slabs equal the whole-grid handle bit for bit."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = tmp_path / "phi.npy"
    nsteps = 15
    mp.start_processes(_rank_main, args=(world, port, "f32", nsteps, str(out)), nprocs=world, join=True,
                       start_method="spawn")
    p, phi0 = CASES["vortex"]()
    assert np.array_equal(np.load(out), _whole(p, phi0, nsteps, "f32"))
