"""Domain decomposition of one periodic grid into slabs of rows, on the CPU: gloo ranks each step their slab
with the oracle and exchange, before every step, exactly the halo the CUDA library's lb_ch_halo_export /
lb_ch_halo_import move -- three rows of phi and one row of populations from each neighbour -- through the
same exchange routine (paper_1805_00007_gb300.shard) the GPU ranks use.  The gathered slabs equal the
single-grid oracle bit for bit: the halo is sufficient, and the protocol pairs the right rows.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import shard
from paper_1805_00007_gb300 import workloads as wl

torch = pytest.importorskip("torch")

H = shard.HALO_ROWS


def _problem(kind):
    """Uniform flows (the oracle evaluates a flow at a node's own row, and a uniform flow is the same at the
    global row a ghost row stands for); the library's slabs evaluate any flow at global rows, which the GPU
    tests check."""
    n = 40
    if kind == "disk":
        _, phi0, _ = wl.zalesak(n=n)
        p = wl.make_params(nx=n, ny=n, vel=wl.VEL_UNIFORM, ux0=0.02, uy0=0.035, model=2, tau=0.8, M=0.01)
    else:
        p = wl.make_params(nx=n, ny=n, vel=wl.VEL_UNIFORM, ux0=0.03, uy0=-0.04, model=1, tau=1.3, M=0.02,
                           sigma=0.02, W=3.0)
        phi0 = wl.random_smooth_phi(n, n, seed=5)
    return p, phi0


def _export(g, side):
    """The halo of one side as the library lays it out: 3 rows of phi, then one row of populations."""
    phi = oracle.phi_of(g)
    rows = slice(0, H) if side == 0 else slice(g.shape[1] - H, g.shape[1])
    grow = g[:, 0, :] if side == 0 else g[:, -1, :]
    return np.concatenate([phi[rows].ravel(), grow.ravel()])


def _slab_step(p, y0, g, recv_lo, recv_hi, n):
    """One oracle step of a slab from its rows and the two halos: the slab is extended by H ghost rows on each
    side -- the row next to it with the neighbour's populations, the two beyond it carrying only phi (as g_0;
    the other populations there are never streamed into the slab) -- and stepped as a periodic grid; rows
    within H of the extended edge are wrong and dropped, the slab's own rows are exact."""
    nyl, nx = g.shape[1], g.shape[2]
    ext = np.zeros((9, nyl + 2 * H, nx))
    for halo, rows, grow_at in ((recv_lo, range(0, H), H - 1), (recv_hi, range(nyl + H, nyl + 2 * H), nyl + H)):
        phi = halo[:H * nx].reshape(H, nx)
        ext[0, list(rows)] = phi
        ext[:, grow_at] = halo[H * nx:].reshape(9, nx)
    ext[:, H:H + nyl] = g
    assert p["vel"] == wl.VEL_UNIFORM
    return oracle.step(dict(p, ny=nyl + 2 * H), ext, n)[:, H:H + nyl]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, kind, nsteps, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, phi0 = _problem(kind)
    g_all = oracle.init(p, phi0)
    y0, nyl = shard.slab_rows(p["ny"], world)[rank]
    g = g_all[:, y0:y0 + nyl].copy()
    nb = H * p["nx"] + 9 * p["nx"]
    recv_lo, recv_hi = torch.empty(nb, dtype=torch.float64), torch.empty(nb, dtype=torch.float64)
    for n in range(nsteps):
        send_lo, send_hi = torch.from_numpy(_export(g, 0)), torch.from_numpy(_export(g, 1))
        shard.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world)
        g = _slab_step(p, y0, g, recv_lo.numpy(), recv_hi.numpy(), n)
    parts = [None] * world
    dist.all_gather_object(parts, (y0, oracle.phi_of(g)))
    if rank == 0:
        np.save(out_path, np.concatenate([ph for _, ph in sorted(parts, key=lambda t: t[0])], axis=0))
    dist.barrier()
    dist.destroy_process_group()


def test_slab_rows_cover_the_grid():
    for ny, world in ((40, 2), (41, 3), (64, 16), (9, 2)):
        rows = shard.slab_rows(ny, world)
        assert rows[0][0] == 0 and sum(n for _, n in rows) == ny
        assert all(rows[k][0] + rows[k][1] == rows[k + 1][0] for k in range(world - 1))
        assert max(n for _, n in rows) - min(n for _, n in rows) <= 1 and min(n for _, n in rows) >= 4
    with pytest.raises(ValueError):
        shard.slab_rows(7, 2)


def test_halo_field_wraps_periodically():
    phi = np.arange(10.0)[:, None] * np.ones((1, 3))
    f = shard.halo_field(phi, 8, 2)
    assert f.shape == (2 + 2 * H, 3) and list(f[:, 0]) == [5, 6, 7, 8, 9, 0, 1, 2]


@pytest.mark.parametrize("world,kind", [(2, "disk"), (3, "random"), (1, "disk"), (4, "random")])
def test_gloo_slabs_equal_one_grid(tmp_path, world, kind):
    import torch.multiprocessing as mp
    nsteps = 9
    out = tmp_path / "phi.npy"
    mp.start_processes(_rank_main, args=(world, _free_port(), kind, nsteps, str(out)), nprocs=world, join=True,
                       start_method="spawn")
    p, phi0 = _problem(kind)
    ref, _ = oracle.simulate(p, phi0, nsteps)
    assert np.array_equal(np.load(out), ref)
