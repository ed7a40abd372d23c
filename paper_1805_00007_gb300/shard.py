"""Work over ranks, two ways.

Ensembles: every instance is an independent problem, so ranks share the instances and exchange nothing
while they step; only per-instance observables are gathered at the end.

One grid: a grid periodic in y is split into slabs of consecutive rows, one per rank (or several handles on
one device); before every step each slab receives the three rows of phi and the one row of populations
next to it from each neighbour (the halo the library's lb_ch_halo_export / lb_ch_halo_import move), and the
slabs together give the whole grid's result bit for bit.

One process per GPU (torch.distributed); this module holds the host-side logic only -- every step of the
method runs in the CUDA library.
"""
from __future__ import annotations


def partition(sizes, world: int) -> list[list[int]]:
    """Instance indices per rank, balanced by lattice nodes: instances in decreasing size, each to the
    rank with the least work so far (ties to the lowest rank, then the lower index).  Deterministic, so
    every rank computes the same assignment without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(ix) for ix in out]


def shard(ensemble, rank: int, world: int):
    """(indices, params, fields) of this rank's share of a list of (params, phi0) instances."""
    sizes = [int(p["nx"]) * int(p["ny"]) for p, _ in ensemble]
    idx = partition(sizes, world)[rank]
    return idx, [ensemble[i][0] for i in idx], [ensemble[i][1] for i in idx]


def gather(values, indices, n_total: int, group=None) -> list:
    """Every rank's per-instance values, placed at their instance indices (an all-gather of Python objects
    over the process group; a list of n_total on every rank)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, list(zip(indices, values)), group=group)
    out = [None] * n_total
    for part in parts:
        for i, v in part:
            out[i] = v
    return out


# ----------------------------------------------------------------------------- one grid split into slabs

HALO_ROWS = 3  # rows of phi a slab needs from each neighbour (mu, its gradient and the pull: Eqs. mu, LB)


def slab_rows(ny: int, world: int) -> list[tuple[int, int]]:
    """(first row, rows) of each rank's slab of a grid of ny rows: consecutive, balanced to one row, in rank
    order (rank r's upper neighbour is r + 1, periodically).  Every slab needs at least 4 rows."""
    if world < 1 or ny < 4 * world:
        raise ValueError(f"cannot split {ny} rows into {world} slabs of at least 4 rows")
    base, extra = divmod(ny, world)
    out, y0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((y0, n))
        y0 += n
    return out


def halo_field(phi0, y0: int, ny_local: int):
    """The slab's initial field with HALO_ROWS rows of each neighbour (global rows taken periodically)."""
    import numpy as np
    rows = np.arange(y0 - HALO_ROWS, y0 + ny_local + HALO_ROWS)
    return np.take(np.asarray(phi0, dtype=np.float64), rows, axis=0, mode="wrap")


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """The halo exchange between slabs on consecutive ranks of a periodic grid (torch.distributed tensors:
    gloo on the host, NCCL on the GPU).  send_lo / send_hi: this slab's lowest / highest rows; recv_lo /
    recv_hi receive the rows below / above it (the lower neighbour's highest rows, the upper neighbour's
    lowest).  Two phases, each with one send and one receive per rank, so that the pairing is unambiguous
    even when both neighbours are the same rank (two slabs)."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist
    below, above = (rank - 1) % world, (rank + 1) % world
    for send, to, recv, frm in ((send_hi, above, recv_lo, below), (send_lo, below, recv_hi, above)):
        reqs = dist.batch_isend_irecv([dist.P2POp(dist.isend, send, to, group),
                                       dist.P2POp(dist.irecv, recv, frm, group)])
        for r in reqs:
            r.wait()


class SlabStack:
    """A periodic grid stepped as several slabs, each its own handle of the CUDA library on the current device,
    with the halos moved between them by device-to-device copies before every step (the single-device form of
    the decomposition; SlabRank is the one-slab-per-rank form)."""

    def __init__(self, params: dict, phi0, prec="f64", n_slabs: int = 2, stream=None):
        import torch
        from . import abi
        self.params = dict(params)
        self.rows = slab_rows(int(params["ny"]), n_slabs)
        pr = abi.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        dev = torch.device("cuda", torch.cuda.current_device())
        if stream is None:  # one stream for every slab: the exports, imports and steps are then stream-ordered
            self._own_stream = torch.cuda.Stream(device=dev)
            stream = self._own_stream.cuda_stream
        self.handles = [abi.lb_ch_init_slab(self.params, y0, n, halo_field(phi0, y0, n), pr, stream)
                        for y0, n in self.rows]
        nb = abi.lb_ch_halo_bytes(self.handles[0])
        self._lo = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in self.handles]  # each slab's lowest rows
        self._hi = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in self.handles]  # and highest rows
        self.streams = [abi.lb_ch_stream(h) for h in self.handles]
        self._abi = abi

    def _sync(self):
        """Order the slabs' streams: each waits for all (the exports of one feed the imports of another)."""
        import torch
        if len(set(self.streams)) > 1:
            torch.cuda.synchronize()

    def exchange(self):
        abi, k = self._abi, len(self.handles)
        for h, lo, hi in zip(self.handles, self._lo, self._hi):
            abi.lb_ch_halo_export(h, 0, lo.data_ptr())
            abi.lb_ch_halo_export(h, 1, hi.data_ptr())
        self._sync()
        for j, h in enumerate(self.handles):
            abi.lb_ch_halo_import(h, 0, self._hi[(j - 1) % k].data_ptr())
            abi.lb_ch_halo_import(h, 1, self._lo[(j + 1) % k].data_ptr())
        self._sync()

    def step(self, nsteps: int):
        for _ in range(int(nsteps)):
            self.exchange()
            for h in self.handles:
                self._abi.lb_ch_step(h, 1)
        return self

    def phi(self):
        import numpy as np
        nx = int(self.params["nx"])
        return np.concatenate([self._abi.lb_ch_observe(h, 0, self._abi.LBCH_OBS_PHI, (n, nx))
                               for h, (_, n) in zip(self.handles, self.rows)], axis=0)

    def close(self):
        for h in self.handles:
            self._abi.lb_ch_free(h)
        self.handles = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SlabRank:
    """This rank's slab of one periodic grid (one process per GPU): the CUDA library steps it, and the halos
    travel between ranks by `exchange` before every step -- NCCL sends and receives into each GPU's own
    memory, or, with a gloo process group (staging=True, the default for gloo), through pinned host buffers.
    The library, the staging copies and the process group share one stream of the rank's own."""

    def __init__(self, params: dict, phi0, prec="f64", rank: int = 0, world: int = 1, group=None,
                 staging: bool | None = None):
        import torch
        from . import abi
        self.rank, self.world, self.group = rank, world, group
        self.params = dict(params)
        self.y0, self.ny = slab_rows(int(params["ny"]), world)[rank]
        dev = torch.device("cuda", torch.cuda.current_device())
        # the library's work, the staging copies and the process group's transfers all run on this stream
        # (torch's default stream would be the legacy NULL stream, which the library replaces by one of its own)
        self.stream = torch.cuda.Stream(device=dev)
        pr = abi.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.h = abi.lb_ch_init_slab(self.params, self.y0, self.ny, halo_field(phi0, self.y0, self.ny), pr,
                                     self.stream.cuda_stream)
        nb = abi.lb_ch_halo_bytes(self.h)
        self.bufs = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(4)]
        if staging is None:
            import torch.distributed as dist
            staging = world > 1 and dist.get_backend(group) == "gloo"
        self.host = [torch.empty(nb, dtype=torch.uint8).pin_memory() for _ in range(4)] if staging else None
        self._abi = abi

    def step(self, nsteps: int):
        import torch
        abi = self._abi
        send_lo, send_hi, recv_lo, recv_hi = self.bufs
        with torch.cuda.stream(self.stream):
            for _ in range(int(nsteps)):
                abi.lb_ch_halo_export(self.h, 0, send_lo.data_ptr())
                abi.lb_ch_halo_export(self.h, 1, send_hi.data_ptr())
                if self.host is None:
                    exchange(send_lo, send_hi, recv_lo, recv_hi, self.rank, self.world, self.group)
                else:
                    h_slo, h_shi, h_rlo, h_rhi = self.host
                    h_slo.copy_(send_lo)
                    h_shi.copy_(send_hi)
                    self.stream.synchronize()
                    exchange(h_slo, h_shi, h_rlo, h_rhi, self.rank, self.world, self.group)
                    recv_lo.copy_(h_rlo)
                    recv_hi.copy_(h_rhi)
                abi.lb_ch_halo_import(self.h, 0, recv_lo.data_ptr())
                abi.lb_ch_halo_import(self.h, 1, recv_hi.data_ptr())
                abi.lb_ch_step(self.h, 1)
        return self

    def phi(self):
        return self._abi.lb_ch_observe(self.h, 0, self._abi.LBCH_OBS_PHI, (self.ny, int(self.params["nx"])))

    def close(self):
        if self.h:
            self._abi.lb_ch_free(self.h)
            self.h = None
