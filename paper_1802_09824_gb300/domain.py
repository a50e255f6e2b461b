"""Domain decomposition across ranks, one GPU each (Sec. 4.1).

The cut itself (ground cells of each particle, runs of cells along the
space-filling curve balanced by work, ghost cells of each domain) is the
library's host code (``ph_domain_cells``, ``ph_domain_partition``,
``ph_domain_halo``); ``exchange`` moves particles between ranks with
``torch.distributed.all_to_all_single`` (gloo on CPU tensors, NCCL on device
tensors) and calls the library on each rank's local set.  ``exchange_device``
and ``PartitionedStep`` keep the particles on the GPU: cells, counts,
packing and unpacking in the library's kernels, the rows moved by NCCL, and
the local step replayed as a captured graph.  A rank's local set
is its own particles first, then the ghosts: together they hold every
particle within rcut of an own particle, so the short-range forces of the own
particles need nothing from other ranks.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import binding as B


@dataclasses.dataclass
class LocalSet:
    pos: object          # [n_local, 3] own particles first, then ghosts (caller's dtype and device)
    mass: object         # [n_local]
    ids: object          # [n_local] int64 identifiers given by the callers
    n_owned: int
    nside: int
    owner: np.ndarray    # owner rank of every ground cell
    domain_cost: np.ndarray


def exchange(pos, mass, ids, params, key_kind=B.PH_KEY_HILBERT, group=None) -> LocalSet:
    """Send every particle of this rank's shard to the rank that owns its
    ground cell and to every rank that holds that cell as a ghost; return
    this rank's local set.  Collective: every rank of ``group`` calls it
    with its own shard (pos [n,3], mass [n], ids [n] int64 on one device)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = pos.device
    nside, cells = B.ph_domain_cells(pos.detach().to("cpu").contiguous(), params)
    counts = torch.from_numpy(np.bincount(cells, minlength=nside ** 3).astype(np.int64)).to(dev)
    dist.all_reduce(counts, group=group)
    owner, cost = B.ph_domain_partition(counts.cpu().numpy(), nside, key_kind, world)
    sel, flag = [], []
    for r in range(world):
        f = B.ph_domain_halo(owner, nside, r)[cells]
        idx = np.nonzero(f)[0]
        sel.append(idx)
        flag.append(f[idx])
    send_counts = [int(s.size) for s in sel]
    sc = torch.tensor(send_counts, dtype=torch.int64, device=dev)
    rc = torch.empty_like(sc)
    dist.all_to_all_single(rc, sc, group=group)
    recv_counts = [int(x) for x in rc.cpu().tolist()]
    idx = torch.from_numpy(np.concatenate(sel).astype(np.int64)).to(dev)
    fl = torch.from_numpy(np.concatenate(flag).astype(np.float64)).to(dev)
    payload = torch.cat([pos[idx].double(), mass[idx].double()[:, None], fl[:, None]], 1).contiguous()
    out = torch.empty((sum(recv_counts), 5), dtype=torch.float64, device=dev)
    dist.all_to_all_single(out, payload, recv_counts, send_counts, group=group)
    id_out = torch.empty(sum(recv_counts), dtype=torch.int64, device=dev)
    dist.all_to_all_single(id_out, ids[idx].contiguous(), recv_counts, send_counts, group=group)
    own = out[:, 4] == 1
    perm = torch.cat([torch.nonzero(own).flatten(), torch.nonzero(~own).flatten()])
    out = out[perm]
    return LocalSet(pos=out[:, :3].to(pos.dtype).contiguous(), mass=out[:, 3].to(mass.dtype).contiguous(),
                    ids=id_out[perm].contiguous(), n_owned=int(own.sum()), nside=nside, owner=owner,
                    domain_cost=cost)


def accel_partitioned(pos, mass, ids, params, g_mode=B.PH_G_EXACT, key_kind=B.PH_KEY_HILBERT, group=None,
                      stream=None):
    """Short-range accelerations of this rank's own particles after one
    exchange: returns (ids of the own particles, their accelerations [n,3]
    float32, the local set).  Device tensors; one GPU per rank."""
    import torch
    local = exchange(pos, mass, ids, params, key_kind, group)
    acc = torch.zeros((local.pos.shape[0], 3), dtype=torch.float32, device=local.pos.device)
    lv, pr = B.ph_accel(local.pos, local.mass, params, g_mode, None, acc, stream)
    n = local.n_owned
    ids_own, acc_own = local.ids[:n], acc[:n]
    torch.cuda.synchronize()
    B.ph_free(pr)
    B.ph_free(lv)
    return ids_own, acc_own, local


def exchange_device(pos, mass, ids, params, key_kind=B.PH_KEY_HILBERT, group=None, send=None, stream=None):
    """The exchange of ``exchange`` with the particles kept on the GPU: cells,
    cell counts, packing and unpacking run in the library's kernels
    (ph_domain_cells_device, ph_domain_pack, ph_domain_unpack); the counts are
    summed and the rows moved by collectives on device tensors (NCCL), the
    cut made on the host from the summed counts.  Returns (LocalSet, send
    buffer) -- pass the buffer back in to reuse it."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = pos.device
    nside, cells, counts = B.ph_domain_cells_device(pos, params, stream)
    dist.all_reduce(counts, group=group)
    owner, cost = B.ph_domain_partition(counts.cpu().numpy(), nside, key_kind, world)
    send, send_counts = B.ph_domain_pack(pos, mass, ids, cells, owner, nside, world, send, stream)
    sc = torch.tensor(send_counts, dtype=torch.int64, device=dev)
    rc = torch.empty_like(sc)
    dist.all_to_all_single(rc, sc, group=group)
    recv_counts = [int(x) for x in rc.cpu().tolist()]
    n_recv = sum(recv_counts)
    recv = torch.empty((max(n_recv, 1), B.PH_DOMAIN_ROW), dtype=torch.float64, device=dev)
    dist.all_to_all_single(recv[:n_recv], send[:sum(send_counts)], recv_counts, send_counts, group=group)
    lpos, lmass, lids, n_own = B.ph_domain_unpack(recv, n_recv, pos.dtype, stream)
    return LocalSet(pos=lpos, mass=lmass, ids=lids, n_owned=n_own, nside=nside, owner=owner, domain_cost=cost), send


class PartitionedStep:
    """One short-range step of a rank's own particles after the device
    exchange: the local set is built with its own particles active (their
    target groups get source lists; the ghosts' groups do not), and the build,
    pairs and PP are captured as a graph that later steps replay as long as
    the local set keeps its size (otherwise it is captured again)."""

    def __init__(self, params, key_kind=B.PH_KEY_HILBERT, group=None):
        self.params = params
        self.key_kind = key_kind
        self.group = group
        self.send = None
        self.n_local = -1
        self.graph = self.lv = self.pr = None
        self.local = None

    def __call__(self, pos, mass, ids, stream=None):
        """Exchange and step; returns (ids of the own particles, their
        accelerations) as device tensors (views into the local set)."""
        import torch
        local, self.send = exchange_device(pos, mass, ids, self.params, self.key_kind, self.group, self.send, stream)
        n = int(local.pos.shape[0])
        if n != self.n_local:
            self.close()
            self.pos = torch.empty_like(local.pos)
            self.mass = torch.empty_like(local.mass)
            self.acc = torch.zeros((n, 3), dtype=torch.float32, device=local.pos.device)
            self.active = torch.zeros(n, dtype=torch.uint8, device=local.pos.device)
            self.pos.copy_(local.pos)
            self.mass.copy_(local.mass)
            self.lv = B.ph_build_leaves(self.pos, self.mass, self.params, stream)
            B.ph_leaves_set_active(self.lv, self.active)
            self.n_local = n
            self.n_own = -1
        if local.n_owned != self.n_own or self.graph is None:
            self.active.zero_()
            self.active[:local.n_owned] = 1
            self.n_own = local.n_owned
            B.ph_free(self.graph)
            self.graph = None
            self.pos.copy_(local.pos)
            self.mass.copy_(local.mass)
            self.lv = B.ph_build_leaves(self.pos, self.mass, self.params, stream, leaves=self.lv)
            self.pr = B.ph_leaf_pairs(self.lv, stream, pairs=self.pr)
            self.graph = B.ph_graph_create(self.lv, self.pr, self.pos, self.mass, B.PH_G_EXACT, None, self.acc,
                                           headroom=0.25, stream=stream)
        else:
            self.pos.copy_(local.pos)
            self.mass.copy_(local.mass)
        B.ph_graph_launch(self.graph, stream)
        self.local = local
        return local.ids[:local.n_owned], self.acc[:local.n_owned]

    def close(self):
        for h in (self.graph, self.pr, self.lv):
            B.ph_free(h)
        self.graph = self.pr = self.lv = None
