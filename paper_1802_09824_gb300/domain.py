"""Domain decomposition across ranks, one GPU each (Sec. 4.1).

The cut itself (ground cells of each particle, runs of cells along the
space-filling curve balanced by work, ghost cells of each domain) is the
library's host code (``ph_domain_cells``, ``ph_domain_partition``,
``ph_domain_halo``); this module only moves particles between ranks with
``torch.distributed.all_to_all_single`` (gloo on CPU tensors, NCCL on device
tensors) and calls the library on each rank's local set.  A rank's local set
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
