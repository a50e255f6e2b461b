"""Domain decomposition across ranks (Sec. 4.1) on CPU: the library's host
code for cells, the cut along the curve and the ghost cells, and the
exchange of paper_1802_09824_gb300.domain between gloo ranks.  The local
set of every rank must give its own particles exactly the short-range
forces of the whole box (checked with the FP64 oracle)."""
import os
import sys

import numpy as np
import pytest

from oracle import force, keys
from paper_1802_09824_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

L, RCUT = 1.0, 0.1            # ground grid 8^3 (cells of side 0.125 >= rcut)
RS = RCUT / 4.5


def _particles(n=6000, seed=31):
    # uniform background plus a dense clump, so that the work per cell varies
    rng = np.random.default_rng(seed)
    u = rng.random((n - n // 3, 3))
    c = (np.array([0.3, 0.6, 0.45]) + 0.04 * rng.normal(size=(n // 3, 3))) % 1.0
    pos = np.concatenate([u, c]).astype(np.float32)
    mass = np.full(n, 1.0 / n, np.float32)
    return pos, mass


def _params():
    return B.make_params(L, 1.0, 1e-3, RS, RCUT, 32)


def test_cells_follow_the_ground_grid():
    pos, _ = _particles()
    shifted = pos.astype(np.float64) + np.array([1.0, -2.0, 0.0])     # outside the box: wrapped
    for p in (pos, pos.astype(np.float64), shifted):
        ns, cells = B.ph_domain_cells(p, _params())
        assert ns == 8
        xw = np.mod(np.asarray(p, np.float64), L)
        ref = np.floor(xw * ns / L).astype(np.int64)
        ref = (ref[:, 0] * ns + ref[:, 1]) * ns + ref[:, 2]
        far = np.all(np.abs(xw * ns / L - np.round(xw * ns / L)) > 1e-9, axis=1)
        assert far.sum() > 0.99 * len(p)
        assert np.array_equal(cells[far], ref[far])


def _curve_rank(ns, key_kind):
    g = int(np.log2(ns))
    i, j, k = np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    key = keys.hilbert3(i, j, k, g) if key_kind == B.PH_KEY_HILBERT else keys.morton3(i, j, k, g)
    return np.argsort(np.argsort(key))


@pytest.mark.parametrize("key_kind", [B.PH_KEY_MORTON, B.PH_KEY_HILBERT])
@pytest.mark.parametrize("n_domains", [1, 2, 3, 7])
def test_partition_is_contiguous_on_the_curve_and_balanced(key_kind, n_domains):
    pos, _ = _particles()
    ns, cells = B.ph_domain_cells(pos, _params())
    counts = np.bincount(cells, minlength=ns ** 3)
    owner, cost = B.ph_domain_partition(counts, ns, key_kind, n_domains)
    assert owner.min() >= 0 and owner.max() < n_domains
    rank = _curve_rank(ns, key_kind)
    along = owner[np.argsort(rank)]
    assert np.all(np.diff(along) >= 0)               # runs of consecutive cells
    # work of a cell: its count times the count of its 27-cell neighbourhood
    c3 = counts.reshape(ns, ns, ns).astype(np.float64)
    reach = sum(np.roll(np.roll(np.roll(c3, a, 0), b, 1), c, 2)
                for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    w = (c3 * reach).ravel()
    assert np.allclose(cost, [w[owner == d].sum() for d in range(n_domains)])
    assert np.all(np.abs(cost - w.sum() / n_domains) <= w.max() + 1e-9)


def test_more_domains_than_cells():
    # 8^3 = 512 cells cut for 700 domains: every cell owned once, some
    # domains empty (their halo is empty too), work still covered
    pos, _ = _particles()
    ns, cells = B.ph_domain_cells(pos, _params())
    counts = np.bincount(cells, minlength=ns ** 3)
    owner, cost = B.ph_domain_partition(counts, ns, B.PH_KEY_HILBERT, 700)
    used = np.unique(owner)
    assert used.size <= ns ** 3 and owner.max() < 700
    empty = sorted(set(range(700)) - set(used.tolist()))
    assert empty and np.all(cost[empty] == 0)
    assert not B.ph_domain_halo(owner, ns, empty[0]).any()
    c3 = counts.reshape(ns, ns, ns).astype(np.float64)
    reach = sum(np.roll(np.roll(np.roll(c3, a, 0), b, 1), c, 2)
                for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    assert np.isclose(cost.sum(), (c3 * reach).sum())


def test_halo_is_the_26_neighbourhood():
    pos, _ = _particles()
    ns, cells = B.ph_domain_cells(pos, _params())
    owner, _ = B.ph_domain_partition(np.bincount(cells, minlength=ns ** 3), ns, B.PH_KEY_HILBERT, 4)
    o3 = owner.reshape(ns, ns, ns)
    for d in range(4):
        need = B.ph_domain_halo(owner, ns, d).reshape(ns, ns, ns)
        near = np.zeros_like(need, dtype=bool)
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                for c in (-1, 0, 1):
                    near |= np.roll(np.roll(np.roll(o3 == d, a, 0), b, 1), c, 2)
        assert np.array_equal(need == 1, o3 == d)
        assert np.array_equal(need == 2, near & (o3 != d))
        assert np.all(need[~near] == 0)


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1802_09824_gb300 import binding as BB
    from paper_1802_09824_gb300 import domain
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pos, mass = _particles()
    ids = np.arange(len(pos))
    mine = ids % world == rank                     # an arbitrary input shard
    loc = domain.exchange(torch.from_numpy(pos[mine]), torch.from_numpy(mass[mine]),
                          torch.from_numpy(ids[mine].astype(np.int64)),
                          BB.make_params(L, 1.0, 1e-3, RS, RCUT, 32))
    q.put((rank, loc.ids.numpy(), loc.n_owned, loc.pos.numpy(), loc.mass.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_own_particles_and_ghosts(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + world * 17 + (os.getpid() % 1500)
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pos, mass = _particles()
    n = len(pos)
    owned = np.concatenate([g[1][:g[2]] for g in got])
    assert np.array_equal(np.sort(owned), np.arange(n))          # every particle owned once
    glob = force.accel(pos, mass, L, 1.0, 1e-3, RS, RCUT)
    for rank, lid, n_own, lpos, lmass in got:
        assert np.array_equal(lpos, pos[lid]) and np.array_equal(lmass, mass[lid])
        assert n_own < len(lid) < n                               # ghosts, but not the whole box
        # every particle within rcut of an own particle is in the local set
        near = np.zeros(n, bool)
        p64 = pos.astype(np.float64)
        for c in range(0, n_own, 256):
            d = p64[None, lid[c:min(c + 256, n_own)]] - p64[:, None]
            d -= L * np.round(d / L)
            near |= np.any(np.sum(d * d, axis=2) < RCUT * RCUT, axis=1)
        assert set(np.nonzero(near)[0]) <= set(lid.tolist())
        # so the local set gives the own particles the forces of the whole box
        loc = force.accel(lpos, lmass, L, 1.0, 1e-3, RS, RCUT, targets=np.arange(n_own))
        ref = glob.acc[lid[:n_own]]
        assert np.max(np.abs(loc.acc - ref)) <= 1e-12 * np.max(glob.abs_sum[lid[:n_own]])


def test_domain_calls_reject_bad_arguments():
    pos, _ = _particles(200)
    with pytest.raises(B.PhError) as ei:
        B.ph_domain_cells(pos, B.make_params(1.0, 1.0, 1e-3, 0.2, 0.6, 32))      # rcut >= L/2
    assert ei.value.code == B.PH_ERR_ARG
    bad = pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(B.PhError) as ei:
        B.ph_domain_cells(bad, _params())
    assert ei.value.code == B.PH_ERR_NONFINITE
    counts = np.ones(8 ** 3, np.int64)
    for ns, kk, nd in ((6, B.PH_KEY_HILBERT, 2), (8, 7, 2), (8, B.PH_KEY_MORTON, 0)):
        with pytest.raises(B.PhError) as ei:
            B.ph_domain_partition(counts[: ns ** 3], ns, kk, nd)
        assert ei.value.code == B.PH_ERR_ARG
    with pytest.raises(B.PhError) as ei:
        B.ph_domain_halo(np.zeros(27, np.int32), 3, 0)                            # not a power of two
    assert ei.value.code == B.PH_ERR_ARG
