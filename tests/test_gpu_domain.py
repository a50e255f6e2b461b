"""The domain decomposition's local sets on one GPU: every domain of a cut
(computed by the library's host code, no collective) is run through the C
ABI on its own particles plus ghosts, one after another; the own particles'
forces must match the FP64 oracle of the whole box (the tolerance of the PP
parity tests) and the single-domain GPU result."""
import numpy as np
import pytest

from helpers import P99_TOL, MAX_TOL
from oracle import force
from test_domain import L, RCUT, RS, _particles

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_domains", [2, 5])
def test_local_sets_give_the_whole_box_forces(gpu_lib, n_domains):
    import torch
    B = gpu_lib
    pos, mass = _particles()
    prm = B.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    ns, cells = B.ph_domain_cells(pos, prm)
    owner, _ = B.ph_domain_partition(np.bincount(cells, minlength=ns ** 3), ns, B.PH_KEY_HILBERT, n_domains)
    whole = torch.zeros((len(pos), 3), device="cuda")
    lv, pr = B.ph_accel(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), prm, B.PH_G_EXACT, None, whole)
    torch.cuda.synchronize()
    whole = whole.cpu().numpy().astype(np.float64)
    ref = force.accel(pos, mass, L, 1.0, 1e-3, RS, RCUT)
    amag = np.linalg.norm(ref.acc, axis=1)
    tau = 1e-3 * np.median(amag)
    got = np.full((len(pos), 3), np.nan)
    for d in range(n_domains):
        need = B.ph_domain_halo(owner, ns, d)[cells]
        own, ghost = np.nonzero(need == 1)[0], np.nonzero(need == 2)[0]
        sel = np.concatenate([own, ghost])
        acc = torch.zeros((sel.size, 3), device="cuda")
        lv2, pr2 = B.ph_accel(torch.from_numpy(pos[sel]).cuda(), torch.from_numpy(mass[sel]).cuda(), prm,
                              B.PH_G_EXACT, None, acc)
        torch.cuda.synchronize()
        got[own] = acc.cpu().numpy()[:own.size]
        for h in (pr2, lv2):
            B.ph_free(h)
    assert not np.isnan(got).any()
    slack = ref.near_abs
    for a in (got, whole):
        e = np.maximum(np.linalg.norm(a - ref.acc, axis=1) - slack, 0) / np.maximum(amag, tau)
        assert np.percentile(e, 99) <= P99_TOL and e.max() <= MAX_TOL
    # the two GPU results differ only by summation order
    e = np.linalg.norm(got - whole, axis=1) / np.maximum(amag, tau)
    assert np.percentile(e, 99) <= P99_TOL
    for h in (pr, lv):
        B.ph_free(h)


def _one_rank_nccl(port, q):
    # one NCCL rank on the one GPU: the exchange (all_to_all_single on device
    # tensors) and ph_accel on the local set, as every rank of a real run does
    import os
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from paper_1802_09824_gb300 import binding as BB
    from paper_1802_09824_gb300 import domain
    from test_domain import L, RCUT, RS, _particles
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1)
    pos, mass = _particles()
    prm = BB.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    ids = torch.arange(len(pos), dtype=torch.int64, device="cuda")
    ids_own, acc_own, local = domain.accel_partitioned(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(),
                                                       ids, prm)
    q.put((ids_own.cpu().numpy(), acc_own.cpu().numpy(), local.n_owned))
    dist.destroy_process_group()


def test_partitioned_call_on_one_nccl_rank(gpu_lib):
    import os
    import torch
    import torch.multiprocessing as mp
    B = gpu_lib
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_one_rank_nccl, args=(29900 + os.getpid() % 1000, q))
    p.start()
    ids, acc, n_owned = q.get(timeout=300)
    p.join(timeout=60)
    assert p.exitcode == 0
    pos, mass = _particles()
    assert n_owned == len(pos) and np.array_equal(np.sort(ids), np.arange(len(pos)))
    prm = B.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    whole = torch.zeros((len(pos), 3), device="cuda")
    lv, pr = B.ph_accel(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), prm, B.PH_G_EXACT, None, whole)
    torch.cuda.synchronize()
    got = np.empty_like(acc)
    got[ids] = acc
    np.testing.assert_array_equal(got, whole.cpu().numpy())      # one rank: the same set, the same bits
    for h in (pr, lv):
        B.ph_free(h)


def test_device_cells_match_the_host(gpu_lib):
    import torch
    B = gpu_lib
    pos, _ = _particles()
    prm = B.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    shifted = pos.astype(np.float64) + np.array([1.0, -2.0, 0.0])    # outside the box: wrapped
    for p in (pos, pos.astype(np.float64), shifted):
        ns_h, cells_h = B.ph_domain_cells(p, prm)
        ns_d, cells_d, counts = B.ph_domain_cells_device(torch.from_numpy(np.ascontiguousarray(p)).cuda(), prm)
        assert ns_d == ns_h
        np.testing.assert_array_equal(cells_d.cpu().numpy(), cells_h)
        np.testing.assert_array_equal(counts.cpu().numpy(), np.bincount(cells_h, minlength=ns_h ** 3))


def _pack_reference(pos, mass, ids, cells, owner, ns, n_ranks):
    """The send rows the documented layout asks for (numpy)."""
    rows, counts = [], []
    for r in range(n_ranks):
        need = B_host.ph_domain_halo(owner, ns, r)[cells]
        idx = np.nonzero(need)[0]
        blk = np.empty((idx.size, 6))
        blk[:, :3] = pos[idx]
        blk[:, 3] = mass[idx]
        blk[:, 4] = need[idx]
        blk[:, 5] = ids[idx].view(np.float64)
        rows.append(blk)
        counts.append(idx.size)
    return np.concatenate(rows), counts


from paper_1802_09824_gb300 import binding as B_host   # noqa: E402  (host calls of the reference)


@pytest.mark.parametrize("n_ranks", [1, 3])
def test_device_exchange_between_simulated_ranks(gpu_lib, n_ranks):
    """Every rank's shard is packed on the device; the all-to-all is done by
    hand on the one GPU (destination r receives the segments for r of ranks
    0, 1, ... in order); the packed rows and the unpacked local sets match
    the layout computed here in numpy, and the local sets, run with their own
    particles active, give the own particles the whole box's forces."""
    import torch
    B = gpu_lib
    pos, mass = _particles()
    n = len(pos)
    ids = np.arange(n, dtype=np.int64) * 7 + 3
    prm = B.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    shards = np.array_split(np.random.default_rng(4).permutation(n), n_ranks)
    dev = [(torch.from_numpy(pos[s]).cuda(), torch.from_numpy(mass[s]).cuda(), torch.from_numpy(ids[s]).cuda())
           for s in shards]
    cells_dev, counts = [], None
    for p_, m_, i_ in dev:
        ns, c_, k_ = B.ph_domain_cells_device(p_, prm)
        cells_dev.append(c_)
        counts = k_ if counts is None else counts + k_
    owner, _ = B.ph_domain_partition(counts.cpu().numpy(), ns, B.PH_KEY_HILBERT, n_ranks)
    segs = []
    for (p_, m_, i_), c_, s in zip(dev, cells_dev, shards):
        send, sc = B.ph_domain_pack(p_, m_, i_, c_, owner, ns, n_ranks)
        ref, rcnt = _pack_reference(pos[s].astype(np.float64), mass[s].astype(np.float64), ids[s],
                                    c_.cpu().numpy(), owner, ns, n_ranks)
        assert sc == rcnt
        got = send[:sum(sc)].cpu().numpy()
        np.testing.assert_array_equal(got.view(np.uint64), ref.view(np.uint64))
        offs = np.concatenate([[0], np.cumsum(sc)])
        segs.append([send[offs[r]:offs[r + 1]] for r in range(n_ranks)])
    ref_all = force.accel(pos, mass, L, 1.0, 1e-3, RS, RCUT)
    amag = np.linalg.norm(ref_all.acc, axis=1)
    tau = 1e-3 * np.median(amag)
    got_acc = np.full((n, 3), np.nan)
    for r in range(n_ranks):
        recv = torch.cat([segs[q][r] for q in range(n_ranks)])
        lpos, lmass, lids, n_own = B.ph_domain_unpack(recv, recv.shape[0], torch.float32)
        rows = recv.cpu().numpy()
        own = rows[:, 4] == 1
        order = np.concatenate([np.nonzero(own)[0], np.nonzero(~own)[0]])
        assert n_own == int(own.sum())
        np.testing.assert_array_equal(lpos.cpu().numpy(), rows[order, :3].astype(np.float32))
        np.testing.assert_array_equal(lmass.cpu().numpy(), rows[order, 3].astype(np.float32))
        np.testing.assert_array_equal(lids.cpu().numpy(), rows[order, 5].view(np.int64))
        # the local set with its own particles active
        active = torch.zeros(lpos.shape[0], dtype=torch.uint8, device="cuda")
        active[:n_own] = 1
        lv = B.ph_build_leaves(lpos, lmass, prm)
        B.ph_leaves_set_active(lv, active)
        lv = B.ph_build_leaves(lpos, lmass, prm, leaves=lv)
        pr = B.ph_leaf_pairs(lv)
        acc = torch.full((lpos.shape[0], 3), float("nan"), device="cuda")
        B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
        torch.cuda.synchronize()
        a = acc.cpu().numpy()
        assert np.all(a[n_own:] == 0)                     # ghosts: no source lists, zero forces
        got_acc[(lids.cpu().numpy()[:n_own] - 3) // 7] = a[:n_own]
        for h in (pr, lv):
            B.ph_free(h)
    assert not np.isnan(got_acc).any()
    e = np.maximum(np.linalg.norm(got_acc - ref_all.acc, axis=1) - ref_all.near_abs, 0) / np.maximum(amag, tau)
    assert np.percentile(e, 99) <= P99_TOL and e.max() <= MAX_TOL


def _one_rank_step(port, q):
    # one NCCL rank on the one GPU: the device exchange and the captured
    # partitioned step, twice (capture, then replay)
    import os
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    from paper_1802_09824_gb300 import binding as BB
    from paper_1802_09824_gb300 import domain
    from test_domain import L, RCUT, RS, _particles
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1)
    pos, mass = _particles()
    prm = BB.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    ids = torch.arange(len(pos), dtype=torch.int64, device="cuda")
    step = domain.PartitionedStep(prm)
    out = []
    for _ in range(2):
        i_, a_ = step(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), ids)
        torch.cuda.synchronize()
        out.append((i_.cpu().numpy().copy(), a_.cpu().numpy().copy()))
    step.close()
    q.put(out)
    dist.destroy_process_group()


def test_partitioned_step_on_one_nccl_rank(gpu_lib):
    import os
    import torch
    import torch.multiprocessing as mp
    B = gpu_lib
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_one_rank_step, args=(30900 + os.getpid() % 1000, q))
    p.start()
    out = q.get(timeout=300)
    p.join(timeout=60)
    assert p.exitcode == 0
    pos, mass = _particles()
    prm = B.make_params(L, 1.0, 1e-3, RS, RCUT, 32)
    whole = torch.zeros((len(pos), 3), device="cuda")
    lv, pr = B.ph_accel(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), prm, B.PH_G_EXACT, None, whole)
    torch.cuda.synchronize()
    for ids, acc in out:
        assert np.array_equal(np.sort(ids), np.arange(len(pos)))
        got = np.empty_like(acc)
        got[ids] = acc
        np.testing.assert_array_equal(got, whole.cpu().numpy())   # one rank: the same set, the same bits
    for h in (pr, lv):
        B.ph_free(h)
