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
