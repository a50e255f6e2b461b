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
