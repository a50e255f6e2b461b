"""The leaf-level tree part on the GPU (theta > 0): accepted leaves enter the
pair list as one mass-centre particle each; parity with the oracle of the
same approximation, theta = 0 identical to the plain path."""
import numpy as np
import pytest

from helpers import check_parity
from oracle import dtt, force
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(B, ps, theta, leaf_max=16, gs=0, g_mode=None):
    import torch
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, leaf_max, 0, gs, 0, 0, theta)
    lv = B.ph_build_leaves(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(), prm)
    pr = B.ph_leaf_pairs(lv)
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT if g_mode is None else g_mode, None, acc)
    torch.cuda.synchronize()
    v = B.ph_leaves_get_view(lv)
    pv = B.ph_pairs_get_view(pr)
    first = pv["entries"].cpu().numpy()[:, 3].copy().view(np.int32)
    n_mono = int(np.sum(first >= ps.n))
    out = acc.cpu().numpy(), n_mono, v["key_bits"], B.ph_pp_counters(pr)
    B.ph_free(pr)
    B.ph_free(lv)
    return out


def test_theta_zero_is_the_plain_path(gpu_lib):
    ps = synth.workload("nfw_mix_256", scale=20)
    a0, n0, _, c0 = _run(gpu_lib, ps, 0.0)
    assert n0 == 0
    import torch
    B = gpu_lib
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 16)
    lv = B.ph_build_leaves(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(), prm)
    pr = B.ph_leaf_pairs(lv)
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a0, acc.cpu().numpy())
    B.ph_free(pr)
    B.ph_free(lv)


@pytest.mark.parametrize("name,scale,theta,leaf_max,gs", [
    ("nfw_mix_256", 20, 0.3, 16, 0),
    ("nfw_mix_256", 24, 0.5, 8, 16),
    ("zeldovich_128", 24, 0.6, 8, 8),
])
def test_tree_part_matches_its_oracle(gpu_lib, name, scale, theta, leaf_max, gs):
    """The oracle decides acceptance in FP64 from the exact boxes (both
    opening angles of Sec. 3.3); the kernel decides in FP32 from its stored
    boxes.  Pairs within the oracle's ambiguity band of the threshold may go
    either way: their whole difference (mass-centre body against the leaf's
    PP sum) is admitted, like pairs within rounding of R_cut."""
    ps = synth.workload(name, scale=scale)
    got, n_mono, T, _ = _run(gpu_lib, ps, theta, leaf_max, gs)
    bp = ps.boxes[0]
    r = dtt.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, theta, leaf_max=leaf_max,
                  group_size=gs or 32, T=T)
    assert n_mono > 0 and r.n_accepted > 0
    # the GPU list also holds pairs within the box test's margin beyond rcut,
    # which contribute nothing either way; the accepted pairs within rcut
    # agree up to the ambiguous ones
    assert r.n_accepted - r.n_ambiguous <= n_mono <= 1.02 * (r.n_accepted + r.n_ambiguous) + 10
    assert r.n_ambiguous <= 1e-3 * r.n_accepted + 10
    res = force.AccelResult(acc=r.acc, abs_sum=None, n_within=None, near_abs=r.near_abs + r.amb_abs)
    check_parity(got, res)


def test_tree_part_with_the_tabulated_factor(gpu_lib):
    """The tree part's mass-centre bodies go through the PP kernel like any
    source, so the tabulated factor (Sec. 3.1's table) applies to them too:
    the same parity with the tree oracle (exact factor), the table's own
    error (~6e-7 of a term) far inside the tolerance."""
    ps = synth.workload("nfw_mix_256", scale=20)
    got, n_mono, T, _ = _run(gpu_lib, ps, 0.3, 16, 0, g_mode=gpu_lib.PH_G_TABLE)
    bp = ps.boxes[0]
    r = dtt.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 0.3, leaf_max=16, group_size=32, T=T)
    assert n_mono > 0 and r.n_accepted > 0
    res = force.AccelResult(acc=r.acc, abs_sum=None, n_within=None, near_abs=r.near_abs + r.amb_abs)
    check_parity(got, res)
