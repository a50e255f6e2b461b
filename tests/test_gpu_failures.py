"""Failure paths on the GPU, made on the host: the library's testing hook
(ph_debug_fail_allocation) makes a chosen device allocation fail exactly as
an out-of-memory error would.  No kernel faults, traps or hangs here: every
refusal happens on the host before a launch.

Checked: every allocation of a fresh step can fail, each time with
PH_ERR_OOM and without leaking device memory; a rebuild that fails part-way
leaves the handle invalid (PH_ERR_STATE from every call that would read it)
until it is built again, after which the step matches the FP64 oracle; a
pair list made for an older build of the leaves is refused; a captured graph
refuses to replay once the handles' buffers have moved; the PM and trainer
entry points recover after a failed allocation."""
import gc

import numpy as np
import pytest

from helpers import check_parity, oracle_accel
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _free_bytes():
    import torch
    gc.collect()
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _tensors(ps):
    import torch
    return (torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(),
            torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda"))


def _params(B, ps):
    bp = ps.boxes[0]
    return B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32)


@pytest.fixture(autouse=True)
def _hook_off(gpu_lib):
    yield
    gpu_lib.ph_debug_fail_allocation(-1)


def test_every_allocation_of_a_fresh_step_can_fail_without_leaking(gpu_lib):
    B = gpu_lib
    ps = synth.workload("uniform_small")
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps)
    lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_EXACT, None, acc)   # settles the context's own allocations
    ref = acc.cpu().numpy().copy()
    B.ph_free(pr)
    B.ph_free(lv)
    before = _free_bytes()
    failures = 0
    for k in range(500):
        B.ph_debug_fail_allocation(k)
        try:
            lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_EXACT, None, acc)
        except B.PhError as e:
            assert e.code == B.PH_ERR_OOM, str(e)
            assert "injected" in str(e)
            failures += 1
            continue
        # the step needs fewer than k + 1 allocations: it ran through
        B.ph_debug_fail_allocation(-1)
        np.testing.assert_array_equal(acc.cpu().numpy(), ref)
        B.ph_free(pr)
        B.ph_free(lv)
        break
    assert failures >= 30           # every buffer of the leaves and the pair list
    assert abs(_free_bytes() - before) <= 8 << 20


def test_a_failed_rebuild_leaves_the_handle_invalid_then_recovers(gpu_lib):
    import torch
    B = gpu_lib
    small = synth.workload("uniform_small", scale=1000)
    large = synth.workload("zeldovich_128", scale=24)
    ps_, pm_, acc_s = _tensors(small)
    pl, ml, acc_l = _tensors(large)
    lv = B.ph_build_leaves(ps_, pm_, _params(B, small))
    pr = B.ph_leaf_pairs(lv)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc_s)
    B.ph_debug_fail_allocation(0)        # growing to the larger set needs new buffers
    with pytest.raises(B.PhError) as ei:
        B.ph_build_leaves(pl, ml, _params(B, large), leaves=lv)
    assert ei.value.code == B.PH_ERR_OOM
    for call in (lambda: B.ph_leaf_pairs(lv, pairs=pr),
                 lambda: B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc_l),
                 lambda: B.ph_pp_accel(lv, None, B.PH_G_EXACT, None, acc_l),
                 lambda: B.ph_count_within(lv, pr),
                 lambda: B.ph_leaves_get_view(lv),
                 lambda: B.ph_graph_create(lv, pr, pl, ml, B.PH_G_EXACT, None, acc_l)):
        with pytest.raises(B.PhError) as ei:
            call()
        assert ei.value.code == B.PH_ERR_STATE
    # built again, the same handles give the oracle's forces
    lv = B.ph_build_leaves(pl, ml, _params(B, large), leaves=lv)
    # the old list was made for an earlier build
    with pytest.raises(B.PhError) as ei:
        B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc_l)
    assert ei.value.code == B.PH_ERR_STATE
    pr = B.ph_leaf_pairs(lv, pairs=pr)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc_l)
    torch.cuda.synchronize()
    check_parity(acc_l.cpu().numpy(), oracle_accel(large))
    # a pair list whose growth fails is refused until it is made again
    lv = B.ph_build_leaves(ps_, pm_, _params(B, small), leaves=lv)
    pr = B.ph_leaf_pairs(lv, pairs=pr)
    pr2 = B.ph_leaf_pairs(lv)                                         # a list sized for the small set
    lv = B.ph_build_leaves(pl, ml, _params(B, large), leaves=lv)      # no growth: these buffers fit already
    B.ph_debug_fail_allocation(0)
    with pytest.raises(B.PhError) as ei:
        B.ph_leaf_pairs(lv, pairs=pr2)                                # grows: fails
    assert ei.value.code == B.PH_ERR_OOM
    with pytest.raises(B.PhError) as ei:
        B.ph_pp_accel(lv, pr2, B.PH_G_EXACT, None, acc_l)
    assert ei.value.code == B.PH_ERR_STATE
    pr2 = B.ph_leaf_pairs(lv, pairs=pr2)
    B.ph_pp_accel(lv, pr2, B.PH_G_EXACT, None, acc_l)
    torch.cuda.synchronize()
    check_parity(acc_l.cpu().numpy(), oracle_accel(large))
    for h in (pr2, pr, lv):
        B.ph_free(h)


def test_a_graph_refuses_to_replay_after_its_buffers_moved(gpu_lib):
    import torch
    B = gpu_lib
    small = synth.workload("uniform_small", scale=1000)
    large = synth.workload("uniform_small")
    pos, mass, acc = _tensors(small)
    lv = B.ph_build_leaves(pos, mass, _params(B, small))
    pr = B.ph_leaf_pairs(lv)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc)
    B.ph_graph_launch(g)
    torch.cuda.synchronize()
    pl, ml, al = _tensors(large)
    lv = B.ph_build_leaves(pl, ml, _params(B, large), leaves=lv)      # larger: the buffers move
    with pytest.raises(B.PhError) as ei:
        B.ph_graph_launch(g)
    assert ei.value.code == B.PH_ERR_STATE
    for h in (g, pr, lv):
        B.ph_free(h)


def test_pm_and_trainer_recover_after_a_failed_allocation(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("uniform_small")
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps)
    h = B.ph_pm_accel(pos, mass, prm, 32, acc)
    torch.cuda.synchronize()
    ref = acc.cpu().numpy().copy()
    B.ph_free(h)
    before = _free_bytes()
    B.ph_debug_fail_allocation(2)
    with pytest.raises(B.PhError) as ei:
        B.ph_pm_accel(pos, mass, prm, 32, acc)
    assert ei.value.code == B.PH_ERR_OOM
    assert abs(_free_bytes() - before) <= 8 << 20
    acc.zero_()
    h = B.ph_pm_accel(pos, mass, prm, 32, acc)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(acc.cpu().numpy(), ref)
    # a failure inside an existing handle's mesh set-up (a new mesh size)
    B.ph_debug_fail_allocation(1)
    with pytest.raises(B.PhError) as ei:
        B.ph_pm_accel(pos, mass, prm, 64, acc, pm=h)
    assert ei.value.code == B.PH_ERR_OOM
    acc.zero_()
    h = B.ph_pm_accel(pos, mass, prm, 32, acc, pm=h)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(acc.cpu().numpy(), ref)
    B.ph_free(h)
    bp = ps.boxes[0]
    tp = B.make_train_params(n_samples=10_000, batch=1024, steps=10)
    B.ph_debug_fail_allocation(3)
    with pytest.raises(B.PhError) as ei:
        B.ph_mlp_train(tp, bp.rs, bp.rcut)
    assert ei.value.code == B.PH_ERR_OOM
    m = B.ph_mlp_train(tp, bp.rs, bp.rcut)
    B.ph_free(m)
