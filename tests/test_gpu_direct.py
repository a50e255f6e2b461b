"""The direct mode of the PP kernel (pairs = NULL): the leaf pairs are found
in the kernel with the pair builder's test and order, so the forces and the
work counters equal those over the stored list bit for bit."""
import numpy as np
import pytest

from helpers import check_parity, oracle_accel
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _both(B, ps, host=False, **kw):
    import torch
    prms = [B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, kw.get("leaf_max", bp.leaf_max), kw.get("key", 0),
                          kw.get("gs", 0), kw.get("lb", 0), kw.get("pv", 0)) for bp in ps.boxes]
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    if len(prms) == 1:
        lv = B.ph_build_leaves(pos, mass, prms[0])
    else:
        lv = B.ph_build_leaves_batched(pos, mass, ps.offsets, prms)
    pr = B.ph_leaf_pairs(lv)
    dev = "cpu" if host else "cuda"
    a_list = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    a_direct = torch.full((ps.n, 3), 7.0, dtype=torch.float32, device=dev)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, a_list)
    c_list = B.ph_pp_counters(pr)
    B.ph_pp_accel(lv, None, B.PH_G_EXACT, None, a_direct)
    c_direct = B.ph_pp_counters(lv)
    torch.cuda.synchronize()
    out = a_list.cpu().numpy(), a_direct.cpu().numpy(), c_list, c_direct
    B.ph_free(pr)
    B.ph_free(lv)
    return out


@pytest.mark.parametrize("name,scale,kw", [
    ("zeldovich_128", 32, {}),
    ("zeldovich_128", 32, {"gs": 16, "key": 1}),
    ("nfw_mix_256", 20, {"lb": 3, "gs": 8}),
    ("nfw_mix_256", 20, {"pv": 1, "leaf_max": 64}),
    ("uniform_small", 3000, {"leaf_max": 1}),
])
def test_direct_mode_equals_the_list_bit_for_bit(gpu_lib, name, scale, kw):
    ps = synth.workload(name, scale=scale)
    a_list, a_direct, c_list, c_direct = _both(gpu_lib, ps, **kw)
    np.testing.assert_array_equal(a_direct, a_list)
    assert c_direct == c_list
    check_parity(a_direct, oracle_accel(ps))


def test_direct_mode_batched_boxes_and_host_buffer(gpu_lib):
    ps = synth.batch_boxes(7, seed=21, n_min=200, n_max=5000)
    a_list, a_direct, c_list, c_direct = _both(gpu_lib, ps, host=True)
    np.testing.assert_array_equal(a_direct, a_list)
    assert c_direct == c_list
    for b in range(3):
        check_parity(a_direct[ps.box_slice(b)], oracle_accel(ps, box=b))


def test_direct_graph_replays_match_direct_calls(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("zeldovich_128", scale=24)
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, 1)
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    lv = B.ph_build_leaves(pos, mass, prm)
    B.ph_pp_accel(lv, None, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    ref = acc.cpu().numpy().copy()
    g = B.ph_graph_create(lv, None, pos, mass, B.PH_G_EXACT, None, acc)
    for _ in range(2):
        acc.zero_()
        B.ph_graph_launch(g)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(acc.cpu().numpy(), ref)
    B.ph_status(lv)
    check_parity(ref, oracle_accel(ps))
    B.ph_free(g)
    B.ph_free(lv)


def test_direct_mode_refuses_the_learned_factor(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("uniform_small", scale=500)
    bp = ps.boxes[0]
    from oracle import mlp as M
    m = B.ph_mlp_create(M.init_params(1).astype(np.float32), bp.rs, bp.rcut, tol=1.0)
    lv = B.ph_build_leaves(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(),
                           B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32))
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.PhError) as ei:
        B.ph_pp_accel(lv, None, B.PH_G_LEARNED, m, acc)
    assert ei.value.code == B.PH_ERR_ARG
    B.ph_free(lv)
    B.ph_free(m)


@pytest.mark.parametrize("name,scale,gs", [("zeldovich_128", 32, 0), ("nfw_mix_256", 20, 16),
                                            ("uniform_small", 3000, 8)])
def test_tabulated_factor_matches_the_oracle(gpu_lib, name, scale, gs):
    """PH_G_TABLE (the factor at 4097 nodes, nearest node plus slope): parity
    with the FP64 oracle and closeness to the exact factor on the same lists."""
    import torch
    B = gpu_lib
    ps = synth.workload(name, scale=scale)
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, 0, gs)
    lv = B.ph_build_leaves(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(), prm)
    pr = B.ph_leaf_pairs(lv)
    a_ex = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    a_tb = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, a_ex)
    c_ex = B.ph_pp_counters(pr)
    B.ph_pp_accel(lv, pr, B.PH_G_TABLE, None, a_tb)
    c_tb = B.ph_pp_counters(pr)
    torch.cuda.synchronize()
    assert c_tb == c_ex
    got, ex = a_tb.cpu().numpy(), a_ex.cpu().numpy()
    check_parity(got, oracle_accel(ps))
    mag = np.maximum(np.linalg.norm(ex, axis=1, keepdims=True), 1e-30)
    assert np.max(np.abs(got - ex) / mag) < 1e-3
    B.ph_free(pr)
    B.ph_free(lv)


def test_tabulated_factor_needs_one_rcut(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.batch_boxes(3, seed=4, n_min=300, n_max=800)
    prms = [B.make_params(bp.L, bp.G, bp.eps, bp.rs * (1 + 0.1 * k), bp.rcut * (1 + 0.1 * k), 32)
            for k, bp in enumerate(ps.boxes)]
    lv = B.ph_build_leaves_batched(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(), ps.offsets,
                                   prms)
    pr = B.ph_leaf_pairs(lv)
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.PhError) as ei:
        B.ph_pp_accel(lv, pr, B.PH_G_TABLE, None, acc)
    assert ei.value.code == B.PH_ERR_ARG
    B.ph_free(pr)
    B.ph_free(lv)
