"""Batched boxes, the graph-captured step, kernel variants and the autotuner."""
import numpy as np
import pytest

from helpers import check_parity, gpu_accel, oracle_accel
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _tensors(ps):
    import torch
    return (torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(),
            torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda"))


def _params(B, ps, **kw):
    return [B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, kw.get("leaf_max", 32), 0, 0,
                          kw.get("level_bits", 0), kw.get("pp_variant", 0)) for bp in ps.boxes]


@pytest.mark.parametrize("nboxes", [1, 12])
def test_graph_replay_matches_direct_calls(gpu_lib, nboxes):
    import torch
    B = gpu_lib
    ps = (synth.workload("uniform_small", scale=5000) if nboxes == 1
          else synth.batch_boxes(nboxes, seed=5, n_min=300, n_max=5000))
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps)
    lv = B.ph_build_leaves_batched(pos, mass, ps.offsets, prm)
    pr = B.ph_leaf_pairs(lv)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    direct = acc.cpu().numpy().copy()
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25)
    assert B.ph_graph_kernels(g) > 10
    for _ in range(2):
        acc.zero_()
        B.ph_graph_launch(g)
        torch.cuda.synchronize()
        B.ph_status(pr)
        np.testing.assert_array_equal(acc.cpu().numpy(), direct)
    # new positions written in place are picked up by the next replay
    rng = np.random.default_rng(3)
    moved = ps.pos + rng.uniform(-1e-3, 1e-3, ps.pos.shape).astype(np.float32)
    moved = np.mod(moved, 1.0).astype(np.float32)
    pos.copy_(torch.from_numpy(moved))
    B.ph_graph_launch(g)
    torch.cuda.synchronize()
    B.ph_status(pr)
    ps2 = synth.ParticleSet(moved, ps.mass, ps.boxes, ps.offsets, "moved")
    for b in range(min(nboxes, 3)):
        sl = ps2.box_slice(b)
        check_parity(acc.cpu().numpy()[sl], oracle_accel(ps2, box=b))
    for h in (g, pr, lv):
        B.ph_free(h)


def test_graph_capacity_overflow_is_latched(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("uniform_small", scale=6000)
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps)
    lv = B.ph_build_leaves(pos, mass, prm[0])
    pr = B.ph_leaf_pairs(lv)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.0)
    # the same particles squeezed into a corner need many more leaf pairs
    squeezed = (ps.pos * 0.15).astype(np.float32)
    pos.copy_(torch.from_numpy(squeezed))
    B.ph_graph_launch(g)
    torch.cuda.synchronize()
    with pytest.raises(B.PhError) as ei:
        B.ph_status(pr)
    assert ei.value.code == B.PH_ERR_CAPACITY
    B.ph_free(g)
    # rebuilding sizes the list again and the result is right
    lv = B.ph_build_leaves(pos, mass, prm[0], leaves=lv)
    pr2 = B.ph_leaf_pairs(lv)
    B.ph_pp_accel(lv, pr2, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    sq = synth._single(squeezed, ps.mass, ps.boxes[0], "sq")
    check_parity(acc.cpu().numpy(), oracle_accel(sq))
    for h in (pr2, pr, lv):
        B.ph_free(h)


def test_graph_replay_with_host_buffers(gpu_lib):
    # ph_graph_launch_host: host positions and masses copied in, the step
    # replayed, accelerations copied out -- the same bits as a device replay,
    # from pinned and from pageable host memory; an overflow is reported
    import torch
    B = gpu_lib
    ps = synth.workload("uniform_small", scale=5000)
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps)
    lv = B.ph_build_leaves(pos, mass, prm[0])
    pr = B.ph_leaf_pairs(lv)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.1)
    B.ph_graph_launch(g)
    torch.cuda.synchronize()
    ref = acc.cpu().numpy().copy()
    pos.zero_()                                  # the host replay must bring the positions back
    for pinned in (True, False):
        hp = torch.from_numpy(ps.pos.copy())
        hm = torch.from_numpy(ps.mass.copy())
        ha = torch.full((ps.n, 3), float("nan"))
        if pinned:
            hp, hm, ha = hp.pin_memory(), hm.pin_memory(), ha.pin_memory()
        B.ph_graph_launch_host(g, hp, hm, ha)
        np.testing.assert_array_equal(ha.numpy(), ref)
    check_parity(ref, oracle_accel(ps))
    squeezed = torch.from_numpy((ps.pos * 0.15).astype(np.float32))
    with pytest.raises(B.PhError) as ei:
        B.ph_graph_launch_host(g, squeezed, None, torch.zeros((ps.n, 3)))
    assert ei.value.code == B.PH_ERR_CAPACITY
    for h in (g, pr, lv):
        B.ph_free(h)


def test_overlapped_host_replays_on_two_streams(gpu_lib):
    # ph_graph_launch_host_async: two graphs over separate handles and
    # buffers, replayed alternately on two streams from pinned host buffers
    # holding two different particle sets; every step's result equals a
    # synchronous replay of the same set, bit for bit
    import torch
    B = gpu_lib
    ps = synth.workload("uniform_small", scale=5000)
    prm = _params(B, ps)[0]
    rng = np.random.default_rng(8)
    inputs = [ps.pos.copy(), np.mod(ps.pos + rng.uniform(0, 0.01, ps.pos.shape), 1.0).astype(np.float32)]
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    sets, refs = [], []
    for i in range(2):
        pos, mass, acc = _tensors(ps)
        pos.copy_(torch.from_numpy(inputs[i]))
        torch.cuda.synchronize()
        lv = B.ph_build_leaves(pos, mass, prm, streams[i])
        pr = B.ph_leaf_pairs(lv, streams[i])
        g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25, stream=streams[i])
        hp = torch.from_numpy(inputs[i].copy()).pin_memory()
        hm = torch.from_numpy(ps.mass.copy()).pin_memory()
        ha = torch.full((ps.n, 3), float("nan")).pin_memory()
        B.ph_graph_launch_host(g, hp, hm, ha, streams[i])
        refs.append(ha.numpy().copy())
        sets.append((g, pr, lv, hp, hm, ha, streams[i]))
    assert not np.array_equal(refs[0], refs[1])
    for k in range(6):
        g, pr, lv, hp, hm, ha, s = sets[k % 2]
        B.ph_graph_launch_host_async(g, hp, hm, ha, s)
    torch.cuda.synchronize()
    for i in range(2):
        g, pr, lv, hp, hm, ha, s = sets[i]
        B.ph_status(lv)
        B.ph_status(pr)
        np.testing.assert_array_equal(ha.numpy(), refs[i])
        for h in (g, pr, lv):
            B.ph_free(h)


@pytest.mark.parametrize("gs", [8, 16, 32])
def test_group_sizes_match_the_oracle(gpu_lib, gs):
    ps = synth.workload("zeldovich_128", scale=32)
    got, lv, pr = gpu_accel(gpu_lib, ps, group_size=gs)
    check_parity(got, oracle_accel(ps))
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)
    nfw = synth.workload("nfw_mix_256", scale=20)
    got, lv, pr = gpu_accel(gpu_lib, nfw, group_size=gs, level_bits=3)
    check_parity(got, oracle_accel(nfw))
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_kernel_variants_give_identical_forces(gpu_lib):
    ps = synth.workload("nfw_mix_256", scale=24)
    a, l1, p1 = gpu_accel(gpu_lib, ps)
    import torch
    B = gpu_lib
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps, pp_variant=1)
    lv = B.ph_build_leaves(pos, mass, prm[0])
    pr = B.ph_leaf_pairs(lv)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(acc.cpu().numpy(), a)
    for h in (pr, lv, p1, l1):
        B.ph_free(h)


def _queue_keys(view):
    """The documented queue key of every group, restated on the host from
    the list: a group's cost is the source particles of its entries (a leaf
    entry holds count + 1 particles, a mass-centre entry one); the key is 255
    minus its quarter-octave class (0 for cost 0, else 1 + 4 e + f with
    2^e <= cost < 2^(e+1) and f the two bits below the leading one)."""
    off = view["group_off"].cpu().numpy()
    per_entry = view["counts"].cpu().numpy().astype(np.int64) + 1
    csum = np.concatenate([[0], np.cumsum(per_entry)])
    cost = csum[off[1:]] - csum[off[:-1]]
    key = np.full(cost.size, 255, np.int64)
    for g, c in enumerate(cost.tolist()):
        if c > 0:
            e = int(c).bit_length() - 1
            f = (c >> (e - 2)) & 3 if e >= 2 else (c << (2 - e)) & 3
            key[g] = 255 - (1 + 4 * e + f)
    return key, cost


@pytest.mark.parametrize("case", ["batch", "nfw_tree"])
def test_queue_takes_groups_by_decreasing_cost(gpu_lib, case):
    import torch
    B = gpu_lib
    if case == "batch":
        ps = synth.batch_boxes(12, seed=7, n_min=300, n_max=6000)
        theta = 0.0
    else:
        ps = synth.workload("nfw_mix_256", scale=24)
        theta = 0.3
    pos, mass, acc = _tensors(ps)
    outs = []
    for order in (0, 1):
        prm = [B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, theta=theta,
                             queue_order=order) for bp in ps.boxes]
        lv = B.ph_build_leaves_batched(pos, mass, ps.offsets, prm)
        pr = B.ph_leaf_pairs(lv)
        B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
        torch.cuda.synchronize()
        outs.append(acc.cpu().numpy().copy())
        v = B.ph_pairs_get_view(pr)
        if order == 0:
            key, cost = _queue_keys(v)
            got = v["group_order"].cpu().numpy()
            # a permutation of the groups in non-decreasing key (decreasing cost class)
            np.testing.assert_array_equal(np.sort(got), np.arange(key.size))
            assert np.all(np.diff(key[got]) >= 0)
            assert np.all(np.diff(cost[got]) <= cost[got][:-1] * 0.25 + 1e-9)   # within a class: < 25 %
            assert not np.array_equal(got, np.arange(got.size))                 # the case is reordered
        else:
            assert v["group_order"] is None
        for h in (pr, lv):
            B.ph_free(h)
    # the order changes which warp takes a group, not the sums
    np.testing.assert_array_equal(outs[0], outs[1])


def test_autotuner_picks_a_tried_candidate(gpu_lib, tmp_path):
    import torch
    B = gpu_lib
    from paper_1802_09824_gb300 import tuning
    ps = synth.workload("zeldovich_128", scale=32)
    pos, mass, acc = _tensors(ps)
    prm = _params(B, ps)
    res = B.ph_autotune(pos, mass, ps.offsets, prm, reps=1)
    assert res.n_tried == 24
    ms = np.array(res.ms[:res.n_tried])
    assert np.all(ms > 0) and abs(res.best_ms - ms.min()) < 1e-6
    k = int(np.argmin(ms))
    assert (res.best.leaf_max, res.best.level_bits, res.best.pp_variant, res.best.group_size, res.best.key_kind) == (
        res.leaf_max[k], res.level_bits[k], res.pp_variant[k], res.group_size[k], res.key_kind[k])
    p2, info = tuning.tuned(B, pos, mass, ps.offsets, _params(B, ps), reps=1, path=str(tmp_path / "t.json"))
    assert info["cache"] == "miss"
    got, lv, pr = gpu_accel(B, ps, leaf_max=p2[0].leaf_max, level_bits=p2[0].level_bits,
                            group_size=p2[0].group_size, key_kind=p2[0].key_kind)
    check_parity(got, oracle_accel(ps))
    B.ph_free(pr)
    B.ph_free(lv)
