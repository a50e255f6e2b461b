"""GPU tree build (keys, sort, leaves, groups, frames, pair list) against the
oracle: bit-exact for the integer and index work."""
import numpy as np
import pytest

from oracle import keys as K
from oracle import tree as T
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _set(n=3000, seed=11, clustered=False, L=1.0):
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3)) * L
    if clustered:
        m = n // 2
        p[:m] = L * 0.3 + L * 0.01 * rng.standard_normal((m, 3))
        p = np.mod(p, L)
    p = p.astype(np.float32)
    p[p >= np.float32(L)] = 0
    rs = 1.25 / 32 * L
    bp = synth.BoxParams(L=L, G=1.0, eps=1e-3 * L, rs=rs, rcut=4.5 * rs, leaf_max=16)
    return synth._single(p, np.full(n, 1.0 / n, np.float32), bp, "t")


def _snapped(centre, half):
    lo, hi = centre - half, centre + half
    U = np.ldexp(1.0, np.frexp(np.maximum(np.abs(lo), np.abs(hi)))[1] - 24)
    ref = np.rint(centre / U) * U
    return ref, np.maximum(hi - ref, ref - lo)


def _build(B, ps, kind=0, leaf_max=16, level_bits=1, group_size=32):
    import torch
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, leaf_max, kind, group_size, level_bits)
    lv = B.ph_build_leaves(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(), prm)
    torch.cuda.synchronize()
    return lv, B.ph_leaves_get_view(lv)


@pytest.mark.parametrize("level_bits", [1, 3])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("clustered", [False, True])
@pytest.mark.parametrize("n", [1, 2, 33, 3000, 20000])
def test_keys_sort_leaves_groups_bit_exact(gpu_lib, kind, clustered, n, level_bits):
    B = gpu_lib
    ps = _set(n=n, clustered=clustered)
    gs = (8, 16, 32)[n % 3]
    lv, v = _build(B, ps, kind, level_bits=level_bits, group_size=gs)
    t = T.BoxTree(ps.pos, 1.0, ps.boxes[0].rcut, 16, gs, kind, T=v["key_bits"], level_bits=level_bits)
    assert v["n_leaves"] == len(t.leaf_first) - 1
    assert v["n_groups"] == len(t.group_first) - 1
    np.testing.assert_array_equal(v["keys"].cpu().numpy().astype(np.uint64), t.keys)
    np.testing.assert_array_equal(v["perm"].cpu().numpy(), t.order)
    np.testing.assert_array_equal(v["leaf_first"].cpu().numpy(), t.leaf_first)
    np.testing.assert_array_equal(v["group_first"].cpu().numpy(), t.group_first)
    # reference points: box centres snapped to the FP32 spacing of the box's
    # largest coordinate
    lc, lh = _snapped(*t.leaf_boxes())
    np.testing.assert_array_equal(v["leaf_ref"].cpu().numpy(), lc)
    half = v["leaf_half"].cpu().numpy()[:, :3].astype(np.float64)
    assert np.all(half >= lh) and np.all(half <= lh * (1 + 2 ** -23) + 1e-300)
    gc, gh = _snapped(*t.group_boxes())
    np.testing.assert_array_equal(v["group_ref"].cpu().numpy(), gc)
    # leaf-relative FP32 positions: one rounding of the FP64 difference
    pl = v["pos_leaf"].cpu().numpy()
    li = t.particle_leaf()
    np.testing.assert_array_equal(pl[:, :3], (t.xw - lc[li]).astype(np.float32))
    np.testing.assert_array_equal(pl[:, 3], ps.mass[t.order])
    # group frame = leaf frame + FP32(offset), the source shift of the PP kernel
    pg = v["pos_group"].cpu().numpy()
    gi = t.particle_group()
    off = (lc[li] - gc[gi]).astype(np.float32)
    np.testing.assert_array_equal(pg[:, :3], pl[:, :3] + off)
    B.ph_free(lv)


def test_coincident_particles_chunk(gpu_lib):
    p = np.tile(np.array([[0.1, 0.2, 0.3]], np.float32), (70, 1))
    bp = synth.BoxParams(L=1.0, G=1.0, eps=1e-3, rs=1.25 / 32, rcut=4.5 * 1.25 / 32, leaf_max=32)
    ps = synth._single(p, np.full(70, 1 / 70, np.float32), bp, "c")
    for lb in (1, 3):
        lv, v = _build(gpu_lib, ps, 0, leaf_max=32, level_bits=lb)
        assert v["leaf_first"].cpu().numpy().tolist() == [0, 32, 64, 70]
        gpu_lib.ph_free(lv)


@pytest.mark.parametrize("level_bits", [1, 3])
@pytest.mark.parametrize("clustered", [False, True])
@pytest.mark.parametrize("L,rcut", [(1.0, 0.17578125), (1.0, 0.3)])
def test_pair_list_matches_box_relation(gpu_lib, clustered, L, rcut, level_bits):
    import torch
    B = gpu_lib
    ps = _set(n=4000, clustered=clustered, L=L)
    bp = ps.boxes[0]
    prm = B.make_params(L, 1.0, bp.eps, rcut / 4.5, rcut, 16, 0, 0, level_bits)
    lv = B.ph_build_leaves(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(), prm)
    pr = B.ph_leaf_pairs(lv)
    torch.cuda.synchronize()
    v = B.ph_leaves_get_view(lv)
    pv = B.ph_pairs_get_view(pr)
    t = T.BoxTree(ps.pos, L, rcut, 16, 32, 0, T=v["key_bits"], level_bits=level_bits)
    lc, _ = _snapped(*t.leaf_boxes())
    gc, _ = _snapped(*t.group_boxes())
    off = pv["group_off"].cpu().numpy()
    ent = pv["entries"].cpu().numpy()
    first = ent[:, 3].view(np.int32)
    leaf = np.searchsorted(t.leaf_first, first)
    np.testing.assert_array_equal(t.leaf_first[leaf], first)
    np.testing.assert_array_equal(pv["counts"].cpu().numpy().astype(np.int64) + 1,
                                  t.leaf_first[leaf + 1] - t.leaf_first[leaf])
    got = set()
    for g in range(len(off) - 1):
        for e in range(off[g], off[g + 1]):
            l = int(leaf[e])
            s = np.rint((ent[e, :3].astype(np.float64) - (lc[l] - gc[g])) / L).astype(int)
            # the stored offset is the FP64 difference rounded once to FP32
            exp = (lc[l] + s * L - gc[g]).astype(np.float32)
            np.testing.assert_array_equal(ent[e, :3], exp)
            got.add((g, l, *s.tolist()))
    need = t.pair_set()
    allowed = t.pair_set(slack=1e-4)
    assert need <= got, f"{len(need - got)} required pairs missing"
    assert got <= allowed, f"{len(got - allowed)} pairs beyond rcut(1+1e-4)"
    B.ph_free(pr)
    B.ph_free(lv)


def test_batched_build_equals_per_box(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.batch_boxes(5, seed=99, n_min=300, n_max=3000)
    prms = [B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32) for bp in ps.boxes]
    lv = B.ph_build_leaves_batched(torch.from_numpy(ps.pos).cuda(), torch.from_numpy(ps.mass).cuda(),
                                   ps.offsets, prms)
    torch.cuda.synchronize()
    v = B.ph_leaves_get_view(lv)
    lf = v["leaf_first"].cpu().numpy()
    perm = v["perm"].cpu().numpy()
    T_ = v["key_bits"]
    base_leaf = 0
    for b in range(5):
        sl = ps.box_slice(b)
        t = T.BoxTree(ps.pos[sl], 1.0, ps.boxes[b].rcut, 32, 32, 0, T=T_, box_index=b)
        nlb = len(t.leaf_first) - 1
        np.testing.assert_array_equal(lf[base_leaf:base_leaf + nlb + 1], t.leaf_first + sl.start)
        np.testing.assert_array_equal(perm[sl], t.order + sl.start)
        base_leaf += nlb
    assert base_leaf == v["n_leaves"]
    B.ph_free(lv)
