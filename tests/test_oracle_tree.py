"""Pins of the oracle's keys, leaves, groups and cutoff pair relation."""
import itertools

import numpy as np
import pytest

from oracle import keys as K
from oracle import tree as T
from oracle import force


# ------------------------------------------------------------------ keys
def _grid(bits):
    n = 1 << bits
    c = np.array(list(itertools.product(range(n), repeat=3)), np.int64)
    return c


def test_morton_small_values():
    assert int(K.morton3(1, 0, 0, 1)) == 4
    assert int(K.morton3(0, 1, 0, 1)) == 2
    assert int(K.morton3(0, 0, 1, 1)) == 1
    assert int(K.morton3(3, 0, 0, 2)) == 0b100100
    assert int(K.morton3(2, 1, 3, 2)) == 0b101011


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("bits", [1, 2, 3])
def test_keys_bijective_and_octree_contiguous(kind, bits):
    c = _grid(bits)
    f = K.morton3 if kind == 0 else K.hilbert3
    k = f(c[:, 0], c[:, 1], c[:, 2], bits).astype(np.int64)
    assert sorted(k.tolist()) == list(range(8 ** bits))
    # every aligned sub-cube of side 2^l is one contiguous key range (the
    # octree property the paper relies on, Sec. 3.2)
    for lvl in range(bits + 1):
        side = 1 << lvl
        cell = (c // side)
        cid = (cell[:, 0] * 64 + cell[:, 1]) * 64 + cell[:, 2]
        for v in np.unique(cid):
            ks = np.sort(k[cid == v])
            assert ks[-1] - ks[0] + 1 == ks.size == side ** 3
            assert ks[0] % (side ** 3) == 0


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_steps_are_face_adjacent(bits):
    c = _grid(bits)
    k = K.hilbert3(c[:, 0], c[:, 1], c[:, 2], bits).astype(np.int64)
    path = c[np.argsort(k)]
    steps = np.abs(np.diff(path, axis=0)).sum(axis=1)
    assert np.all(steps == 1)
    assert k[0] == 0      # the curve starts at the origin cell


def test_ground_level_and_quantise():
    assert K.ground_level(1.0, 0.17578125) == 2          # N_side = 4
    assert K.ground_level(100.0, 4.39453125) == 4        # N_side = 16
    assert K.ground_level(200.0, 4.39453125) == 5
    for L, rc in [(1.0, 0.17578125), (100.0, 4.39453125), (3.0, 1.4)]:
        g = K.ground_level(L, rc)
        assert L / 2 ** g >= rc and (g == K.G_MAX or L / 2 ** (g + 1) < rc)
    q = K.quantise(np.array([0.0, 0.999999999, 1.0, -1e-300]), 1.0, 4)
    assert q.tolist() == [0, 15, 15, 0]


def test_keys_box_prefix_orders_boxes():
    rng = np.random.default_rng(1)
    p = rng.random((50, 3))
    k0, _, _ = K.particle_keys(p, 1.0, 0.17578125, 20, 0, box_index=0)
    k1, _, _ = K.particle_keys(p, 1.0, 0.17578125, 20, 0, box_index=1)
    assert k0.max() < k1.min()


# ------------------------------------------------------------------ tree
def _tree(n=3000, seed=2, leaf_max=16, group=32, kind=0, clustered=False, level_bits=1):
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3))
    if clustered:
        p[: n // 2] = 0.3 + 0.01 * rng.standard_normal((n // 2, 3))
        p = np.mod(p, 1.0)
    return p, T.BoxTree(p, 1.0, 0.17578125, leaf_max, group, kind, level_bits=level_bits)


@pytest.mark.parametrize("level_bits", [1, 3])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("clustered", [False, True])
def test_leaves_are_maximal_cells(kind, clustered, level_bits):
    p, t = _tree(kind=kind, clustered=clustered, level_bits=level_bits)
    lf = t.leaf_first
    cnt = np.diff(lf)
    assert lf[0] == 0 and lf[-1] == len(p) and np.all(cnt >= 1)
    assert np.all(cnt <= t.leaf_max)
    b = t.b
    keys = t.keys
    for a, e in zip(lf[:-1], lf[1:]):
        # walk down from the ground cell (level 0) of the leaf's first
        # particle: the first cell holding <= leaf_max particles must be
        # exactly this leaf (a maximal octree cell under the count rule)
        k0 = int(keys[a])
        s = level_bits
        for lvl in range(3 * b // s + 1):
            shift = 3 * b - s * lvl
            pre = k0 >> shift
            lo = int(np.searchsorted(keys, np.uint64(pre << shift)))
            hi = int(np.searchsorted(keys, np.uint64((pre + 1) << shift))) if pre + 1 < (1 << (64 - shift)) else len(keys)
            if hi - lo <= t.leaf_max:
                assert (lo, hi) == (a, e)
                break
        else:
            # finest level still too full: consecutive chunks of leaf_max
            assert e - a <= t.leaf_max


@pytest.mark.parametrize("level_bits", [1, 3])
def test_coincident_keys_are_chunked(level_bits):
    p = np.tile(np.array([[0.1, 0.2, 0.3]]), (70, 1))
    t = T.BoxTree(p, 1.0, 0.17578125, 32, 32, level_bits=level_bits)
    assert np.diff(t.leaf_first).tolist() == [32, 32, 6]


def test_binary_levels_give_fuller_leaves():
    # a uniform cell of 512 particles: octree leaves hold ~8, binary-level
    # leaves ~16-32 (the cells halve instead of dividing by 8)
    _, t3 = _tree(n=32768, leaf_max=32, level_bits=3)
    _, t1 = _tree(n=32768, leaf_max=32, level_bits=1)
    assert np.diff(t1.leaf_first).mean() > 1.8 * np.diff(t3.leaf_first).mean()


def test_groups_stay_inside_ground_cells():
    p, t = _tree(n=5000, group=32)
    gf = t.group_first
    assert gf[0] == 0 and gf[-1] == len(p)
    assert np.all(np.diff(gf) >= 1) and np.all(np.diff(gf) <= 32)
    for a, e in zip(gf[:-1], gf[1:]):
        assert len(set(t.ground[a:e].tolist())) == 1


@pytest.mark.parametrize("L,rcut,n", [(1.0, 0.17578125, 1500), (1.0, 0.3, 400), (1.0, 0.45, 200)])
def test_pair_relation_covers_every_pair_once(L, rcut, n):
    # Brute force: every particle pair within rcut (minimum image) appears
    # exactly once among (group(i), leaf(j), image) of the relation; N_side
    # 4 and 2 (where the -1 and +1 neighbours are one cell seen through two
    # different images) are covered.
    rng = np.random.default_rng(3)
    p = rng.random((n, 3)) * L
    t = T.BoxTree(p, L, rcut, 8, 16)
    g, l, s, d = t.pair_distances()
    keep = d < rcut
    g, l, s = g[keep], l[keep], s[keep]
    pl, pg = t.particle_leaf(), t.particle_group()
    xw = t.xw
    cover = {}
    for gi, li, sh in zip(g, l, s):
        I = np.arange(t.group_first[gi], t.group_first[gi + 1])
        J = np.arange(t.leaf_first[li], t.leaf_first[li + 1])
        dd = xw[J][None, :, :] + sh[None, None, :] * L - xw[I][:, None, :]
        r = np.sqrt(np.sum(dd * dd, axis=2))
        for a, b_ in zip(*np.nonzero(r < rcut)):
            key = (int(I[a]), int(J[b_]))
            cover[key] = cover.get(key, 0) + 1
    brute = set()
    for i in range(n):
        dd = xw - xw[i]
        dd -= L * np.round(dd / L)
        r = np.sqrt(np.sum(dd * dd, axis=1))
        for j in np.nonzero(r < rcut)[0]:
            brute.add((i, int(j)))
    assert set(cover) == brute
    assert all(v == 1 for v in cover.values())


def test_tree_does_not_change_the_force():
    # The oracle force depends on positions only: a permutation into tree
    # order gives the same accelerations (sanity of ``order``).
    p, t = _tree(n=800)
    m = np.ones(len(p)) / len(p)
    a = force.accel(p, m, 1.0, 1.0, 1e-3, 1.25 / 32, 0.17578125).acc
    b = force.accel(p[t.order], m, 1.0, 1.0, 1e-3, 1.25 / 32, 0.17578125).acc
    np.testing.assert_allclose(b, a[t.order], rtol=1e-12, atol=1e-12)
