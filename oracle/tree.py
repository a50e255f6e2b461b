"""Octree leaves, i-groups and the cutoff leaf-pair relation (oracle side).

Test infrastructure only.

* Sort (Sec. 3.2): particles ordered by key, ties by original index.
* Leaves (Sec. 3.1 N_pp, Sec. 3.2, Sec. 4.4): starting from each ground cell
  (the root of a local octree), a cell holding at most ``leaf_max`` particles
  is a leaf; a larger one is split into its children, the cells of the next
  ``level_bits`` key bits (3: the 8 octree children; 1: the two halves, so
  that every octree level becomes three binary levels).  A cell at the
  finest key level that still holds more than ``leaf_max`` particles
  (coincident keys) is cut into consecutive runs of ``leaf_max``.
* i-groups: within each ground cell, consecutive runs of ``group_size``
  sorted particles (the last run of a cell may be shorter).
* Pair relation (Sec. 3.3 leaf-leaf PP, Sec. 4.3 a ground cell and its 26
  neighbours): for every i-group and every leaf of the 27 ground cells around
  the group's cell -- each neighbour taken with the periodic image shift that
  the neighbour offset implies -- the pair is kept when the distance between
  the group's and the leaf's bounding boxes is below rcut.
"""
from __future__ import annotations

import numpy as np

from . import keys as K


class BoxTree:
    """Oracle tree of one periodic box."""

    def __init__(self, pos, L, rcut, leaf_max, group_size=32, key_kind=0, T=21, box_index=0, level_bits=1):
        pos = np.asarray(pos, np.float64)
        n = pos.shape[0]
        self.L, self.rcut, self.T = float(L), float(rcut), T
        self.leaf_max, self.group_size = int(leaf_max), int(group_size)
        self.level_bits = int(level_bits)
        key, g, b = K.particle_keys(pos, L, rcut, T, key_kind, box_index)
        self.g, self.b = g, b
        self.nside = 1 << g
        order = np.lexsort((np.arange(n), key))        # stable by key
        self.order = order
        self.keys = key[order]
        self.xw = K.wrap(pos, L)[order]                 # wrapped, sorted
        sh = np.uint64(3 * b)
        cellkey = (self.keys >> sh).astype(np.int64)   # box|ground prefix
        self.ground = (self.keys >> sh).astype(np.int64) & ((1 << (3 * g)) - 1)
        # ground-cell runs
        starts = np.flatnonzero(np.r_[True, cellkey[1:] != cellkey[:-1]]) if n else np.zeros(0, np.int64)
        ends = np.r_[starts[1:], n].astype(np.int64) if n else np.zeros(0, np.int64)
        self.cell_ranges = list(zip(starts.tolist(), ends.tolist()))
        self.leaf_first = []
        for a, e in self.cell_ranges:
            self._split(a, e, 0)
        self.leaf_first = np.array(self.leaf_first + [n], np.int64)
        gf = []
        for a, e in self.cell_ranges:
            gf.extend(range(a, e, self.group_size))
        self.group_first = np.array(gf + [n], np.int64)

    def _split(self, lo, hi, level):
        cnt = hi - lo
        if cnt <= self.leaf_max:
            self.leaf_first.append(lo)
            return
        used = level * self.level_bits          # local key bits fixed so far
        if used >= 3 * self.b:
            for a in range(lo, hi, self.leaf_max):
                self.leaf_first.append(a)
            return
        sh = np.uint64(3 * self.b - used - self.level_bits)
        pref = (self.keys[lo:hi] >> sh).astype(np.int64)
        cut = np.flatnonzero(pref[1:] != pref[:-1]) + 1
        bounds = np.r_[0, cut, cnt] + lo
        for a, e in zip(bounds[:-1], bounds[1:]):
            self._split(int(a), int(e), level + 1)

    # ----- bounding boxes ------------------------------------------------
    @staticmethod
    def _aabb(xw, first):
        n = len(first) - 1
        lo = np.empty((n, 3))
        hi = np.empty((n, 3))
        for k in range(n):
            s = xw[first[k]:first[k + 1]]
            lo[k] = s.min(axis=0)
            hi[k] = s.max(axis=0)
        return 0.5 * (lo + hi), 0.5 * (hi - lo)

    def leaf_boxes(self):
        return self._aabb(self.xw, self.leaf_first)

    def group_boxes(self):
        return self._aabb(self.xw, self.group_first)

    def particle_leaf(self):
        return np.repeat(np.arange(len(self.leaf_first) - 1), np.diff(self.leaf_first))

    def particle_group(self):
        return np.repeat(np.arange(len(self.group_first) - 1), np.diff(self.group_first))

    # ----- cutoff pair relation -------------------------------------------
    def pair_distances(self):
        """All (group, leaf, shift) candidates with their box-box distance.

        Returns arrays group, leaf, shift[.,3] (in units of L) and dist.
        """
        gc, gh = self.group_boxes()
        lc, lh = self.leaf_boxes()
        nside = self.nside
        leaf_cell = self.ground[self.leaf_first[:-1]]
        cell_leaves = {}
        for li, c in enumerate(leaf_cell.tolist()):
            cell_leaves.setdefault(c, []).append(li)
        out_g, out_l, out_s, out_d = [], [], [], []
        gcell = self.ground[self.group_first[:-1]]
        for gi, c in enumerate(gcell.tolist()):
            cx, cy, cz = c // (nside * nside), (c // nside) % nside, c % nside
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        ax, ay, az = cx + dx, cy + dy, cz + dz
                        sx, sy, sz = ax // nside, ay // nside, az // nside
                        nc = ((ax % nside) * nside + (ay % nside)) * nside + (az % nside)
                        ls = cell_leaves.get(nc)
                        if not ls:
                            continue
                        ls = np.array(ls)
                        shift = np.array([sx, sy, sz], np.float64)
                        dc = lc[ls] + shift * self.L - gc[gi]
                        gap = np.maximum(np.abs(dc) - (gh[gi] + lh[ls]), 0.0)
                        d = np.sqrt(np.sum(gap * gap, axis=1))
                        out_g.append(np.full(ls.size, gi))
                        out_l.append(ls)
                        out_s.append(np.tile(shift, (ls.size, 1)))
                        out_d.append(d)
        if not out_g:
            return (np.zeros(0, np.int64),) * 2 + (np.zeros((0, 3)), np.zeros(0))
        return (np.concatenate(out_g), np.concatenate(out_l),
                np.concatenate(out_s).astype(np.int64), np.concatenate(out_d))

    def pair_set(self, slack=0.0):
        """Set of (group, leaf, sx, sy, sz) with box distance < rcut (1+slack)."""
        g, l, s, d = self.pair_distances()
        keep = d < self.rcut * (1.0 + slack)
        return set(zip(g[keep].tolist(), l[keep].tolist(), s[keep, 0].tolist(),
                       s[keep, 1].tolist(), s[keep, 2].tolist()))
