"""Tree part of the short-range force at the leaf level (oracle side).

Test infrastructure only: nothing in the library imports it.

Written from the paper's description of the dual tree traversal (Sec. 3.3):
for two nodes of side widths A and B whose centres are a distance R apart,
the two opening angles are theta_1 = (A + B) / R and theta_2 = B / (R - A).
When an opening angle exceeds the criterion theta the pair is not accepted
(a node is opened); when both stay below it, every particle of the target
node feels the mass centre of the other node as one body (the 1-to-N case);
a pair of leaves that is never accepted ends in the PP sum (N-to-M).  The
target node is kept and the source node opened (the paper's choice on MIC).

Readings taken here (none of them fixed by the paper):

* Nodes.  The target node is an i-group (the PP kernel's target unit), the
  source node a tree leaf; interior tree nodes are not used.  A is the
  target's width, B the source's.
* Width and distance.  A node's side width is the largest side of the
  bounding box of its particles (FP64, wrapped coordinates); R is the
  distance between the two box centres, the source taken in the periodic
  image the neighbour cell implies.
* Acceptance is strict: theta_1 < theta and theta_2 < theta, both evaluated
  (theta_2 is infinite when R <= A).
* The accepted node's body interacts through the same pair law as a
  particle: Eq. (split), Plummer softening, and the hard cutoff at the
  distance to the mass centre.
* theta = 0 accepts nothing and gives back the plain short-range sum.

The decision is taken here in FP64 from the exact boxes.  A single-precision
implementation decides from rounded boxes, so pairs whose distance lies
within a small band around the acceptance threshold may be decided either
way there.  For such pairs ``accel`` reports, per target, the magnitude of
the difference between the two treatments (mass-centre body or PP sum of
the leaf), which a parity test admits the way it admits pairs within
rounding of R_cut.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import force
from .tree import BoxTree


def side_width(half_extents):
    """Side width of a node: the largest side of its bounding box."""
    return 2.0 * float(np.max(half_extents))


def opening_angles(A, B, R):
    """theta_1 = (A + B) / R and theta_2 = B / (R - A) of Sec. 3.3 (FP64).

    A is the target node's width, B the source node's, R the distance between
    the node centres; an angle whose denominator is not positive is infinite."""
    th1 = (A + B) / R if R > 0 else math.inf
    th2 = B / (R - A) if R > A else math.inf
    return th1, th2


def accepted(A, B, R, theta):
    """Both opening angles below the criterion theta (Sec. 3.3)."""
    th1, th2 = opening_angles(A, B, R)
    return th1 < theta and th2 < theta


def threshold_distance(A, B, theta):
    """The centre distance at which the acceptance flips: theta_1 < theta needs
    R > (A + B) / theta and theta_2 < theta needs R > A + B / theta."""
    return max((A + B) / theta, A + B / theta)


def leaf_mass_centres(tree: BoxTree, mass_sorted):
    """Mass and mass centre of every leaf, summed in particle order in FP64."""
    lf = tree.leaf_first
    n = len(lf) - 1
    M = np.zeros(n)
    mc = np.zeros((n, 3))
    m64 = np.asarray(mass_sorted, np.float64)
    for l in range(n):
        a, e = lf[l], lf[l + 1]
        w = m64[a:e]
        M[l] = np.sum(w)
        if M[l] > 0:
            mc[l] = np.sum(w[:, None] * tree.xw[a:e], axis=0) / M[l]
    return M, mc


@dataclass
class DttResult:
    acc: np.ndarray          # [n, 3] accelerations in the caller's order
    n_accepted: int          # (group, leaf) pairs within R_cut taken as mass-centre bodies
    n_ambiguous: int         # pairs whose distance lies within ``band`` of the threshold
    near_abs: np.ndarray     # [n] summed |term| of pairs within near_tol R_cut of the cutoff
    amb_abs: np.ndarray      # [n] summed |body - leaf PP| over the ambiguous pairs


def _terms(X, Mw, xi, ids, i_ids, G, eps2, rs, rcut):
    """Pair terms of sources X (masses Mw) on targets xi: the cutoff sum, the
    unrestricted |term| of each pair and r."""
    d = X[None, :, :] - xi[:, None, :]
    r2 = np.sum(d * d, axis=2)
    r = np.sqrt(r2)
    self_pair = ids[None, :] == i_ids[:, None]
    w_all = G * Mw[None, :] * force.split_factor_np(r, rs) / (r2 + eps2) ** 1.5
    w = np.where((r2 < rcut * rcut) & ~self_pair, w_all, 0.0)
    return np.sum(w[:, :, None] * d, axis=1), np.where(self_pair, 0.0, np.abs(w_all) * r), r


def accel(pos, mass, L, G, eps, rs, rcut, theta, leaf_max=32, group_size=32, key_kind=0, T=21, level_bits=1,
          near_tol=1e-5, band=None) -> DttResult:
    """Accelerations with leaf mass-centre bodies accepted at opening angle theta.

    ``band`` is the half width, in distance, of the ambiguous band around the
    acceptance threshold.  Its default, 2^-18 (L / theta + R_threshold), is
    four times a bound on what single precision can move the comparison by in
    a box of side L: box centres and half extents rounded to the FP32 spacing
    of coordinates below L (2^-23 L) shift R by about 2^-23 L and A + B by up
    to 2^-22 L, which the criterion divides by theta, and the FP32 products
    of the comparison add a few 2^-24 R_threshold."""
    pos = np.asarray(pos, np.float64)
    mass = np.asarray(mass, np.float32)
    n = pos.shape[0]
    t = BoxTree(pos, L, rcut, leaf_max, group_size, key_kind, T=T, level_bits=level_bits)
    ms = mass[t.order].astype(np.float64)
    M, mc = leaf_mass_centres(t, ms)
    lc, lh = t.leaf_boxes()
    gc, gh = t.group_boxes()
    ns = t.nside
    lcell = t.ground[t.leaf_first[:-1]]
    gcell = t.ground[t.group_first[:-1]]
    cell_leaves = {}
    for l, c in enumerate(lcell.tolist()):
        cell_leaves.setdefault(c, []).append(l)
    acc_sorted = np.zeros((n, 3))
    near_sorted = np.zeros(n)
    amb_sorted = np.zeros(n)
    eps2 = eps * eps
    n_acc = n_amb = 0
    for g in range(len(t.group_first) - 1):
        i0, i1 = t.group_first[g], t.group_first[g + 1]
        xi = t.xw[i0:i1]
        i_ids = np.arange(i0, i1)
        A = side_width(gh[g])
        c = int(gcell[g])
        cx, cy, cz = c // (ns * ns), (c // ns) % ns, c % ns
        src_x, src_m, src_id = [], [], []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    ax, ay, az = cx + dx, cy + dy, cz + dz
                    sh = np.array([ax // ns, ay // ns, az // ns], np.float64) * t.L
                    nc = ((ax % ns) * ns + (ay % ns)) * ns + (az % ns)
                    for l in cell_leaves.get(nc, []):
                        d = lc[l] + sh - gc[g]
                        gap = np.maximum(np.abs(d) - (gh[g] + lh[l]), 0.0)
                        if np.sqrt(np.sum(gap * gap)) >= rcut:
                            continue            # no particle pair within R_cut
                        a, e = t.leaf_first[l], t.leaf_first[l + 1]
                        body = False
                        if theta > 0:
                            B = side_width(lh[l])
                            R = float(np.sqrt(np.sum(d * d)))
                            body = accepted(A, B, R, theta)
                            Rt = threshold_distance(A, B, theta)
                            w_band = band if band is not None else 2.0 ** -18 * (t.L / theta + Rt)
                            if abs(R - Rt) <= w_band:
                                # either decision is admissible: the difference
                                # between the two treatments is the slack
                                n_amb += 1
                                f_body, _, _ = _terms(mc[l][None, :] + sh, M[l:l + 1], xi, np.array([-1]), i_ids,
                                                      G, eps2, rs, rcut)
                                f_leaf, _, _ = _terms(t.xw[a:e] + sh, ms[a:e], xi, np.arange(a, e), i_ids,
                                                      G, eps2, rs, rcut)
                                amb_sorted[i0:i1] += np.linalg.norm(f_body - f_leaf, axis=1)
                        if body:
                            n_acc += 1
                            src_x.append(mc[l][None, :] + sh)
                            src_m.append(M[l:l + 1])
                            src_id.append(np.array([-1]))
                        else:
                            src_x.append(t.xw[a:e] + sh)
                            src_m.append(ms[a:e])
                            src_id.append(np.arange(a, e))
        if not src_x:
            continue
        f, absw, r = _terms(np.concatenate(src_x), np.concatenate(src_m), xi, np.concatenate(src_id), i_ids,
                            G, eps2, rs, rcut)
        acc_sorted[i0:i1] = f
        near_sorted[i0:i1] = np.sum(np.where(np.abs(r - rcut) < near_tol * rcut, absw, 0.0), axis=1)
    out = DttResult(np.empty_like(acc_sorted), n_acc, n_amb, np.empty_like(near_sorted), np.empty_like(amb_sorted))
    out.acc[t.order] = acc_sorted
    out.near_abs[t.order] = near_sorted
    out.amb_abs[t.order] = amb_sorted
    return out
