"""Tree part of the short-range force at the leaf level (oracle side).

Test infrastructure only.  Written from the paper's description of the dual
tree traversal (Sec. 3.3): for a target node A and a source node B of side
widths A and B at distance R, the pair is accepted when both opening angles
theta_1 = (A + B) / R and theta_2 = B / (R - A) are below the criterion
theta; then every particle of the target node feels the mass centre of the
source node (one body carrying the node's mass), otherwise the source node
is opened, and a pair of leaves ends in the PP sum.  The target node is kept
and the source node opened (the paper's choice on MIC).

Readings taken here (none of them fixed by the paper):

* Nodes.  The target node is an i-group (the PP kernel's target unit), the
  source node a tree leaf; interior tree nodes are not used.
* Widths and distance.  A and B are the largest extents of the bounding
  boxes (group and leaf), R the distance between the two box centres.
  theta_1 < theta means R > (A + B) / theta, which also gives
  theta_2 < theta (R - A > B / theta follows since A / theta >= A), so the
  test is R > (A + B) / theta.
* The accepted node's body interacts through the same pair law as a
  particle: Eq. (split), Plummer softening, and the hard cutoff at the
  distance to the mass centre.
* The acceptance decision is an integer outcome of floating-point input;
  it is taken in FP32 with the kernel's operations and roundings (box centres
  and widths as the build stores them), so both sides accept the same
  pairs; the forces are then summed in FP64.  theta = 0 accepts nothing and
  gives back the plain short-range sum.
"""
from __future__ import annotations

import numpy as np

from . import force
from .tree import BoxTree

f32 = np.float32


def _ru32(x):
    """Round FP64 values up to FP32."""
    f = np.asarray(x, np.float64).astype(np.float32)
    up = f.astype(np.float64) < x
    f[up] = np.nextafter(f[up], np.float32(np.inf))
    return f


def stored_boxes(tree: BoxTree, first):
    """Boxes as the build stores them: FP64 reference point (the centre
    snapped to the FP32 spacing of the box's largest coordinate), the FP32
    centre relative to the lower corner of the box's ground cell, and the FP32
    half extents rounded up."""
    n = len(first) - 1
    lo = np.empty((n, 3))
    hi = np.empty((n, 3))
    for k in range(n):
        s = tree.xw[first[k]:first[k + 1]]
        lo[k] = s.min(axis=0)
        hi[k] = s.max(axis=0)
    cen = 0.5 * (lo + hi)
    m = np.maximum(np.abs(lo), np.abs(hi))
    U = np.ldexp(1.0, np.frexp(m)[1] - 24)
    ref = np.rint(cen / U) * U
    half = np.maximum(hi - ref, ref - lo)
    ns = tree.nside
    h = tree.L / ns
    cell = tree.ground[np.asarray(first[:-1], np.int64)]
    gxyz = np.stack([cell // (ns * ns), (cell // ns) % ns, cell % ns], axis=1).astype(np.float64)
    c32 = (ref - gxyz * h).astype(np.float32)
    return ref, c32, _ru32(half), cell


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
        M[l] = np.cumsum(w)[-1]
        if M[l] > 0:
            mc[l] = np.cumsum(w[:, None] * tree.xw[a:e], axis=0)[-1] / M[l]
    return M, mc


def accept(lc, lh, gc, gh, odx, hc, c_acc):
    """The kernel's FP32 acceptance test for one (group, leaf) pair."""
    o = f32(odx) * hc
    ex = f32(f32(lc[0] + f32(o[0])) - gc[0])
    ey = f32(f32(lc[1] + f32(o[1])) - gc[1])
    ez = f32(f32(lc[2] + f32(o[2])) - gc[2])
    R2 = f32(f32(f32(ex * ex) + f32(ey * ey)) + f32(ez * ez))
    A = f32(f32(2.0) * max(gh[0], gh[1], gh[2]))
    Bw = f32(f32(2.0) * max(lh[0], lh[1], lh[2]))
    D = f32(f32(A + Bw) * c_acc)
    return bool(R2 > f32(D * D))


def accel(pos, mass, L, G, eps, rs, rcut, theta, leaf_max=32, group_size=32, key_kind=0, T=21, level_bits=1,
          with_near=False, near_tol=1e-5):
    """Accelerations with leaf monopoles accepted at opening angle theta.

    Returns (acc [n,3] in the caller's order, number of accepted pairs), and
    with ``with_near`` also the summed magnitude of each target's terms within
    near_tol rcut of the cutoff (which FP32 may keep or drop)."""
    pos = np.asarray(pos, np.float64)
    mass = np.asarray(mass, np.float32)
    n = pos.shape[0]
    t = BoxTree(pos, L, rcut, leaf_max, group_size, key_kind, T=T, level_bits=level_bits)
    ms = mass[t.order].astype(np.float64)
    lref, lc, lh, lcell = stored_boxes(t, t.leaf_first)
    gref, gc, gh, gcell = stored_boxes(t, t.group_first)
    M, mc = leaf_mass_centres(t, ms)
    ns = t.nside
    hc = f32(t.L / ns)
    c_acc = f32(1.0 / theta) if theta > 0 else f32(np.inf)
    cell_leaves = {}
    for l, c in enumerate(lcell.tolist()):
        cell_leaves.setdefault(c, []).append(l)
    # exact box-box distances (FP64) decide which pairs can contribute at all
    ltrue_c, ltrue_h = t.leaf_boxes()
    gtrue_c, gtrue_h = t.group_boxes()
    acc_sorted = np.zeros((n, 3))
    near_sorted = np.zeros(n)
    rcut2, eps2 = rcut * rcut, eps * eps
    n_acc = 0
    for g in range(len(t.group_first) - 1):
        i0, i1 = t.group_first[g], t.group_first[g + 1]
        xi = t.xw[i0:i1]
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
                        d = ltrue_c[l] + sh - gtrue_c[g]
                        gap = np.maximum(np.abs(d) - (gtrue_h[g] + ltrue_h[l]), 0.0)
                        if np.sqrt(np.sum(gap * gap)) >= rcut:
                            continue
                        if theta > 0 and accept(lc[l], lh[l], gc[g], gh[g], np.array([dx, dy, dz]), hc, c_acc):
                            n_acc += 1
                            src_x.append(mc[l][None, :] + sh)
                            src_m.append(np.array([M[l]]))
                            src_id.append(np.array([-1]))
                        else:
                            a, e = t.leaf_first[l], t.leaf_first[l + 1]
                            src_x.append(t.xw[a:e] + sh)
                            src_m.append(ms[a:e])
                            src_id.append(np.arange(a, e))
        if not src_x:
            continue
        X = np.concatenate(src_x)
        Mw = np.concatenate(src_m)
        ids = np.concatenate(src_id)
        d = X[None, :, :] - xi[:, None, :]
        r2 = np.sum(d * d, axis=2)
        self_pair = ids[None, :] == np.arange(i0, i1)[:, None]
        keep = (r2 < rcut2) & ~self_pair
        r = np.sqrt(r2)
        w_all = G * Mw[None, :] * force.split_factor_np(r, rs) / (r2 + eps2) ** 1.5
        w = np.where(keep, w_all, 0.0)
        acc_sorted[i0:i1] = np.sum(w[:, :, None] * d, axis=1)
        near = (np.abs(r - rcut) < near_tol * rcut) & ~self_pair
        near_sorted[i0:i1] = np.sum(np.where(near, np.abs(w_all) * r, 0.0), axis=1)
    acc = np.empty_like(acc_sorted)
    acc[t.order] = acc_sorted
    if with_near:
        near_abs = np.empty_like(near_sorted)
        near_abs[t.order] = near_sorted
        return acc, n_acc, near_abs
    return acc, n_acc
