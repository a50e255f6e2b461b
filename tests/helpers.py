"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it element by element with the FP64 oracle."""
from __future__ import annotations

import numpy as np

from oracle import force

# Tolerances (relative force error e_i = |a - a_ref| / max(|a_ref|, tau),
# tau = 1e-3 median |a_ref|).  The exact path is FP32 with SFU rsqrt/sqrt/ex2
# (relative error ~2^-22 each), a degree-10 polynomial for the factor
# (~3e-7) and leaf-relative coordinates (d_ij exact to ~1e-7 of the leaf
# size); per pair that is a few 1e-7, so 1e-5 at the 99th percentile leaves
# room for the cancellation of many terms, and 1e-3 bounds any single
# particle (one cutoff-boundary pair classified the other way excepted, which
# the oracle's near-cutoff sum accounts for).
P99_TOL = 1e-5
MAX_TOL = 1e-3


def rel_errors(got, ref_res):
    ref = ref_res.acc
    amag = np.linalg.norm(ref, axis=1)
    tau = 1e-3 * np.median(amag) if amag.size else 0.0
    den = np.maximum(amag, tau)
    diff = np.linalg.norm(np.asarray(got, np.float64) - ref, axis=1)
    # a pair within FP32 rounding of rcut may be kept or dropped: its whole
    # term (G included, as the oracle sums it) is an admissible difference
    slack = ref_res.near_abs
    e = np.maximum(diff - slack, 0.0) / np.where(den > 0, den, 1.0)
    return e


def check_parity(got, ref_res, p99=P99_TOL, emax=MAX_TOL):
    e = rel_errors(got, ref_res)
    if e.size == 0:
        return 0.0, 0.0
    q = float(np.percentile(e, 99))
    m = float(e.max())
    assert q <= p99, f"p99 relative error {q:.3e} > {p99:.1e}"
    assert m <= emax, f"max relative error {m:.3e} > {emax:.1e} at {int(np.argmax(e))}"
    return q, m


def gpu_accel(B, ps, key_kind=0, leaf_max=None, pos_dtype=np.float32, host=False, group_size=0, level_bits=0):
    """Accelerations of a ParticleSet through the C ABI (batched if B > 1)."""
    import torch
    pos = ps.pos.astype(pos_dtype)
    prms = [B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, leaf_max or bp.leaf_max, key_kind, group_size,
                          level_bits) for bp in ps.boxes]
    if host:
        tpos = torch.from_numpy(np.ascontiguousarray(pos))
        tmass = torch.from_numpy(ps.mass)
        acc = torch.zeros((ps.n, 3), dtype=torch.float32)
    else:
        tpos = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
        tmass = torch.from_numpy(ps.mass).cuda()
        acc = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    if len(prms) == 1:
        lv = B.ph_build_leaves(tpos, tmass, prms[0])
    else:
        lv = B.ph_build_leaves_batched(tpos, tmass, ps.offsets, prms)
    pr = B.ph_leaf_pairs(lv)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    B.ph_status(lv)
    B.ph_status(pr)
    return acc.cpu().numpy(), lv, pr


def oracle_accel(ps, targets=None, box=0):
    bp = ps.boxes[box]
    sl = ps.box_slice(box)
    return force.accel(ps.pos[sl], ps.mass[sl], bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=targets)
