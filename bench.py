"""Benchmark of the short-range PP hot path on GB300.

A step is one pass of the whole path over one particle set already resident
in HBM: keys + sort + leaves + groups (ph_build_leaves), the cutoff leaf-pair
list (ph_leaf_pairs) and the exact-factor PP sum (ph_pp_accel), replayed as
the library's captured step graph (ph_graph_create / ph_graph_launch: the
same kernels with no host round trip between them).  The default workload
is the 128^3 Zel'dovich lattice (L=100, rs=1.25 L/128, rcut=4.5 rs,
eps=L/128/30).

value     = interactions within rcut (ordered pairs j != i, r < rcut) per
            second of whole-step time, summed over ranks;
e2e       = the same through the public host-buffer replay of the captured
            step (ph_graph_launch_host: positions/masses copied in from
            pinned memory, accelerations copied out, inside the timed
            region); the one-call ph_accel path is timed beside it;
roofline  = the PP kernel's FP32 rate (interactions it evaluated x the stated
            flop count per interaction / its CUDA-event time) against the FP32
            FMA peak: SMs x 128 lanes x 2 flop x max SM clock;
cpu_baseline / --impl reference = the FP64 oracle on the host's cores over a
            bounded sample of the same workload (all sources, a subset of
            targets), in the same unit.

With N > 1 (torchrun) the box is cut into N domains along the Peano-Hilbert
curve of its ground cells (Sec. 4.1): every rank holds a shard, exchanges
particles and ghosts with the others over NCCL (the packing in the
library's kernels) and computes its own particles' forces; value is the
whole box's interactions per second of the slowest rank (strong scaling).
--replicas runs N independent whole-box replicas instead (weak scaling);
--partitioned runs the domain path with one rank too.  --jsonl PATH also
appends the result line to PATH, one line per run.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PP interactions/sec and % of GB300 FP32 peak; learned-g vs exact-g speedup at error"
UNIT = "interactions/s"

# FP32 operations per evaluated pair in the exact PP kernel (counted from the
# source, FADD/FMUL = 1 flop, FFMA = 2, SFU rsqrt/sqrt/ex2 = 0, Kahan adds and
# the cutoff select not counted): d 3 FADD; r^2 1 FMUL + 2 FFMA; scaled
# r^2 s2 + eps2s 1 FFMA; its cube 2 FMUL (one SFU rsqrt then gives the
# inverse cube); t = sqrt(r^2) 2/rcut - 1 1 FFMA; degree-10 Horner 10 FFMA;
# ex2 argument 1 FMUL; f 1 FMUL; w 2 FMUL; accumulation 3 FFMA
#   ->  3 FADD + 7 FMUL + 17 FFMA = 44 flop.
# The ncu counters of one 128^3 launch (sm__sass_thread_inst_executed_op_
# {fadd2,fmul2,ffma2}_pred_on) give 44.13 flop per evaluated pair for the
# packed pair arithmetic (the excess is the padded lanes of partial runs).
FLOPS_PER_INTERACTION = 44
PAPER_FLOPS_PER_INTERACTION = 22   # the convention of Sec. 5
# DRAM traffic (read + write) of one PP launch on the 128^3 Zel'dovich lattice,
# from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of one
# k_pp launch of this benchmark's configurations the autotuner picks between:
# leaf_max 32 or 16, binary levels, kernel shape 0, 32-particle groups,
# Peano-Hilbert keys.  None for any other configuration, or once the kernel
# has changed since the capture.
PP_TRAFFIC = {   # (workload, scale, leaf_max, levels, variant, group, key) -> bytes
    ("zeldovich_128", 0, 32, 1, 0, 32, 1): 239986432 + 24170496,
    ("zeldovich_128", 0, 16, 1, 0, 32, 1): 345537536 + 29011968,
}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, period_ms=100):
        self.gpu_index = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms", str(self.period_ms), "-i", str(self.gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "0x1") or v == "1":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v.strip() for v in vis.split(",") if v.strip()]
    if ids and ids[min(local_rank, len(ids) - 1)].isdigit():
        return int(ids[min(local_rank, len(ids) - 1)])
    return local_rank


def _params(B, bp, leaf_max, key_kind, pp_variant=0):
    return B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, leaf_max or bp.leaf_max, key_kind, 0, 0, pp_variant)


def _oracle_rate(ps, seconds, seed=5):
    """Oracle over a bounded target sample: (useful interactions/s, targets, s, cores)."""
    from oracle import force
    bp = ps.boxes[0]
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    ncal = min(ps.n, 256)
    cal = rng.choice(ps.n, ncal, replace=False)
    force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=cal)
    per_target = (time.perf_counter() - t0) / ncal
    nt = int(min(ps.n, max(32, seconds / max(per_target, 1e-9))))
    tg = rng.choice(ps.n, nt, replace=False)
    t0 = time.perf_counter()
    r = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=tg)
    dt = time.perf_counter() - t0
    return float(r.n_within.sum()) / dt, nt, dt, force.num_threads()


def _learned_extra(B, ps, lv, pr, stream, t_exact_pp):
    """The learned factor on the same lists: training, time, errors."""
    import torch
    from oracle import force
    bp = ps.boxes[0]
    # 400k Adam steps of 4096 samples (about 6 s on the GPU) bring the
    # validated max |g_hat/g - 1| to ~6.5e-4, inside the 1e-3 tolerance
    tp = B.make_train_params(n_samples=1_000_000, batch=4096, steps=400_000, lr0=2e-3, lr_min=1e-6, tol=1e-3,
                             seed=2024)
    t0 = time.perf_counter()
    mlp = B.ph_mlp_train(tp, bp.rs, bp.rcut)
    train_s = time.perf_counter() - t0
    w, err, loss = B.ph_mlp_get(mlp)
    # time the learned kernel whatever its validation against the exact factor says (tolerance 1)
    timed = B.ph_mlp_create(w, bp.rs, bp.rcut, tol=1.0)
    acc_l = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    acc_e = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc_e, stream)
    B.ph_pp_accel(lv, pr, B.PH_G_LEARNED, timed, acc_l, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        B.ph_pp_accel(lv, pr, B.PH_G_LEARNED, timed, acc_l, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_l = e0.elapsed_time(e1) / reps
    rng = np.random.default_rng(11)
    tg = rng.choice(ps.n, 256, replace=False)
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=tg)
    am = np.linalg.norm(ref.acc, axis=1)
    tau = 1e-3 * np.median(am)

    def p99(a):
        e = np.linalg.norm(a[tg].astype(np.float64) - ref.acc, axis=1) / np.maximum(am, tau)
        return float(np.percentile(e, 99))

    out = {"config": "learned factor on the same workload and lists (MLP 1-16-16-1 SiLU, BF16 MMA layer 2)",
           "train_steps": tp.steps, "train_batch": tp.batch, "train_s": train_s, "train_loss": loss,
           "g_max_rel_err": err, "validation_tolerance": 1e-3, "falls_back": bool(err > 1e-3),
           "pp_ms": t_l, "exact_pp_ms": t_exact_pp, "speedup_vs_exact": t_exact_pp / t_l,
           "force_p99_rel_err_learned": p99(acc_l.cpu().numpy()),
           "force_p99_rel_err_exact": p99(acc_e.cpu().numpy()), "oracle_targets": int(tg.size)}
    B.ph_free(timed)
    B.ph_free(mlp)
    return out


def _table_extra(B, ps, lv, pr, stream, t_exact_pp, flush):
    """The tabulated factor (PH_G_TABLE) on the same lists: time and errors."""
    import torch
    from oracle import force
    bp = ps.boxes[0]
    acc_t = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    acc_e = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc_e, stream)
    B.ph_pp_accel(lv, pr, B.PH_G_TABLE, None, acc_t, stream)
    torch.cuda.synchronize()
    reps = 5
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.ph_pp_accel(lv, pr, B.PH_G_TABLE, None, acc_t, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    t_t = float(np.median(ts))
    rng = np.random.default_rng(12)
    tg = rng.choice(ps.n, 256, replace=False)
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=tg)
    am = np.linalg.norm(ref.acc, axis=1)
    tau = 1e-3 * np.median(am)

    def p99(a):
        e = np.linalg.norm(a[tg].astype(np.float64) - ref.acc, axis=1) / np.maximum(am, tau)
        return float(np.percentile(e, 99))

    return {"config": "tabulated factor on the same workload and lists (4097 nodes in r, nearest node + slope)",
            "pp_ms": t_t, "exact_pp_ms": t_exact_pp, "speedup_vs_exact": t_exact_pp / t_t,
            "force_p99_rel_err_table": p99(acc_t.cpu().numpy()),
            "force_p99_rel_err_exact": p99(acc_e.cpu().numpy()), "oracle_targets": int(tg.size)}


def _group16_extra(B, ps, pos, mass, stream, flush, peak, n_within):
    """16-particle target groups (two lanes per target, leaf 16, kernel shape
    1) on the same particles: fewer pairs beyond R_cut, against the whole
    step's cost.  The autotuner measures this among its candidates; here it is
    reported beside the headline configuration."""
    import torch
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 16, B.PH_KEY_HILBERT, 16, 1, 1)
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    lv = B.ph_build_leaves(pos, mass, prm, stream)
    pr = B.ph_leaf_pairs(lv, stream)
    B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc, stream)
    torch.cuda.synchronize()
    inter, _ = B.ph_pp_counters(pr)
    graph = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25, stream=stream)
    B.ph_graph_launch(graph, stream)
    torch.cuda.synchronize()

    def timed(fn, reps=8):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_step = timed(lambda: B.ph_graph_launch(graph, stream))
    t_pp = timed(lambda: B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc, stream))
    for h in (graph, pr, lv):
        B.ph_free(h)
    return {"config": "leaf 16, 16-particle groups (2 lanes per target), kernel shape 1, same particles",
            "step_ms": t_step, "pp_ms": t_pp, "interactions_evaluated": inter, "within_fraction": n_within / max(inter, 1),
            "frac_evaluated": inter * FLOPS_PER_INTERACTION / (t_pp * 1e-3) / 1e12 / peak,
            "frac_within_rcut": n_within * FLOPS_PER_INTERACTION / (t_pp * 1e-3) / 1e12 / peak,
            "value": n_within / (t_step * 1e-3)}


def _tree_extra(B, stream, flush, peak, theta=0.3):
    """The 256^3 NFW mixture (16.8M particles, the largest single-GPU
    configuration): the plain short-range step (theta = 0) with its PP kernel
    timed alone, its FP32 roofline and within-R_cut fraction, and the tree
    part (leaf monopoles at opening angle theta) beside it; force errors of
    both against the plain FP64 oracle on sampled targets."""
    import torch
    from oracle import force
    from paper_1802_09824_gb300 import synth
    ps = synth.workload("nfw_mix_256")
    bp = ps.boxes[0]
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    rng = np.random.default_rng(13)
    tg = rng.choice(ps.n, 256, replace=False)
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=tg)
    am = np.linalg.norm(ref.acc, axis=1)
    tau = 1e-3 * np.median(am)
    out = {"workload": "nfw_mix_256", "n": ps.n, "theta": theta, "leaf_max": 32, "key": "hilbert", "group_size": 32,
           "kernel_shape": 0}

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for th in (0.0, theta):
        prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, 1, 32, 1, 0, th)
        acc = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
        lv = B.ph_build_leaves(pos, mass, prm, stream)
        pr = B.ph_leaf_pairs(lv, stream)
        g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25, stream=stream)
        B.ph_graph_launch(g, stream)
        torch.cuda.synchronize()
        t_step = timed(lambda: B.ph_graph_launch(g, stream))
        B.ph_status(pr)
        inter, staged = B.ph_pp_counters(pr)
        a = acc.cpu().numpy()[tg].astype(np.float64)
        e = np.linalg.norm(a - ref.acc, axis=1) / np.maximum(am, tau)
        key = "theta0" if th == 0 else "theta"
        row = {"step_ms": t_step, "pairs_evaluated": inter,
               "force_p99_rel_err": float(np.percentile(e, 99)), "force_max_rel_err": float(e.max())}
        if th == 0:
            # the PP kernel alone on the same lists, its roofline, and the
            # useful (r < R_cut) share of the pairs it evaluates
            t_pp = timed(lambda: B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc, stream))
            inter, staged = B.ph_pp_counters(pr)
            n_within = B.ph_count_within(lv, pr, stream)
            achieved = inter * FLOPS_PER_INTERACTION / (t_pp * 1e-3) / 1e12
            row.update({"pp_ms": t_pp, "build_and_pairs_ms": t_step - t_pp, "interactions_within_rcut": n_within,
                        "within_fraction": n_within / max(inter, 1),
                        "value": n_within / (t_step * 1e-3), "unit": UNIT,
                        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                     "frac": achieved / peak, "flops_per_interaction": FLOPS_PER_INTERACTION}})
        out[key] = row
        for h in (g, pr, lv):
            B.ph_free(h)
    out["speedup_vs_theta0"] = out["theta0"]["step_ms"] / out["theta"]["step_ms"]
    out["oracle_targets"] = int(tg.size)
    return out


def _pm_extra(B, ps, pos, mass, prm, graph, acc, stream, flush, n_mesh):
    """The long-range PM side on the same particles (mesh n_mesh^3): its time
    alone, the time of the whole split force (the captured short-range step
    followed by PM added to its result), and its error against the FP64
    oracle's PM on sampled targets."""
    import torch
    from oracle import pm as opm
    bp = ps.boxes[0]
    acc_pm = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    h = B.ph_pm_accel(pos, mass, prm, n_mesh, acc_pm, stream=stream)
    for _ in range(3):
        B.ph_pm_accel(pos, mass, prm, n_mesh, acc_pm, stream=stream, pm=h)
    torch.cuda.synchronize()

    def timed(fn, reps=7):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_pm = timed(lambda: B.ph_pm_accel(pos, mass, prm, n_mesh, acc_pm, stream=stream, pm=h))

    def total():
        B.ph_graph_launch(graph, stream)
        B.ph_pm_accel(pos, mass, prm, n_mesh, acc, accumulate=True, stream=stream, pm=h)

    t_total = timed(total)
    B.ph_status(h)
    rng = np.random.default_rng(14)
    tg = rng.choice(ps.n, 2000, replace=False)
    ref = opm.accel(ps.pos, ps.mass, bp.L, bp.G, bp.rs, n_mesh, targets=tg).acc
    am = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(acc_pm.cpu().numpy()[tg].astype(np.float64) - ref, axis=1) / np.maximum(am, 1e-3 * np.median(am))
    B.ph_free(h)
    return {"n_mesh": n_mesh, "pm_ms": t_pm, "split_force_step_ms": t_total,
            "force_p99_rel_err": float(np.percentile(e, 99)), "force_max_rel_err": float(e.max()),
            "oracle_targets": int(tg.size)}


def _kdk_extra(B, ps, prm, n_mesh, acc_total, steps=2):
    """Adaptive KDK block steps on the same particles (at rest at t = 0) with
    the split force (PP + PM): force passes, time per top step and per force
    pass.  Each event synchronises the host once (the next event tick)."""
    import torch
    bp = ps.boxes[0]
    pos = np.ascontiguousarray(ps.pos.astype(np.float64))
    mom = np.zeros_like(pos)
    # top step chosen so that the median acceleration asks for level 1
    # ((dt/2)^2 |a| = thr / 2 with thr = 2 eta eps); particles pulled 4 or 16
    # times harder go to levels 2 and 3
    eta = 0.02
    a_med = float(torch.linalg.vector_norm(acc_total.double(), dim=1).median())
    dt = math.sqrt(2.0 * (2.0 * eta * bp.eps) / a_med)
    kp = B.make_kdk_params(dt=dt, eta=eta, max_level=3, n_mesh=n_mesh)
    sim = B.ph_sim_create(pos, mom, torch.from_numpy(ps.mass).cuda(), prm, kp, 0.0)
    _, _, _, _, _, fp0 = B.ph_sim_get(sim, ps.n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.ph_sim_step(sim, steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    _, _, _, lv, _, fp = B.ph_sim_get(sim, ps.n)
    B.ph_free(sim)
    passes = fp - fp0
    return {"top_steps": steps, "dt": kp.dt, "eta": eta, "force_passes": passes,
            "ms_per_top_step": 1e3 * wall / steps, "ms_per_force_pass": 1e3 * wall / max(passes, 1),
            "max_level": 3, "n_mesh": n_mesh, "level_counts": np.bincount(lv, minlength=4).tolist()}


def _batched_extra(B, args, dev, stream):
    """512 boxes: one graph-captured step (the autotuner's leaf size, key,
    group size and kernel shape for this batch) against the same boxes as
    512 separately captured per-box steps replayed back to back (per-box
    launches without host synchronisation), and against one ph_accel call per
    box (the sizing path: three host synchronisations per box)."""
    import torch
    from paper_1802_09824_gb300 import synth, tuning
    ps = synth.workload("batch_512")
    prms = [_params(B, bp, 32, 1) for bp in ps.boxes]
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    t0 = time.perf_counter()
    prms, tune_info = tuning.tuned(B, pos, mass, ps.offsets, prms, reps=2)
    tune_s = time.perf_counter() - t0
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    lv = B.ph_build_leaves_batched(pos, mass, ps.offsets, prms, stream)
    pr = B.ph_leaf_pairs(lv, stream)
    n_within = B.ph_count_within(lv, pr, stream)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, 0.25, stream)
    kernels = B.ph_graph_kernels(g)
    for _ in range(3):
        B.ph_graph_launch(g, stream)
    torch.cuda.synchronize()
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        B.ph_graph_launch(g, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    B.ph_status(pr)
    t_graph = e0.elapsed_time(e1) / reps
    # the PP kernel alone on the batch's lists (one persistent launch over
    # all boxes' groups), its FP32 roofline and the within-R_cut share
    e0.record(stream)
    for _ in range(reps):
        B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pp = e0.elapsed_time(e1) / reps
    inter, _ = B.ph_pp_counters(pr)
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * 2 * 2070.0 * 1e6 / 1e12
    pp = {"ms": t_pp, "interactions_evaluated": inter, "within_fraction": n_within / max(inter, 1),
          "roofline_frac": inter * FLOPS_PER_INTERACTION / (t_pp * 1e-3) / 1e12 / peak,
          "peak_tflops": peak}
    # the same boxes, each its own captured step (same knobs), replayed one
    # after another on the stream
    views = [(pos[ps.box_slice(b)], mass[ps.box_slice(b)], acc[ps.box_slice(b)]) for b in range(len(ps.boxes))]
    per = []
    for b, (p_, m_, a_) in enumerate(views):
        l_ = B.ph_build_leaves(p_, m_, prms[b], stream)
        r_ = B.ph_leaf_pairs(l_, stream)
        per.append((B.ph_graph_create(l_, r_, p_, m_, B.PH_G_EXACT, None, a_, 0.25, stream), r_, l_))
    for _ in range(2):
        for gb, _, _ in per:
            B.ph_graph_launch(gb, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        for gb, _, _ in per:
            B.ph_graph_launch(gb, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_graphs = e0.elapsed_time(e1) / 3
    for hs in per:
        for h in hs:
            B.ph_free(h)
    # one ph_accel call per box (handles reused per box)
    handles = [(None, None)] * len(ps.boxes)

    def per_box():
        for b, (p_, m_, a_) in enumerate(views):
            l_, r_ = handles[b]
            handles[b] = B.ph_accel(p_, m_, prms[b], B.PH_G_EXACT, None, a_, stream, leaves=l_, pairs=r_)

    per_box()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        per_box()
    torch.cuda.synchronize()
    t_box = 1e3 * (time.perf_counter() - t0) / 2
    for l_, r_ in handles:
        B.ph_free(r_)
        B.ph_free(l_)
    B.ph_free(g)
    B.ph_free(pr)
    B.ph_free(lv)
    p0 = prms[0]
    return {"workload": "batch_512", "n": ps.n, "boxes": len(ps.boxes), "interactions_within_rcut": n_within,
            "tuned": {"leaf_max": p0.leaf_max, "level_bits": p0.level_bits, "pp_variant": p0.pp_variant,
                      "group_size": p0.group_size or 32, "key_kind": p0.key_kind, "cache": tune_info["cache"],
                      "tune_s": tune_s},
            "graph_ms_per_step": t_graph, "graph_kernels_per_step": kernels, "pp": pp,
            "per_box_graphs_ms_per_step": t_graphs, "speedup_graph_vs_per_box_graphs": t_graphs / t_graph,
            "per_box_calls_ms_per_step": t_box, "speedup_graph_vs_per_box_calls": t_box / t_graph,
            "value_graph": n_within / (t_graph * 1e-3), "unit": UNIT}


class Ranks:
    """Barrier and max / sum reductions of one float over the ranks of a
    torch.distributed job (dist = None: a single process, identity).  The
    replicas' step times combine by max, their counts by sum."""

    def __init__(self, dist, device):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def run_reference(args, rank):
    if rank != 0:
        return
    from paper_1802_09824_gb300 import synth
    ps = synth.workload(args.workload, scale=args.scale or None)
    per_step = max(1.0, args.ref_seconds / max(1, args.steps))
    for _ in range(args.warmup):
        _oracle_rate(ps, 0.2)
    rates, nts, secs = [], [], []
    cores = 1
    for k in range(args.steps):
        r, nt, dt, cores = _oracle_rate(ps, per_step, seed=100 + k)
        rates.append(r)
        nts.append(nt)
        secs.append(dt)
    value = float(np.mean(rates))
    sample = (f"{args.workload}: all {ps.n} sources against {int(np.mean(nts))} random targets per step, "
              f"FP64 C/OpenMP oracle")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "n": ps.n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line, args)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1802_09824_gb300 import binding as B
    from paper_1802_09824_gb300 import synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ranks = Ranks(dist, dev)

    def barrier():
        ranks.barrier()
        torch.cuda.synchronize()

    max_over_ranks = ranks.max
    sum_over_ranks = ranks.sum

    ps = synth.workload(args.workload, scale=args.scale or None)
    bp = ps.boxes[0]
    prm = _params(B, bp, args.leaf_max, args.key, args.pp_variant)
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    tune_info = None
    if not args.leaf_max and not args.no_tune:
        # leaf size / hierarchy / kernel shape from the in-project autotuner
        from paper_1802_09824_gb300 import tuning
        (prm,), tune_info = tuning.tuned(B, pos, mass, ps.offsets, [prm], reps=3)
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    lv = pr = None

    def step(events=None):
        nonlocal lv, pr
        lv = B.ph_build_leaves(pos, mass, prm, stream, leaves=lv)
        pr = B.ph_leaf_pairs(lv, stream, pairs=pr)
        if events is not None:
            events[1].record(stream)
        B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc, stream)
        if events is not None:
            events[2].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    B.ph_status(lv)
    B.ph_status(pr)
    n_within = B.ph_count_within(lv, pr, stream)
    step()
    torch.cuda.synchronize()
    computed, staged = B.ph_pp_counters(pr)

    gpu_idx = _gpu_index(local_rank)
    clocks = ClockSampler(gpu_idx)
    clocks.start()
    time.sleep(0.3)
    # ---- device-resident timed region: the captured whole step
    graph = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25, stream=stream)
    for _ in range(2):
        B.ph_graph_launch(graph, stream)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    launches0 = B.ph_launch_counter()
    barrier()
    for k in range(args.steps):
        flush.zero_()                       # L2 flush between steps (not timed)
        evs[k][0].record(stream)
        B.ph_graph_launch(graph, stream)
        evs[k][1].record(stream)
    barrier()
    launches = B.ph_launch_counter() - launches0
    B.ph_status(lv)
    B.ph_status(pr)                         # no pair-list overflow in the replays
    step_ms = [e[0].elapsed_time(e[1]) for e in evs]
    t_step = max_over_ranks(sum(step_ms) / args.steps)
    # the PP kernel alone (roofline): same lists, L2 flushed before each launch
    pevs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        pevs[k][0].record(stream)
        B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc, stream)
        pevs[k][1].record(stream)
    torch.cuda.synchronize()
    t_pp = sum(e[0].elapsed_time(e[1]) for e in pevs) / args.steps
    # the leaf build and the pair list alone (direct calls on the same
    # handles, L2 flushed first; CUDA events on the stream, so the pair
    # call's host read of its list size is inside its interval)
    tb, tq = [], []
    for _ in range(max(args.steps // 2, 5)):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        lv = B.ph_build_leaves(pos, mass, prm, stream, leaves=lv)
        ev[1].record(stream)
        pr = B.ph_leaf_pairs(lv, stream, pairs=pr)
        ev[2].record(stream)
        torch.cuda.synchronize()
        tb.append(ev[0].elapsed_time(ev[1]))
        tq.append(ev[1].elapsed_time(ev[2]))
    t_build, t_pairs = float(np.median(tb)), float(np.median(tq))

    # ---- end to end through the public calls with host buffers: the
    # captured step replayed from pinned host buffers (ph_graph_launch_host:
    # positions and masses copied in, accelerations copied out, one
    # synchronisation), and the one-call step ph_accel (three host
    # synchronisations: leaf sizing, pair sizing, the copy out)
    pos_h = torch.from_numpy(ps.pos).pin_memory()
    mass_h = torch.from_numpy(ps.mass).pin_memory()
    acc_h = torch.empty((ps.n, 3), dtype=torch.float32).pin_memory()
    for _ in range(3):
        B.ph_graph_launch_host(graph, pos_h, mass_h, acc_h, stream)
    barrier()
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.ph_graph_launch_host(graph, pos_h, mass_h, acc_h, stream)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()
    t_e2e_sync = max_over_ranks(sum(e2e_ms) / args.steps)
    # the same replay overlapped: a second set of handles, device buffers
    # and pinned host buffers on a second stream; steps alternate between
    # the two sets (ph_graph_launch_host_async), so one step's copies run
    # under the other's kernels.  Each step's stream first writes the L2
    # flush buffer (inside the timed region, as conservative as the
    # device-timed steps' flush outside it).
    stream_b = torch.cuda.Stream()
    pos_b, mass_b = pos.clone(), mass.clone()
    acc_b = torch.empty_like(acc)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream_b):
        lv_b = B.ph_build_leaves(pos_b, mass_b, prm, stream_b)
        pr_b = B.ph_leaf_pairs(lv_b, stream_b)
        graph_b = B.ph_graph_create(lv_b, pr_b, pos_b, mass_b, B.PH_G_EXACT, None, acc_b, headroom=0.25,
                                    stream=stream_b)
    torch.cuda.synchronize()
    sets = [(graph, pos_h, mass_h, acc_h, stream),
            (graph_b, pos_h.clone().pin_memory(), mass_h.clone().pin_memory(),
             torch.empty_like(acc_h).pin_memory(), stream_b)]

    def overlapped(k_steps):
        for k in range(k_steps):
            g_, p_, m_, a_, s_ = sets[k % 2]
            with torch.cuda.stream(s_):
                flush.zero_()
            B.ph_graph_launch_host_async(g_, p_, m_, a_, s_)
        torch.cuda.synchronize()

    overlapped(4)
    barrier()
    t0 = time.perf_counter()
    overlapped(args.steps)
    t_e2e = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.steps)
    barrier()
    for h_ in (lv_b, pr_b):
        B.ph_status(h_)
    B.ph_status(lv)
    B.ph_status(pr)
    if not (np.all(np.isfinite(sets[1][3].numpy())) and np.array_equal(sets[0][3].numpy(), sets[1][3].numpy())):
        raise RuntimeError("the overlapped replays disagree")
    for h_ in (graph_b, pr_b, lv_b):
        B.ph_free(h_)
    lv2 = pr2 = None
    for _ in range(3):
        lv2, pr2 = B.ph_accel(pos_h, mass_h, prm, B.PH_G_EXACT, None, acc_h, stream, leaves=lv2, pairs=pr2)
    torch.cuda.synchronize()
    acc_ms = []
    for k in range(max(args.steps // 4, 3)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lv2, pr2 = B.ph_accel(pos_h, mass_h, prm, B.PH_G_EXACT, None, acc_h, stream, leaves=lv2, pairs=pr2)
        torch.cuda.synchronize()
        acc_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()
    clk = clocks.stop()
    if not np.all(np.isfinite(acc_h.numpy())):
        raise RuntimeError("non-finite accelerations")

    value = sum_over_ranks(n_within) / (t_step * 1e-3)
    e2e_value = sum_over_ranks(n_within) / (t_e2e * 1e-3)
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12                    # TFLOP/s
    achieved = computed * FLOPS_PER_INTERACTION / (t_pp * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": PP_TRAFFIC.get((args.workload, args.scale, prm.leaf_max, prm.level_bits or 1, prm.pp_variant,
                                       prm.group_size or 32, prm.key_kind)),
            "kernel": "k_pp (exact factor)", "flops_per_interaction": FLOPS_PER_INTERACTION,
            "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)"}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / (peak * clk["sm_mhz"] / sm_max)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload + (f"@{args.scale}" if args.scale else ""), "n": ps.n, "leaf_max": prm.leaf_max,
                   "key": "hilbert" if prm.key_kind else "morton", "group_size": prm.group_size or 32,
                   "l2": "flushed between steps (256 MB write), per-step CUDA events",
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": t_e2e,
                "h2d_bytes_per_step": ps.n * 16, "d2h_bytes_per_step": ps.n * 12,
                "call": "ph_graph_launch_host_async (captured step from pinned host buffers, two buffer sets "
                        "alternating on two streams: one step's copies under the other's kernels; every step "
                        "copies its positions and masses in and its accelerations out)",
                "l2": "flushed on each step's stream before its copies (inside the timed region)",
                "ms_per_step_one_call_at_a_time": t_e2e_sync,
                "ph_accel_ms_per_step": max_over_ranks(sum(acc_ms) / len(acc_ms))},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk,
        "pp": {"ms": t_pp, "interactions_evaluated": computed, "interactions_within_rcut": n_within,
               "evaluated_per_s": computed / (t_pp * 1e-3), "within_fraction": n_within / max(computed, 1),
               "staged_sources": staged, "paper_convention_tflops": computed * PAPER_FLOPS_PER_INTERACTION /
               (t_pp * 1e-3) / 1e12},
        "build_and_pairs_ms": t_step - t_pp,
        "build_ms": t_build, "pairs_ms": t_pairs,
    }
    if tune_info is not None:
        line["config"]["tuned"] = {"leaf_max": prm.leaf_max, "level_bits": prm.level_bits,
                                   "pp_variant": prm.pp_variant, "group_size": prm.group_size or 32,
                                   "key_kind": prm.key_kind,
                                   "cache": tune_info["cache"]}
    if not args.no_extras:
        line["learned"] = _learned_extra(B, ps, lv, pr, stream, t_pp)
        line["table"] = _table_extra(B, ps, lv, pr, stream, t_pp, flush)
        line["tree"] = _tree_extra(B, stream, flush, peak)
        line["group16"] = _group16_extra(B, ps, pos, mass, stream, flush, peak, n_within)
        n_mesh = int(round(bp.L / (bp.rs / 1.25)))       # R_s = 1.25 mesh cells
        line["pm"] = _pm_extra(B, ps, pos, mass, prm, graph, acc, stream, flush, n_mesh)
        line["kdk"] = _kdk_extra(B, ps, prm, n_mesh, acc)
        line["batched"] = _batched_extra(B, args, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, nt, dt, cores = _oracle_rate(ps, args.cpu_seconds)
        tests_per_s = float(ps.n) * nt / dt
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"all {ps.n} sources x {nt} random targets, {dt:.1f} s",
                                "pair_tests_per_s_per_core": tests_per_s / cores,
                                "extrapolated_full_step_s": float(ps.n) * ps.n / tests_per_s,
                                "extrapolated": "all N targets at the sample's rate"}
        # the small configuration (4096 uniform particles) in full: every
        # target against every source, no extrapolation
        from oracle import force
        small = synth.workload("uniform_small")
        sb = small.boxes[0]
        t0 = time.perf_counter()
        rs_ = force.accel(small.pos, small.mass, sb.L, sb.G, sb.eps, sb.rs, sb.rcut)
        dts = time.perf_counter() - t0
        line["cpu_baseline"]["small_config_full"] = {
            "workload": "uniform_small", "n": small.n, "s": dts,
            "interactions_per_s": float(rs_.n_within.sum()) / dts,
            "pair_tests_per_s_per_core": float(small.n) * small.n / dts / cores}
    # the paper's PP kernel efficiencies (fraction of the node's peak, Sec. 5):
    # other hardware and a 22-flop convention, context only
    line["paper_context"] = {"pp_efficiency_cpu": 0.744, "pp_efficiency_mic": 0.686,
                             "ours_paper_convention_frac": line["pp"]["paper_convention_tflops"] / peak}
    for h in (graph, pr, lv, pr2, lv2):
        B.ph_free(h)
    if rank == 0:
        emit(line, args)
    if dist is not None:
        dist.destroy_process_group()


def run_partitioned(args, rank, world, local_rank):
    """The domain decomposition of Sec. 4.1 (strong scaling of one box over
    the ranks): every rank holds a contiguous shard of the particles; a step
    is the device exchange (cells and counts on the device, the cut on the
    host from the summed counts, packing, NCCL all-to-all, unpacking) plus the
    captured build + pairs + PP of the rank's local set with its own
    particles active.  value = the whole box's interactions within R_cut per
    second of the slowest rank's step."""
    import torch
    import torch.distributed as dist
    from paper_1802_09824_gb300 import binding as B
    from paper_1802_09824_gb300 import domain, synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist.init_process_group("nccl", device_id=dev) if world > 1 else dist.init_process_group(
        "nccl", init_method="tcp://127.0.0.1:%d" % (29500 + os.getpid() % 1000), rank=0, world_size=1, device_id=dev)
    ranks = Ranks(dist, dev)
    ps = synth.workload(args.workload, scale=args.scale or None)
    bp = ps.boxes[0]
    prm = _params(B, bp, args.leaf_max or 32, 1, args.pp_variant)
    sl = slice(rank * ps.n // world, (rank + 1) * ps.n // world)
    pos = torch.from_numpy(ps.pos[sl]).to(dev)
    mass = torch.from_numpy(ps.mass[sl]).to(dev)
    ids = torch.arange(sl.start, sl.stop, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    step = domain.PartitionedStep(prm)
    for _ in range(max(args.warmup, 3)):
        step(pos, mass, ids, stream)
    torch.cuda.synchronize()
    B.ph_status(step.lv)
    B.ph_status(step.pr)
    n_local, n_own = step.n_local, step.n_own
    clocks = ClockSampler(_gpu_index(local_rank))
    clocks.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    ranks.barrier()
    torch.cuda.synchronize()
    launches0 = B.ph_launch_counter()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step(pos, mass, ids, stream)
        evs[k][1].record(stream)
    ranks.barrier()
    torch.cuda.synchronize()
    launches = B.ph_launch_counter() - launches0
    B.ph_status(step.pr)
    t_step = ranks.max(sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps)
    # end to end: the shard copied in from pinned host memory, the step, the
    # own particles' accelerations copied out
    pos_h = torch.from_numpy(ps.pos[sl]).pin_memory()
    acc_h = torch.empty((n_own, 3), dtype=torch.float32).pin_memory()
    ranks.barrier()
    e2e_ms = []
    for k in range(max(args.steps // 2, 3)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pos.copy_(pos_h, non_blocking=True)
        _, a_own = step(pos, mass, ids, stream)
        acc_h[:a_own.shape[0]].copy_(a_own, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    ranks.barrier()
    clk = clocks.stop()
    t_e2e = ranks.max(sum(e2e_ms) / len(e2e_ms))
    # the whole box's interactions within R_cut (counted once, untimed)
    n_within = 0
    if rank == 0:
        wp = torch.from_numpy(ps.pos).to(dev)
        wm = torch.from_numpy(ps.mass).to(dev)
        lv = B.ph_build_leaves(wp, wm, prm, stream)
        pr = B.ph_leaf_pairs(lv, stream)
        n_within = B.ph_count_within(lv, pr, stream)
        B.ph_free(pr)
        B.ph_free(lv)
        del wp, wm
    n_within = ranks.sum(n_within)
    own_total = ranks.sum(n_own)
    local_max = ranks.max(n_local)
    step.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": n_within / (t_step * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload + (f"@{args.scale}" if args.scale else ""), "n": ps.n,
                       "leaf_max": prm.leaf_max, "key": "hilbert", "group_size": 32,
                       "l2": "flushed between steps (256 MB write), per-step CUDA events",
                       "parallelism": f"domains{world} (Sec. 4.1 cut along the Peano-Hilbert curve, ghost cells, "
                                      "device exchange over NCCL)"},
            "e2e": {"value": n_within / (t_e2e * 1e-3), "unit": UNIT, "ms_per_step": t_e2e,
                    "h2d_bytes_per_step": int(ps.n * 12), "d2h_bytes_per_step": int(own_total * 12),
                    "call": "domain.PartitionedStep from pinned host shards"},
            "gpu_launches": launches, "clocks": clk,
            "partition": {"own_particles": own_total, "largest_local_set": local_max},
        }
        emit(line, args)
    dist.destroy_process_group()


def emit(line, args):
    """The run's one JSON line: on stdout, and appended to the --jsonl file
    (one line per run, so successive runs form a JSONL log)."""
    text = json.dumps(line)
    print(text, flush=True)
    path = getattr(args, "jsonl", None)
    if path:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "a") as f:
            f.write(text + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="zeldovich_128")
    ap.add_argument("--scale", type=int, default=0, help="side count of a smaller lattice (profiling)")
    ap.add_argument("--leaf-max", type=int, default=0)
    ap.add_argument("--key", type=int, default=0)
    ap.add_argument("--pp-variant", type=int, default=0, help="PP kernel shape when the autotuner is off")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the learned-factor and 512-box measurements")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (leaf_max 32)")
    ap.add_argument("--partitioned", action="store_true",
                    help="the domain-decomposed step (default with several ranks; with one rank the whole-box step "
                         "is the default)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several ranks: independent whole-box replicas instead of the domain decomposition")
    ap.add_argument("--jsonl", default="", help="also append the result line to this file (a JSONL run log)")
    args = ap.parse_args()
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.partitioned or (world > 1 and not args.replicas):
        run_partitioned(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
