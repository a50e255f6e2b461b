"""Parity at the full sizes of the benchmark workloads, on sampled targets the
FP64 oracle computes one by one (all sources, minimum image, cutoff):

* the 128^3 Zel'dovich lattice in the configuration bench.py times (leaf 32,
  binary levels, Peano-Hilbert keys, 32-particle groups, kernel shape 0,
  the captured step graph), 10^4 random targets plus every particle of the
  8 target groups with the longest source lists;
* the 256^3 NFW mixture (16.8M particles), 10^4 random targets plus every
  particle of the 8 target groups with the longest source lists (the dense
  halo cores that stress the leaf-pair imbalance);
* the 512 batched boxes (9.8M particles) in one graph, random targets in 16
  random boxes;
* the learned factor on the 128^3 lattice against the oracle's FP64 network,
  10^4 random targets (inference parity), and, trained to the benchmark's
  schedule, against the exact FP64 oracle (its 1e-3 force gate).
Tolerances are those of the smaller parity tests (helpers.P99_TOL, MAX_TOL;
the learned path's inference tolerance of tests/test_gpu_mlp.py)."""
import numpy as np
import pytest

from helpers import check_parity, rel_errors
from oracle import force
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _dense_targets(B, lv, pr, n_groups=8):
    lview = B.ph_leaves_get_view(lv)
    pview = B.ph_pairs_get_view(pr)
    off = pview["group_off"].cpu().numpy()
    longest = np.argsort(np.diff(off))[-n_groups:]
    gf = lview["group_first"].cpu().numpy()
    perm = lview["perm"].cpu().numpy()
    return np.concatenate([perm[gf[g]:gf[g + 1]] for g in longest])


def test_zeldovich_128_bench_configuration(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("zeldovich_128")
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, 32, 1, 0)
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    acc = torch.zeros((ps.n, 3), device="cuda")
    lv = B.ph_build_leaves(pos, mass, prm)
    pr = B.ph_leaf_pairs(lv)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25)
    for _ in range(2):
        B.ph_graph_launch(g)
    torch.cuda.synchronize()
    B.ph_status(pr)
    rng = np.random.default_rng(101)
    t = np.concatenate([rng.choice(ps.n, 10_000, replace=False), _dense_targets(B, lv, pr)])
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=t)
    q, m = check_parity(acc.cpu().numpy()[t], ref)
    print(f"zeldovich 128^3 (bench configuration): p99 {q:.2e} max {m:.2e}")
    for h in (g, pr, lv):
        B.ph_free(h)


def test_nfw_mixture_256_sampled(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("nfw_mix_256")
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, 32, 1, 0)
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    acc = torch.zeros((ps.n, 3), device="cuda")
    lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    B.ph_status(pr)
    rng = np.random.default_rng(102)
    t = np.concatenate([rng.choice(ps.n, 10_000, replace=False), _dense_targets(B, lv, pr)])
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=t)
    q, m = check_parity(acc.cpu().numpy()[t], ref)
    print(f"NFW mixture 256^3: p99 {q:.2e} max {m:.2e} over {t.size} targets")
    for h in (pr, lv):
        B.ph_free(h)


def test_batch_512_sampled(gpu_lib):
    import torch
    B = gpu_lib
    ps = synth.workload("batch_512")
    prm = [B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, 32, 1, 0) for bp in ps.boxes]
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    acc = torch.zeros((ps.n, 3), device="cuda")
    lv = B.ph_build_leaves_batched(pos, mass, ps.offsets, prm)
    pr = B.ph_leaf_pairs(lv)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25)
    B.ph_graph_launch(g)
    torch.cuda.synchronize()
    B.ph_status(pr)
    got = acc.cpu().numpy()
    rng = np.random.default_rng(103)
    for b in rng.choice(len(ps.boxes), 16, replace=False):
        sl = ps.box_slice(b)
        bp = ps.boxes[b]
        n_b = sl.stop - sl.start
        t = rng.choice(n_b, min(128, n_b), replace=False)
        ref = force.accel(ps.pos[sl], ps.mass[sl], bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=t)
        check_parity(got[sl][t], ref)
    for h in (g, pr, lv):
        B.ph_free(h)


def test_learned_factor_128_sampled(gpu_lib):
    # inference parity: the GPU's tensor-core network against the oracle's
    # FP64 evaluation of the same weights (a network trained briefly on the
    # GPU; its accuracy against the exact factor is judged elsewhere)
    import torch
    B = gpu_lib
    ps = synth.workload("zeldovich_128")
    bp = ps.boxes[0]
    tp = B.make_train_params(n_samples=1_000_000, batch=4096, steps=20_000, lr0=1e-2, lr_min=1e-5, tol=1.0, seed=9)
    m = B.ph_mlp_train(tp, bp.rs, bp.rcut)
    w, err, loss = B.ph_mlp_get(m)
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, 32, 1, 0)
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    acc = torch.zeros((ps.n, 3), device="cuda")
    lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_LEARNED, m, acc)
    torch.cuda.synchronize()
    rng = np.random.default_rng(104)
    t = rng.choice(ps.n, 10_000, replace=False)
    ref = force.accel_mlp(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rcut, w.astype(np.float64), targets=t)
    got = acc.cpu().numpy()[t].astype(np.float64)
    am = np.linalg.norm(ref, axis=1)
    e = np.linalg.norm(got - ref, axis=1) / np.maximum(am, 1e-3 * np.median(am))
    print(f"learned 128^3: p99 {np.percentile(e, 99):.2e} max {e.max():.2e} (network error {err:.2e})")
    assert np.percentile(e, 99) <= 1e-4 and e.max() <= 1e-3
    for h in (pr, lv, m):
        B.ph_free(h)


def test_learned_factor_meets_its_force_gate_at_128(gpu_lib):
    """The learned factor's accuracy gate at full size: a network trained to
    the benchmark's schedule (400k Adam steps of 4096 samples, learning rate
    2e-3 cosine to 1e-6) is accepted by the exact path's validation (no
    fallback), and the learned forces on the 128^3 lattice in the benchmark
    configuration are within 1e-3 (p99) of the exact FP64 oracle on 10^4
    random targets plus every particle of the 8 densest groups."""
    import warnings

    import torch
    B = gpu_lib
    ps = synth.workload("zeldovich_128")
    bp = ps.boxes[0]
    tp = B.make_train_params(n_samples=1_000_000, batch=4096, steps=400_000, lr0=2e-3, lr_min=1e-6, tol=1e-3,
                             seed=2024)
    m = B.ph_mlp_train(tp, bp.rs, bp.rcut)
    w, err, loss = B.ph_mlp_get(m)
    assert err <= 1e-3, f"validated network error {err:.3e}"
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, 32, 1, 0)
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    acc = torch.zeros((ps.n, 3), device="cuda")
    with warnings.catch_warnings():
        warnings.simplefilter("error")           # a fallback to the exact factor would warn
        lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_LEARNED, m, acc)
    torch.cuda.synchronize()
    rng = np.random.default_rng(105)
    t = np.concatenate([rng.choice(ps.n, 10_000, replace=False), _dense_targets(B, lv, pr)])
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=t)
    e = rel_errors(acc.cpu().numpy()[t], ref)
    print(f"learned factor vs exact FP64 oracle at 128^3: p99 {np.percentile(e, 99):.2e} max {e.max():.2e} "
          f"(network max |g_hat/g - 1| {err:.2e})")
    assert np.percentile(e, 99) <= 1e-3
    for h in (pr, lv, m):
        B.ph_free(h)

