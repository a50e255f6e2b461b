"""Exact-factor PP forces through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from helpers import check_parity, gpu_accel, oracle_accel, rel_errors
from oracle import force
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1])
def test_uniform_4096_full(gpu_lib, kind):
    ps = synth.workload("uniform_small")
    got, lv, pr = gpu_accel(gpu_lib, ps, key_kind=kind)
    ref = oracle_accel(ps)
    q, m = check_parity(got, ref)
    print(f"uniform 4096 p99 {q:.2e} max {m:.2e}")
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


@pytest.mark.parametrize("level_bits", [1, 3])
@pytest.mark.parametrize("leaf_max", [1, 8, 64, 256])
def test_leaf_size_does_not_change_result(gpu_lib, leaf_max, level_bits):
    ps = synth.workload("uniform_small", scale=3000)
    got, lv, pr = gpu_accel(gpu_lib, ps, leaf_max=leaf_max, level_bits=level_bits)
    check_parity(got, oracle_accel(ps))
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_zeldovich_32cubed_full(gpu_lib):
    ps = synth.workload("zeldovich_128", scale=32)
    got, lv, pr = gpu_accel(gpu_lib, ps)
    q, m = check_parity(got, oracle_accel(ps))
    print(f"zeldovich 32^3 p99 {q:.2e} max {m:.2e}")
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_nfw_mixture_small_full(gpu_lib):
    ps = synth.workload("nfw_mix_256", scale=32)
    got, lv, pr = gpu_accel(gpu_lib, ps)
    q, m = check_parity(got, oracle_accel(ps))
    print(f"nfw mix 32^3 p99 {q:.2e} max {m:.2e}")
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_float64_and_host_buffers(gpu_lib):
    ps = synth.workload("uniform_small", scale=2500)
    ref = oracle_accel(ps)
    a, lv, pr = gpu_accel(gpu_lib, ps, pos_dtype=np.float64)
    check_parity(a, ref)
    b, lv2, pr2 = gpu_accel(gpu_lib, ps, host=True)
    check_parity(b, ref)
    for h in (pr, lv, pr2, lv2):
        gpu_lib.ph_free(h)


def test_batched_equals_per_box_bitwise(gpu_lib):
    ps = synth.batch_boxes(6, seed=7, n_min=500, n_max=4000)
    got, lv, pr = gpu_accel(gpu_lib, ps)
    for b in range(6):
        sl = ps.box_slice(b)
        one = synth._single(ps.pos[sl], ps.mass[sl], ps.boxes[b], "one")
        a1, l1, p1 = gpu_accel(gpu_lib, one)
        np.testing.assert_array_equal(got[sl], a1)
        check_parity(a1, oracle_accel(ps, box=b))
        gpu_lib.ph_free(p1)
        gpu_lib.ph_free(l1)
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_momentum_and_lattice(gpu_lib):
    ps = synth.workload("uniform_small", scale=3000)
    got, lv, pr = gpu_accel(gpu_lib, ps)
    ref = oracle_accel(ps)
    net = np.abs((ps.mass[:, None] * got.astype(np.float64)).sum(0))
    assert np.all(net <= 1e-5 * np.sum(ps.mass * ref.abs_sum))
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)
    rs = 1.25 / 32
    lat = synth.cubic_lattice(16, synth.BoxParams(1.0, 1.0, 1e-3, rs, 4.5 * rs, 32))
    got, lv, pr = gpu_accel(gpu_lib, lat)
    ref = oracle_accel(lat)
    assert np.max(np.abs(got)) <= 1e-6 * np.max(ref.abs_sum)
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_tiny_and_degenerate(gpu_lib):
    import torch
    B = gpu_lib
    rs = 1.25 / 32
    bp = synth.BoxParams(1.0, 1.0, 1e-3, rs, 4.5 * rs, 32)
    # N = 0
    e = synth._single(np.zeros((0, 3), np.float32), np.zeros(0, np.float32), bp, "e")
    got, lv, pr = gpu_accel(B, e)
    assert got.shape == (0, 3)
    B.ph_free(pr); B.ph_free(lv)
    # N = 1: no force
    one = synth._single(np.array([[0.5, 0.5, 0.5]], np.float32), np.ones(1, np.float32), bp, "1")
    got, lv, pr = gpu_accel(B, one)
    assert np.all(got == 0)
    B.ph_free(pr); B.ph_free(lv)
    # two bodies across the periodic face: closed form
    p = np.array([[0.99, 0.5, 0.5], [0.03, 0.51, 0.49]], np.float32)
    two = synth._single(p, np.array([0.3, 0.7], np.float32), bp, "2")
    got, lv, pr = gpu_accel(B, two)
    check_parity(got, oracle_accel(two), p99=1e-6, emax=1e-6)
    B.ph_free(pr); B.ph_free(lv)
    # coincident distinct particles contribute nothing to each other
    p = np.array([[0.2, 0.2, 0.2], [0.2, 0.2, 0.2], [0.25, 0.2, 0.2]], np.float32)
    co = synth._single(p, np.ones(3, np.float32), bp, "co")
    got, lv, pr = gpu_accel(B, co)
    check_parity(got, oracle_accel(co), p99=1e-6, emax=1e-6)
    B.ph_free(pr); B.ph_free(lv)


def test_errors(gpu_lib):
    import torch
    B = gpu_lib
    pos = torch.rand((100, 3), device="cuda")
    with pytest.raises(B.PhError) as ei:
        B.ph_build_leaves(pos, None, B.make_params(1.0, 1.0, 1e-3, 0.1, 0.5, 32))
    assert ei.value.code == B.PH_ERR_RCUT_GE_HALF_L
    with pytest.raises(B.PhError) as ei:
        B.ph_build_leaves(pos, None, B.make_params(1.0, 1.0, 1e-3, 0.1, 0.2, 0))
    assert ei.value.code == B.PH_ERR_ARG
    bad = pos.clone()
    bad[5, 1] = float("nan")
    lv = B.ph_build_leaves(bad, None, B.make_params(1.0, 1.0, 1e-3, 0.04, 0.18, 32))
    with pytest.raises(B.PhError) as ei:
        B.ph_status(lv)
    assert ei.value.code == B.PH_ERR_NONFINITE
    B.ph_free(lv)


def test_zeldovich_128_full_size_sampled(gpu_lib):
    ps = synth.workload("zeldovich_128")
    got, lv, pr = gpu_accel(gpu_lib, ps)
    rng = np.random.default_rng(1)
    t = rng.choice(ps.n, 1500, replace=False)
    bp = ps.boxes[0]
    ref = force.accel(ps.pos, ps.mass, bp.L, bp.G, bp.eps, bp.rs, bp.rcut, targets=t)
    q, m = check_parity(got[t], ref)
    print(f"zeldovich 128^3 sampled p99 {q:.2e} max {m:.2e}")
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_count_within_matches_oracle(gpu_lib):
    B = gpu_lib
    for ps in (synth.workload("uniform_small"), synth.workload("nfw_mix_256", scale=24)):
        got, lv, pr = gpu_accel(B, ps)
        ev, st = B.ph_pp_counters(pr)
        n = B.ph_count_within(lv, pr)
        ref = oracle_accel(ps, box=0)
        exp = int(ref.n_within.sum())
        # pairs within FP32 rounding of rcut may be counted either way
        near = int(np.sum(ref.near_abs > 0))
        assert abs(n - exp) <= near, (n, exp, near)
        assert ev >= n + ps.n and st > 0
        B.ph_free(pr)
        B.ph_free(lv)


def test_large_box_keeps_relative_precision(gpu_lib):
    # FP64 positions near 5e4 in a box of side 1e5 with a clump 0.05 across
    # (mean separation 1.6e-3): FP32 absolute coordinates there are spaced
    # 4e-3 apart (d_ij would be off by tens of percent); the leaf-relative
    # FP32 frames keep the usual parity.  The softening stays above the
    # kernel's floor of ~1e-6 rcut.
    import torch
    B = gpu_lib
    rng = np.random.default_rng(55)
    L = 1.0e5
    centre = np.array([51234.567, 40000.123, 33333.3])
    clump = centre + 0.02 * rng.normal(size=(2000, 3))
    pos = np.concatenate([rng.random((2000, 3)) * L, clump])
    mass = np.full(len(pos), 1.0 / len(pos), np.float32)
    rs = 100.0
    prm = B.make_params(L, 1.0, 1e-3, rs, 4.5 * rs, 32)
    acc = torch.zeros((len(pos), 3), device="cuda")
    lv, pr = B.ph_accel(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), prm, B.PH_G_EXACT, None, acc)
    torch.cuda.synchronize()
    ref = force.accel(pos, mass, L, 1.0, 1e-3, rs, 4.5 * rs)
    q, m = check_parity(acc.cpu().numpy(), ref)
    print(f"large box: p99 {q:.2e} max {m:.2e}")
    for h in (pr, lv):
        B.ph_free(h)


@pytest.mark.parametrize("rcut_rs", [6.0, 8.0, 9.0])
def test_larger_cutoffs_use_higher_degree_factors(gpu_lib, rcut_rs):
    # rcut / rs = 6, 8, 9 take the degree-12, 14 and 16 polynomials of the
    # factor (4.5 takes degree 10)
    rs = 1.25 / 32
    bp = synth.BoxParams(1.0, 1.0, 1e-3, rs, rcut_rs * rs, 32)
    base = synth.workload("uniform_small", scale=3000)
    ps = synth._single(base.pos, base.mass, bp, f"rcut{rcut_rs}")
    got, lv, pr = gpu_accel(gpu_lib, ps)
    q, m = check_parity(got, oracle_accel(ps))
    print(f"rcut = {rcut_rs} rs: p99 {q:.2e} max {m:.2e}")
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)


def test_batched_boxes_with_different_constants(gpu_lib):
    # boxes with their own L, rs, eps and G: the factor constants are read per
    # box (the kernel instantiation without shared constants), each box
    # against its own oracle
    rng = np.random.default_rng(61)
    boxes, pos, mass = [], [], []
    for k, (L, rs_frac, eps, G, n) in enumerate([(1.0, 1.25 / 32, 1e-3, 1.0, 1500), (3.0, 1.25 / 20, 5e-3, 0.5, 2000),
                                                 (0.5, 1.25 / 24, 2e-4, 2.0, 1200)]):
        rs = rs_frac * L
        boxes.append(synth.BoxParams(L, G, eps, rs, 4.5 * rs, 32))
        pos.append((rng.random((n, 3)) * L).astype(np.float32))
        mass.append(rng.random(n).astype(np.float32) / n)
    offs = np.concatenate([[0], np.cumsum([len(p) for p in pos])]).astype(np.int64)
    ps = synth.ParticleSet(np.concatenate(pos), np.concatenate(mass), boxes, offs, "mixed")
    got, lv, pr = gpu_accel(gpu_lib, ps)
    for b in range(len(boxes)):
        sl = ps.box_slice(b)
        check_parity(got[sl], oracle_accel(ps, box=b))
    gpu_lib.ph_free(pr)
    gpu_lib.ph_free(lv)
