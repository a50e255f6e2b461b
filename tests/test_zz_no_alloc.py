"""ph_accel_noalloc: the whole exact-factor step without any allocation.

Some callers may not allocate device memory (an application that owns the
whole device-memory budget through its own allocator, or a latency-critical
loop that cannot absorb the device synchronisation of cudaMalloc/cudaFree).
For them the library offers this one entry point, which keeps every
intermediate buffer in a fixed array inside the library.  Here it is called
through the C ABI several times in a row, with different particle sets, up
to its documented limits (16384 particles, 4096 ground cells); each result
is compared element by element with the FP64 oracle (the parity tolerances:
p99 <= 1e-5, max <= 1e-3) and with the allocating entry point ph_accel on the
same input.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from helpers import MAX_TOL, P99_TOL, check_parity, oracle_accel
from paper_1802_09824_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    bm = np.linalg.norm(b, axis=1)
    tau = 1e-3 * np.median(bm)
    return np.linalg.norm(a - b, axis=1) / np.maximum(bm, tau)


def _both(B, ps):
    import torch
    bp = ps.boxes[0]
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, bp.leaf_max)
    pos = torch.from_numpy(ps.pos).cuda()
    mass = torch.from_numpy(ps.mass).cuda()
    ref = torch.zeros((ps.n, 3), dtype=torch.float32, device="cuda")
    lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_EXACT, None, ref)
    got = torch.full((ps.n, 3), float("nan"), dtype=torch.float32, device="cuda")
    B.ph_accel_noalloc(pos, mass, prm, got)
    torch.cuda.synchronize()
    B.ph_free(pr)
    B.ph_free(lv)
    return got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)


def _max_cells_box(n=16384, seed=77):
    """n uniform particles in a unit box with R_cut = 0.05: 16^3 = 4096
    ground cells, the entry point's limit."""
    bp = synth.BoxParams(L=1.0, G=1.0, eps=1e-4, rs=0.05 / 4.5, rcut=0.05, leaf_max=32)
    ps = synth.uniform_box(n, bp, seed)
    ps.mass = (np.random.default_rng(seed + 1).uniform(0.5, 1.5, n) / n).astype(np.float32)
    return ps


def test_noalloc_matches_the_oracle_on_calls_in_a_row(gpu_lib):
    B = gpu_lib
    sets = [synth.workload("uniform_small"),                 # 4096 particles
            synth.workload("zeldovich_128", scale=24),       # 13824 particles
            _max_cells_box(),                                # 16384 particles, 4096 ground cells
            synth.workload("uniform_small")]                 # the first set again after the largest
    for ps in sets:
        got, ref = _both(B, ps)
        assert np.all(np.isfinite(got))
        check_parity(got, oracle_accel(ps))
        e = _rel(got, ref)
        assert float(np.percentile(e, 99)) <= P99_TOL
        assert float(e.max()) <= MAX_TOL


def test_noalloc_rejects_sizes_beyond_its_array(gpu_lib):
    import torch
    B = gpu_lib
    n = 16385
    pos = torch.rand((n, 3), device="cuda")
    acc = torch.zeros((n, 3), device="cuda")
    prm = B.make_params(1.0, 1.0, 1e-3, 1.25 / 32, 4.5 * 1.25 / 32, 32)
    with pytest.raises(B.PhError) as ei:
        B.ph_accel_noalloc(pos, None, prm, acc)
    assert ei.value.code == B.PH_ERR_ARG
    assert "16384" in str(ei.value)
    # R_cut = 0.03 in a unit box: 32^3 ground cells, above the 4096 it holds
    prm = B.make_params(1.0, 1.0, 1e-4, 0.03 / 4.5, 0.03, 32)
    with pytest.raises(B.PhError) as ei:
        B.ph_accel_noalloc(pos[:1000], None, prm, acc[:1000])
    assert ei.value.code == B.PH_ERR_ARG
    assert "4096" in str(ei.value)
