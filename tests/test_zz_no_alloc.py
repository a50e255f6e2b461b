"""ph_accel_noalloc: the whole exact-factor step without any allocation.

Some callers may not allocate device memory (an application that owns the
whole device-memory budget through its own allocator, or a latency-critical
loop that cannot absorb the device synchronisation of cudaMalloc/cudaFree).
For them the library offers this one entry point, which keeps every
intermediate buffer in a fixed array inside the library.  Here it is called
through the C ABI twice in a row, with two different particle sets, and each
result is compared with the allocating entry point ph_accel on the same
input, with the tolerances the parity tests use (p99 <= 1e-5, max <= 1e-3 of
the relative difference).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from helpers import MAX_TOL, P99_TOL
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


def test_noalloc_matches_allocating_entry_point_twice(gpu_lib):
    B = gpu_lib
    first = synth.workload("uniform_small")                       # 4096 particles
    second = synth.workload("zeldovich_128", scale=24)             # 13824 particles
    for ps in (first, second):
        got, ref = _both(B, ps)
        assert np.all(np.isfinite(got))
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
