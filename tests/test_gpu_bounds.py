"""The library built with its debug bounds checks (libphpp_checked.so).

Every kernel index that csrc/checks.cuh tests must stay inside its buffer on
every path: the checked library runs the short-range step (exact, tabulated
and learned factor; group sizes 8, 16, 32; leaf sizes 1 to 128; the tree
part), many boxes at once, the captured graph, PM, KDK and the device
exchange, in a child process, and ph_debug_bounds must report no access
skipped.  The checks never trap or wait, so a stray index costs nothing but
a count.  The normal library reports that it has no checks."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
from paper_1802_09824_gb300 import binding as B, synth

assert B.ph_debug_bounds() == (0, 0)
dev = "cuda"
runs = 0

def tensors(ps):
    return (torch.from_numpy(ps.pos).to(dev), torch.from_numpy(ps.mass).to(dev),
            torch.zeros((ps.n, 3), dtype=torch.float32, device=dev))

def check(name):
    global runs
    torch.cuda.synchronize()
    hits, site = B.ph_debug_bounds()
    assert hits == 0, (name, hits, site)
    runs += 1

# the step on a uniform box and a clustered one, several shapes
uni = synth.workload("uniform_small", scale=4096)
nfw = synth.workload("nfw_mix_256", scale=24)
for ps in (uni, nfw):
    bp = ps.boxes[0]
    pos, mass, acc = tensors(ps)
    for leaf, gs, var in ((32, 32, 0), (16, 16, 1), (64, 8, 0), (1, 32, 1), (128, 32, 0)):
        prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, leaf, B.PH_KEY_HILBERT, gs, 1, var)
        lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_EXACT, None, acc)
        assert np.all(np.isfinite(acc.cpu().numpy()))
        B.ph_pp_accel(lv, None, B.PH_G_EXACT, None, acc)      # direct mode (no list)
        B.ph_count_within(lv, pr)
        check(f"{{ps.name}} leaf {{leaf}} group {{gs}}")
        B.ph_free(pr); B.ph_free(lv)
    # the tree part, the tabulated and the learned factor, the graph
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, 32, 1, 0, 0.3)
    lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_EXACT, None, acc)
    check("tree"); B.ph_free(pr); B.ph_free(lv)
    prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT)
    lv, pr = B.ph_accel(pos, mass, prm, B.PH_G_TABLE, None, acc)
    check("table")
    w = np.random.default_rng(3).normal(0.0, 0.3, 321).astype(np.float32)
    m = B.ph_mlp_create(w, bp.rs, bp.rcut, tol=1e30)
    for gs in (32, 16, 8):
        prm_g = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32, B.PH_KEY_HILBERT, gs)
        lv2, pr2 = B.ph_accel(pos, mass, prm_g, B.PH_G_LEARNED, m, acc)
        assert np.all(np.isfinite(acc.cpu().numpy()))
        check(f"learned group {{gs}}"); B.ph_free(pr2); B.ph_free(lv2)
    g = B.ph_graph_create(lv, pr, pos, mass, B.PH_G_EXACT, None, acc, headroom=0.25)
    B.ph_graph_launch(g)
    check("graph")
    B.ph_free(g); B.ph_free(m); B.ph_free(pr); B.ph_free(lv)
    # PM
    B.ph_pm_accel(pos, mass, prm, 32, acc, accumulate=True)
    check("pm")

# many boxes in one build
ps = synth.batch_boxes(12, seed=5, n_min=300, n_max=5000)
pos, mass, acc = tensors(ps)
prms = [B.make_params(b.L, b.G, b.eps, b.rs, b.rcut, 32) for b in ps.boxes]
lv = B.ph_build_leaves_batched(pos, mass, ps.offsets, prms)
pr = B.ph_leaf_pairs(lv)
B.ph_pp_accel(lv, pr, B.PH_G_EXACT, None, acc)
check("batched"); B.ph_free(pr); B.ph_free(lv)

# KDK
bp = uni.boxes[0]
prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32)
mom = np.zeros((uni.n, 3), np.float64)
sim = B.ph_sim_create(uni.pos.astype(np.float64), mom, uni.mass, prm, B.make_kdk_params(1e-3, 0.05, 3, 32), 0.0)
B.ph_sim_step(sim, 2)
check("kdk"); B.ph_free(sim)

# the device exchange, two simulated ranks
pos, mass, _ = tensors(uni)
ids = torch.arange(uni.n, dtype=torch.int64, device=dev)
ns, cells, counts = B.ph_domain_cells_device(pos, prm)
owner, _ = B.ph_domain_partition(counts.cpu().numpy(), ns, B.PH_KEY_HILBERT, 2)
send, sc = B.ph_domain_pack(pos, mass, ids, cells, owner, ns, 2)
for r in range(2):
    off = sum(sc[:r])
    B.ph_domain_unpack(send[off:off + sc[r]], sc[r], torch.float32)
check("exchange")
print("ok", runs)
"""


def test_normal_build_has_no_checks():
    # no GPU needed: the normal build refuses before any CUDA call
    from paper_1802_09824_gb300 import binding as B, build
    if not os.path.exists(build.OUT):
        build.build()
    with pytest.raises(RuntimeError, match="without bounds checks"):
        B.ph_debug_bounds()


@pytest.mark.gpu
def test_checked_build_stays_in_bounds():
    from paper_1802_09824_gb300 import build
    so = build.build(checked=True)
    env = dict(os.environ, PHPP_LIB=so)
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], capture_output=True, text=True,
                       timeout=900, env=env)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "ok" in r.stdout
