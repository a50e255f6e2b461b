"""A step whose first PP launch happens inside a stream capture.

The learned and tabulated PP kernels opt in to more than 48 KB of shared
memory; the captured step must work (and replay the direct call bit for bit)
in a fresh process whose very first launch of those kernels is the one that
ph_graph_create captures."""
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

mode = sys.argv[1]
ps = synth.workload("uniform_small", scale=3000)
bp = ps.boxes[0]
prm = B.make_params(bp.L, bp.G, bp.eps, bp.rs, bp.rcut, 32)
pos = torch.from_numpy(ps.pos).cuda()
mass = torch.from_numpy(ps.mass).cuda()
acc = torch.zeros((ps.n, 3), device="cuda")
m = None
if mode == "learned":
    w = np.zeros(321, np.float32)
    rng = np.random.default_rng(3)
    w[:] = rng.normal(0.0, 0.3, 321).astype(np.float32)
    m = B.ph_mlp_create(w, bp.rs, bp.rcut, tol=1e30)
g_mode = B.PH_G_LEARNED if mode == "learned" else B.PH_G_TABLE
lv = B.ph_build_leaves(pos, mass, prm)
pr = B.ph_leaf_pairs(lv)
gr = B.ph_graph_create(lv, pr, pos, mass, g_mode, m, acc, headroom=0.2)
B.ph_graph_launch(gr)
torch.cuda.synchronize()
replay = acc.cpu().numpy().copy()
acc.zero_()
B.ph_pp_accel(lv, pr, g_mode, m, acc)
torch.cuda.synchronize()
direct = acc.cpu().numpy()
assert np.all(np.isfinite(direct)) and np.abs(direct).sum() > 0
np.testing.assert_array_equal(replay, direct)
print("ok", mode)
"""


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["learned", "table"])
def test_first_launch_inside_capture(mode):
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT), mode], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert f"ok {mode}" in r.stdout
