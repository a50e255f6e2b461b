"""Host logic of the autotuner cache (no GPU: the library call is faked)."""
import types

import numpy as np

from paper_1802_09824_gb300 import binding as B
from paper_1802_09824_gb300 import tuning


class FakeLib:
    calls = 0

    def ph_autotune(self, pos, mass, offs, params, reps):
        FakeLib.calls += 1
        r = types.SimpleNamespace()
        r.best = B.make_params(1, 1, 1e-3, 0.04, 0.18, 48, 0, 16, 3, 1)
        r.best_ms = 1.5
        r.n_tried = 2
        r.ms = [2.0, 1.5]
        r.leaf_max = [32, 48]
        r.level_bits = [1, 3]
        r.pp_variant = [0, 1]
        r.group_size = [32, 16]
        r.key_kind = [0, 1]
        r.best.key_kind = 1
        return r


def test_tuned_caches_and_applies(tmp_path):
    path = str(tmp_path / "tune.json")
    prm = [B.make_params(1.0, 1.0, 1e-3, 1.25 / 32, 4.5 * 1.25 / 32, 32)]
    offs = np.array([0, 4096])
    p1, info1 = tuning.tuned(FakeLib(), None, None, offs, prm, path=path)
    assert info1["cache"] == "miss" and FakeLib.calls == 1
    assert (p1[0].leaf_max, p1[0].level_bits, p1[0].pp_variant, p1[0].group_size, p1[0].key_kind) == (48, 3, 1, 16, 1)
    prm2 = [B.make_params(1.0, 1.0, 1e-3, 1.25 / 32, 4.5 * 1.25 / 32, 32)]
    p2, info2 = tuning.tuned(FakeLib(), None, None, offs, prm2, path=path)
    assert info2["cache"] == "hit" and FakeLib.calls == 1
    assert (p2[0].leaf_max, p2[0].level_bits, p2[0].pp_variant, p2[0].group_size, p2[0].key_kind) == (48, 3, 1, 16, 1)


def test_signature_separates_shapes():
    a = [B.make_params(1.0, 1.0, 1e-3, 1.25 / 32, 4.5 * 1.25 / 32, 32)]
    b = [B.make_params(100.0, 1.0, 0.03, 0.98, 4.39, 32)]
    assert tuning.signature([0, 4096], a) != tuning.signature([0, 2 ** 21], b)
    assert tuning.signature([0, 4096], a) == tuning.signature([0, 4100], a)
