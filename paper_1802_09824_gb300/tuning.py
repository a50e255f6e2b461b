"""JSON cache for the in-project autotuner (ph_autotune in the library).

The timing itself runs in the library; this module only remembers the
winning knobs per workload signature so that a workload of the same shape
is not re-tuned: the number of boxes, the particle count and the mean
number of particles per ground cell (rounded to a factor of 1.5) and
R_cut/R_s.  The key kind is one of the tuned knobs.
"""
from __future__ import annotations

import json
import math
import os

KNOBS = ("leaf_max", "level_bits", "pp_variant", "group_size", "key_kind")


def default_cache_path() -> str:
    return os.environ.get("PHPP_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "phpp", "tune.json"))


def _ground_cells(L, rcut):
    g = 0
    while g < 7 and L / 2.0 ** (g + 1) >= rcut:
        g += 1
    return 8 ** g


def signature(box_offsets, params_list) -> str:
    nb = len(params_list)
    n = int(box_offsets[-1])
    cells = sum(_ground_cells(p.L, p.rcut) for p in params_list)
    dens = n / max(cells, 1)
    dbin = round(math.log(max(dens, 1e-9)) / math.log(1.5))
    nbin = round(math.log(max(n, 1)) / math.log(1.5))
    p0 = params_list[0]
    return f"b{nb}-n{nbin}-d{dbin}-u{p0.rcut / p0.rs:.4g}"


def load(path=None) -> dict:
    path = path or default_cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(entry_key, knobs, ms, path=None):
    path = path or default_cache_path()
    data = load(path)
    data[entry_key] = {"knobs": knobs, "ms": ms}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(params_list, knobs):
    for p in params_list:
        for k in KNOBS:
            setattr(p, k, int(knobs[k]))
    return params_list


def tuned(B, pos, mass, box_offsets, params_list, reps=3, path=None, retune=False):
    """params_list with the cached (or freshly measured) best knobs applied.

    Returns (params_list, info) where info says whether the cache was hit and
    carries the per-candidate timings of a fresh run."""
    key = signature(box_offsets, params_list)
    cache = {} if retune else load(path)
    if key in cache:
        return apply(params_list, cache[key]["knobs"]), {"cache": "hit", "key": key, "ms": cache[key]["ms"]}
    res = B.ph_autotune(pos, mass, box_offsets, params_list, reps)
    knobs = {k: int(getattr(res.best, k)) for k in KNOBS}
    tried = [{"leaf_max": res.leaf_max[i], "level_bits": res.level_bits[i], "pp_variant": res.pp_variant[i],
              "group_size": res.group_size[i], "key_kind": res.key_kind[i], "ms": float(res.ms[i])}
             for i in range(res.n_tried)]
    store(key, knobs, float(res.best_ms), path)
    return apply(params_list, knobs), {"cache": "miss", "key": key, "ms": float(res.best_ms), "tried": tried}
