"""The seeded synthetic inputs follow their stated recipes (no GPU).

uniform_small: N = 4096 uniform in the unit box, m = 1/N and the split
parameters of the small configuration.  Zel'dovich lattice: the rms
displacement is 0.3 lattice spacings, the displacement field is
irrotational (psi_k parallel to k) with power |psi_k|^2 ~ k^-4 (density
spectrum k^-2 and psi_k = i k delta_k / k^2).  NFW haloes: radii within
r200 with the enclosed-mass profile mu(x)/mu(c), isotropic directions.
Batches: box sizes log-uniform in [2048, 65536], about half NFW boxes."""
import math

import numpy as np
import pytest

from paper_1802_09824_gb300 import synth


def test_uniform_small_recipe():
    ps = synth.workload("uniform_small")
    bp = ps.boxes[0]
    assert ps.n == 4096 and ps.pos.dtype == np.float32 and ps.mass.dtype == np.float32
    assert np.all((ps.pos >= 0) & (ps.pos < 1.0))
    assert np.all(ps.mass == np.float32(1.0 / 4096))
    assert bp.L == 1.0 and bp.G == 1.0 and bp.eps == 1e-3
    assert bp.rs == 1.25 / 32 and bp.rcut == 4.5 * bp.rs and bp.leaf_max == 32


def _displacements(ps, ns):
    a = ps.boxes[0].L / ns
    g = (np.arange(ns) + 0.5) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    d = ps.pos.astype(np.float64) - q
    d -= ps.boxes[0].L * np.round(d / ps.boxes[0].L)
    return d, a


def test_zeldovich_rms_and_parameters():
    ns = 32
    ps = synth.workload("zeldovich_128", scale=ns)
    bp = ps.boxes[0]
    d, a = _displacements(ps, ns)
    rms = math.sqrt(float(np.mean(np.sum(d * d, axis=1))))
    assert abs(rms / a - 0.3) < 1e-4
    assert np.all((ps.pos >= 0) & (ps.pos < bp.L))
    assert abs(bp.L - 100.0 * ns / 128) < 1e-12
    assert abs(bp.rs - 1.25 * bp.L / ns) < 1e-12 and abs(bp.rcut - 4.5 * bp.rs) < 1e-12
    assert abs(bp.eps - bp.L / ns / 30) < 1e-12


def test_zeldovich_field_is_irrotational_with_k_minus_4_power():
    ns = 32
    ps = synth.workload("zeldovich_128", scale=ns)
    d, a = _displacements(ps, ns)
    psi = d.reshape(ns, ns, ns, 3)
    pk = np.stack([np.fft.fftn(psi[..., i]) for i in range(3)], axis=-1)
    k1 = np.fft.fftfreq(ns) * ns
    K = np.stack(np.meshgrid(k1, k1, k1, indexing="ij"), axis=-1)
    kk = np.sqrt(np.sum(K * K, axis=-1))
    # (the Nyquist planes of an even grid carry only the real part of i k
    # delta_k, so they are left out)
    m = (kk > 0) & np.all(np.abs(K) < ns // 2, axis=-1)
    # psi_k is parallel to k: the component across k is rounding only
    along = np.sum(pk * K, axis=-1) / np.where(m, kk, 1.0)
    across2 = np.sum(np.abs(pk) ** 2, axis=-1) - np.abs(along) ** 2
    assert np.sum(across2[m]) <= 1e-8 * np.sum(np.abs(pk[m]) ** 2)
    # shell-averaged power ~ k^-4 (fit over 2 <= |k| <= ns/4 in grid units)
    p = np.sum(np.abs(pk) ** 2, axis=-1)
    shells = np.rint(kk).astype(int)
    ks, pw = [], []
    for s in range(2, ns // 4 + 1):
        sel = shells == s
        ks.append(np.mean(kk[sel]))
        pw.append(np.mean(p[sel]))
    slope = np.polyfit(np.log(ks), np.log(pw), 1)[0]
    assert abs(slope + 4.0) < 0.4, slope


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def test_nfw_halo_profile_and_isotropy():
    rng = np.random.default_rng(42)
    n, r200, c = 200_000, 2.0, 10.0
    centre = np.array([5.0, 5.0, 5.0])
    p = synth.nfw_halo_positions(rng, n, centre, r200, c)
    v = p - centre
    r = np.linalg.norm(v, axis=1)
    assert r.max() <= r200 * (1 + 1e-12)
    # enclosed-mass fraction against mu(x)/mu(c), x = r c / r200 (KS distance)
    xs = np.sort(r * c / r200)
    cdf = _nfw_mu(xs) / _nfw_mu(c)
    emp = np.arange(1, n + 1) / n
    assert np.max(np.abs(emp - cdf)) < 1.63 / math.sqrt(n) * 1.5   # ~1 % level of a KS test, with margin
    # isotropic directions: mean unit vector ~ 0, second moments ~ 1/3
    u = v / r[:, None]
    assert np.all(np.abs(u.mean(axis=0)) < 5 / math.sqrt(n))
    assert np.all(np.abs(np.mean(u * u, axis=0) - 1 / 3) < 5 / math.sqrt(n))


def test_nfw_mixture_counts_and_masses():
    ns = 32
    ps = synth.workload("nfw_mix_256", scale=ns)
    bp = ps.boxes[0]
    assert ps.n == ns ** 3 and np.all(ps.mass == np.float32(1.0 / ps.n))
    assert np.all((ps.pos >= 0) & (ps.pos < bp.L)) and abs(bp.L - 200.0 * ns / 256) < 1e-12
    # 70 % of the particles in haloes: the densest 1 % of cells of a 16^3
    # grid hold far more than the uniform share (clustering is present)
    h, _ = np.histogramdd(ps.pos.astype(np.float64), bins=16, range=[(0, bp.L)] * 3)
    top = np.sort(h.ravel())[::-1][: h.size // 100].sum() / ps.n
    assert top > 0.1


def test_batch_box_sizes_and_kinds():
    ps = synth.batch_boxes(400, seed=11)
    ns = np.diff(ps.offsets)
    assert ns.min() >= 2048 and ns.max() <= 65536 and len(ps.boxes) == 400
    # log-uniform sizes: KS distance of log N against U[log 2048, log 65536]
    lo, hi = math.log(2048), math.log(65536)
    t = np.sort((np.log(ns) - lo) / (hi - lo))
    emp = np.arange(1, t.size + 1) / t.size
    assert np.max(np.abs(emp - t)) < 1.63 / math.sqrt(t.size) * 1.5
    # masses 1/N_b per box; positions in the unit box
    for b in range(0, 400, 37):
        sl = slice(ps.offsets[b], ps.offsets[b + 1])
        assert np.all(ps.mass[sl] == np.float32(1.0 / ns[b]))
    assert np.all((ps.pos >= 0) & (ps.pos < 1.0))
    # about half of the boxes are single centred haloes: their median radius
    # from the centre is far below a uniform box's (~0.47)
    med = np.array([np.median(np.linalg.norm(ps.pos[ps.offsets[b]:ps.offsets[b + 1]] - 0.5, axis=1))
                    for b in range(400)])
    frac_nfw = float(np.mean(med < 0.3))
    assert abs(frac_nfw - 0.5) < 0.1


@pytest.mark.parametrize("name", ["uniform_small", "zeldovich_128", "nfw_mix_256", "batch_512"])
def test_workloads_are_seeded(name):
    scale = {"uniform_small": 512, "zeldovich_128": 16, "nfw_mix_256": 16, "batch_512": 4}[name]
    a = synth.workload(name, scale=scale)
    b = synth.workload(name, scale=scale)
    np.testing.assert_array_equal(a.pos, b.pos)
    np.testing.assert_array_equal(a.mass, b.mass)
