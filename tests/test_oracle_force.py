"""Pins of the FP64 force oracle against what the paper and mathematics fix.

None of these re-types the oracle's formula: each checks it against an
independent closed form, library routine, invariant or brute force.
"""
import math

import numpy as np
import pytest
from scipy.special import gammaincc
from scipy.stats import chi

from oracle import force

RS = 1.25 / 32
RCUT = 4.5 * RS


# ---------------------------------------------------------------- split factor
def test_split_factor_is_regularised_upper_gamma():
    # Eq. (split) equals Q(3/2, u^2), u = s / 2R_s: d/du of both sides is
    # -(4u^2/sqrt(pi)) e^{-u^2} and both are 1 at u = 0.
    s = np.linspace(0.0, 6.0 * RS, 4001)
    u = s / (2 * RS)
    ref = gammaincc(1.5, u * u)
    got = force.split_factor(s, RS)
    assert np.max(np.abs(got - ref)) < 1e-14   # a few ulp of erfc + exp in double


def test_split_factor_is_gaussian_enclosed_mass_complement():
    # 1 - f(s) is the mass fraction of a 3-D Gaussian of per-axis sigma
    # sqrt(2) R_s that lies inside radius s: the long-range part is the force
    # of the Gaussian-smoothed point mass (the filter of Sec. 3.1).
    s = np.linspace(1e-3, 5.0, 500) * RS
    ref = chi(3).sf(s / (math.sqrt(2.0) * RS))
    got = force.split_factor(s, RS)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_split_factor_mpmath_50_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for sr in [0.0, 0.01, 0.5, 1.0, 2.0, 3.3, 4.5, 6.0]:
        u = mp.mpf(sr) / 2
        ref = mp.gammainc(mp.mpf(3) / 2, u * u, mp.inf, regularized=True)
        got = force.split_factor([sr * RS], RS)[0]
        assert abs(got - float(ref)) < 1e-14


def test_split_factor_printed_constants():
    # f(0) = 1 and the value at R_cut = 4.5 R_s (Sec. 3.1) that makes the
    # hard cutoff a truncation of ~1.75% of the Newtonian force.
    assert force.split_factor([0.0], RS)[0] == 1.0
    assert abs(force.split_factor([4.5 * RS], RS)[0] - 0.017532933) < 1e-8


def test_split_factor_derivative():
    # df/du = -(4 u^2 / sqrt(pi)) exp(-u^2) by central differences.
    u = np.linspace(0.05, 2.9, 60)
    h = 1e-5
    fp = force.split_factor((u + h) * 2 * RS, RS)
    fm = force.split_factor((u - h) * 2 * RS, RS)
    num = (fp - fm) / (2 * h)
    ref = -4.0 * u * u / math.sqrt(math.pi) * np.exp(-u * u)
    assert np.max(np.abs(num - ref)) < 1e-8


def test_split_factor_newtonian_limit():
    # 1 - f ~ (4 / (3 sqrt(pi))) u^3 for u -> 0 (the force is Newtonian for
    # r << R_s).
    u = np.array([1e-3, 3e-3, 1e-2])
    got = 1.0 - force.split_factor(u * 2 * RS, RS)
    ref = 4.0 / (3.0 * math.sqrt(math.pi)) * u ** 3
    assert np.all(np.abs(got / ref - 1.0) < 1e-3)


# ---------------------------------------------------------------- pair force
def _two_body(x1, x2, m1=0.7, m2=0.3, L=1.0, G=1.3, eps=1e-3):
    pos = np.array([x1, x2], np.float64)
    mass = np.array([m1, m2])
    return force.accel(pos, mass, L, G, eps, RS, RCUT).acc


@pytest.mark.parametrize("r", [0.003, 0.02, 0.05, 0.1, 0.17])
def test_two_body_closed_form(r):
    G, eps, m1, m2 = 1.3, 1e-3, 0.7, 0.3
    d = np.array([0.6, -0.48, 0.64])
    d = d / np.linalg.norm(d) * r
    x1 = np.array([0.4, 0.5, 0.45])
    acc = _two_body(x1, x1 + d, m1, m2, G=G, eps=eps)
    f = gammaincc(1.5, (r / (2 * RS)) ** 2)   # factor via the incomplete gamma
    mag = G * r / (r * r + eps * eps) ** 1.5 * f
    np.testing.assert_allclose(acc[0], m2 * mag * d / r, rtol=1e-13, atol=0)
    np.testing.assert_allclose(acc[1], -m1 * mag * d / r, rtol=1e-13, atol=0)


def test_two_body_across_periodic_face():
    # A pair straddling the x face of the box feels the same force as the
    # same pair in the middle of the box (minimum image).
    d = np.array([0.07, 0.01, -0.02])
    inner = _two_body(np.array([0.5, 0.5, 0.5]), np.array([0.5, 0.5, 0.5]) + d)
    across = _two_body(np.array([0.98, 0.5, 0.5]), np.array([0.98 + d[0] - 1.0, 0.5 + d[1], 0.5 + d[2]]))
    np.testing.assert_allclose(across, inner, rtol=1e-11)


def test_cutoff_is_strict():
    # r just below rcut contributes the truncated force, just above nothing.
    x1 = np.array([0.3, 0.3, 0.3])
    inside = _two_body(x1, x1 + np.array([RCUT * (1 - 1e-9), 0, 0]))
    outside = _two_body(x1, x1 + np.array([RCUT * (1 + 1e-9), 0, 0]))
    assert inside[0, 0] > 0 and np.all(outside == 0)


def test_newtonian_limit_many_body():
    # With R_s -> infinity the factor is 1: compare with a plain Plummer sum.
    rng = np.random.default_rng(5)
    pos = rng.random((40, 3)) * 0.2 + 0.4
    mass = rng.random(40)
    L, G, eps = 1.0, 1.0, 1e-2
    got = force.accel(pos, mass, L, G, eps, 1e9, 0.45).acc
    d = pos[None, :, :] - pos[:, None, :]
    r2 = np.sum(d * d, axis=2) + eps * eps
    w = mass[None, :] / r2 ** 1.5
    np.fill_diagonal(w, 0.0)
    ref = G * np.einsum("ij,ijk->ik", w, d)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_perfect_lattice_has_zero_force():
    n = 8
    L = 1.0
    g = (np.arange(n) + 0.5) * L / n
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    mass = np.full(pos.shape[0], 1.0 / pos.shape[0])
    # spacing 0.125: neighbours at 0.125 and 0.1768, none at rcut = 0.17578
    r = force.accel(pos, mass, L, 1.0, 1e-3, RS, RCUT)
    assert np.all(r.n_within == 6)
    assert np.max(np.abs(r.acc)) <= 1e-12 * np.max(r.abs_sum)


def test_momentum_conservation():
    rng = np.random.default_rng(7)
    n = 600
    pos = rng.random((n, 3))
    mass = rng.random(n)
    r = force.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT)
    net = np.sum(mass[:, None] * r.acc, axis=0)
    assert np.max(np.abs(net)) <= 1e-12 * np.sum(mass * r.abs_sum)


def test_translation_and_axis_permutation():
    rng = np.random.default_rng(8)
    n = 300
    pos = rng.random((n, 3))
    mass = rng.random(n)
    base = force.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT)
    shifted = np.mod(pos + np.array([0.3, 0.77, 0.51]), 1.0)
    r2 = force.accel(shifted, mass, 1.0, 1.0, 1e-3, RS, RCUT)
    tol = 1e-11 * np.max(base.abs_sum)
    assert np.max(np.abs(r2.acc - base.acc)) < tol
    perm_axes = pos[:, [2, 0, 1]]
    r3 = force.accel(perm_axes, mass, 1.0, 1.0, 1e-3, RS, RCUT)
    assert np.max(np.abs(r3.acc - base.acc[:, [2, 0, 1]])) < tol
    p = rng.permutation(n)
    r4 = force.accel(pos[p], mass[p], 1.0, 1.0, 1e-3, RS, RCUT)
    assert np.max(np.abs(r4.acc - base.acc[p])) < tol


def test_targets_subset_matches_full():
    rng = np.random.default_rng(9)
    pos = rng.random((500, 3))
    mass = rng.random(500)
    full = force.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT)
    t = np.array([3, 499, 0, 250])
    sub = force.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, targets=t)
    np.testing.assert_array_equal(sub.acc, full.acc[t])


def test_brute_force_mpmath_tiny():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(10)
    n = 7
    pos = rng.random((n, 3)) * 0.3
    pos[0] = [0.99, 0.02, 0.5]   # pairs across faces too
    mass = rng.random(n)
    L, G, eps = 1.0, 1.0, 2e-3
    got = force.accel(pos, mass, L, G, eps, RS, RCUT).acc
    for i in range(n):
        a = [mp.mpf(0)] * 3
        for j in range(n):
            if i == j:
                continue
            d = []
            for k in range(3):
                dk = mp.mpf(float(pos[j, k])) - mp.mpf(float(pos[i, k]))
                dk -= L * mp.nint(dk / L)
                d.append(dk)
            r = mp.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
            if not r < RCUT:
                continue
            f = mp.gammainc(mp.mpf(3) / 2, (r / (2 * RS)) ** 2, mp.inf, regularized=True)
            w = G * mp.mpf(float(mass[j])) * f / (r * r + eps * eps) ** mp.mpf(1.5)
            for k in range(3):
                a[k] += w * d[k]
        for k in range(3):
            assert abs(got[i, k] - float(a[k])) <= 1e-12 * (abs(float(a[k])) + 1e-6)


def test_near_cutoff_bookkeeping():
    x1 = np.array([0.3, 0.3, 0.3])
    pos = np.array([x1, x1 + np.array([RCUT * (1 + 1e-7), 0, 0])])
    r = force.accel(pos, np.ones(2), 1.0, 1.0, 1e-3, RS, RCUT, near_tol=1e-5)
    assert np.all(r.acc == 0) and np.all(r.near_abs > 0)
