"""Pins of the adaptive KDK oracle (oracle/kdk.py): the step criterion
against its closed form, the clocks against closed forms and an independent
change of variable, second-order convergence on a Kepler orbit and on the
paper's three-body test of the force split, time reversibility, and block
steps against a plain fixed-step loop."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import force, kdk


# ---------------------------------------------------------------- criterion
def test_levels_match_closed_form():
    # k = max(0, ceil(log2(dt / t_acc))), t_acc = sqrt(2 eta eps / |a|),
    # capped at max_level; cases within 1e-9 of a level boundary are skipped
    rng = np.random.default_rng(1)
    acc = rng.normal(size=(5000, 3)) * np.exp(rng.uniform(-8, 16, size=(5000, 1)))
    dt, eta, eps, kmax = 0.03, 0.025, 0.01, 9
    got = kdk.step_levels(acc, dt, eta, eps, kmax)
    t_acc = np.sqrt(2 * eta * eps / np.linalg.norm(acc, axis=1))
    x = np.log2(dt / t_acc)
    ref = np.clip(np.ceil(x), 0, kmax).astype(int)
    ok = np.abs(x - np.round(x)) > 1e-9
    assert ok.sum() > 4900
    assert np.array_equal(got[ok], ref[ok])
    assert got.min() == 0 and got.max() == kmax


# ---------------------------------------------------------------- clocks
def test_einstein_de_sitter_factors_closed_form():
    c = kdk.Clock(kdk.CLOCK_LCDM, H0=1.7, omega_m=1.0, omega_l=0.0)
    a1, a2 = 0.13, 0.37
    # H = H0 a^{-3/2}: int da/(a^2 H) = 2 (sqrt a2 - sqrt a1) / H0,
    # int da/(a^3 H) = 2 (a1^{-1/2} - a2^{-1/2}) / H0
    assert abs(c.kick(a1, a2) - 2 * (math.sqrt(a2) - math.sqrt(a1)) / 1.7) < 1e-12
    assert abs(c.drift(a1, a2) - 2 * (1 / math.sqrt(a1) - 1 / math.sqrt(a2)) / 1.7) < 1e-12


def test_lcdm_kick_is_integral_of_dt_over_a():
    # the kick factor is int dt / a(t); a(t) of flat Lambda-CDM in closed
    # form, a = (Om/OL)^{1/3} sinh(1.5 sqrt(OL) H0 t)^{2/3}, integrated in t
    H0, om, ol = 1.0, 0.3, 0.7
    c = kdk.Clock(kdk.CLOCK_LCDM, H0=H0, omega_m=om, omega_l=ol)

    def a_of_t(t):
        return (om / ol) ** (1 / 3) * math.sinh(1.5 * math.sqrt(ol) * H0 * t) ** (2 / 3)

    def t_of_a(a):
        return 2 / (3 * math.sqrt(ol) * H0) * math.asinh(math.sqrt(ol / om) * a ** 1.5)

    a1, a2 = 0.2, 0.45
    t1, t2 = t_of_a(a1), t_of_a(a2)
    kick = integrate.quad(lambda t: 1 / a_of_t(t), t1, t2, epsabs=0, epsrel=1e-13)[0]
    drift = integrate.quad(lambda t: 1 / a_of_t(t) ** 2, t1, t2, epsabs=0, epsrel=1e-13)[0]
    assert abs(c.kick(a1, a2) - kick) < 1e-10 * kick
    assert abs(c.drift(a1, a2) - drift) < 1e-10 * drift
    assert c.kick(0.3, 0.3) == 0.0


# ---------------------------------------------------------------- integration
def _kepler(n_steps):
    # a test mass on a circular orbit of radius r around a unit mass, deep
    # inside R_s (the split factor is 1 to 1e-7) in a box large enough that
    # the periodic images do not matter; one fixed level
    L, rs = 100.0, 10.0
    r = 0.1
    pos = np.array([[50.0, 50.0, 50.0], [50.0 + r, 50.0, 50.0]])
    v = math.sqrt(1.0 / r)
    mom = np.array([[0.0, 0.0, 0.0], [0.0, v, 0.0]])
    mass = np.array([1.0, 1e-12])
    period = 2 * math.pi * math.sqrt(r ** 3)
    s = kdk.Sim(pos, mom, mass, L, 1.0, 0.0, rs, 4.5 * rs, 0, period / n_steps, 1.0, 0, eps_step=1.0)
    for _ in range(n_steps):
        s.top_step()
    return np.linalg.norm(s.x[1] - pos[1]), s


def test_kepler_orbit_closes_to_second_order():
    e1, s = _kepler(200)
    e2, _ = _kepler(400)
    assert e1 < 5e-3 * 0.1
    assert 3.5 < e1 / e2 < 4.5
    # the speed of a circular orbit is conserved to the same order
    assert abs(np.linalg.norm(s.p[1]) - math.sqrt(10.0)) < 1e-3 * math.sqrt(10.0)


def test_time_reversible():
    rng = np.random.default_rng(2)
    n = 24
    pos = rng.random((n, 3)) * 0.2 + 0.4
    mom = rng.normal(size=(n, 3)) * 0.05
    mass = rng.random(n) / n
    s = kdk.Sim(pos, mom, mass, 1.0, 1.0, 1e-3, 0.04, 0.18, 0, 0.01, 1.0, 0, eps_step=1.0)
    x0 = s.x.copy()
    for _ in range(10):
        s.top_step()
    assert np.max(np.abs(s.x - x0)) > 1e-3
    s.p = -s.p
    for _ in range(10):
        s.top_step()
    assert np.max(np.abs(s.x - x0)) < 1e-12


def test_block_step_on_one_level_is_plain_kdk():
    # eta tiny: every particle goes to the finest level 2, so one top step is
    # four plain KDK steps of dt / 4 (written out directly here)
    rng = np.random.default_rng(3)
    n = 40
    L, G, eps, rs, rcut = 1.0, 1.0, 1e-3, 0.04, 0.18
    pos = rng.random((n, 3))
    mom = rng.normal(size=(n, 3)) * 0.1
    mass = rng.random(n) / n
    dt = 0.02
    s = kdk.Sim(pos, mom, mass, L, G, eps, rs, rcut, 16, dt, 1e-12, 2)
    s.top_step()
    assert np.all(s.level == 2)
    x, p = pos.copy(), mom.copy()
    from oracle import pm

    def F(x):
        return force.accel(x, mass, L, G, eps, rs, rcut).acc + pm.accel(x, mass, L, G, rs, 16).acc

    a = F(x)
    h = dt / 4
    for _ in range(4):
        p = p + a * (h / 2)
        x = x + p * h
        x = x - L * np.floor(x / L)
        a = F(x)
        p = p + a * (h / 2)
    assert np.max(np.abs(s.x - x)) < 1e-12
    assert np.max(np.abs(s.p - p)) < 1e-11 * np.max(np.abs(p))
    assert s.force_passes == 1 + 4


def test_adaptive_levels_follow_fine_reference():
    # a close pair (short steps) among slow particles: the adaptive block
    # steps agree with all particles on the finest level to the step error
    # (3e-5 here) and need fewer force passes
    rng = np.random.default_rng(4)
    n = 16
    pos = rng.random((n, 3))
    pos[1] = pos[0] + np.array([0.004, 0.0, 0.0])
    mom = np.zeros((n, 3))
    mom[1, 1] = 0.5
    mass = np.full(n, 1.0 / n)
    kw = dict(L=1.0, G=1.0, eps=1e-3, rs=0.04, rcut=0.18, n_mesh=16, dt=0.004, max_level=4)
    ad = kdk.Sim(pos, mom, mass, eta=0.02, **kw)
    fine = kdk.Sim(pos, mom, mass, eta=1e-14, **kw)
    for _ in range(3):
        ad.top_step()
        fine.top_step()
    assert ad.level.max() > ad.level.min()
    assert np.all(fine.level == 4)
    d = np.abs(ad.x - fine.x)
    d = np.minimum(d, 1.0 - d)
    assert d.max() < 2e-4
    assert ad.force_passes < fine.force_passes


def three_body(dt, eta, max_level, steps):
    """Sec. 3.4's test of KDK under the force split: a close binary (two
    masses 0.01 at separation 0.05 < R_s, bound by the short-range force)
    on an orbit of radius 1 > R_cut around a unit mass (the long-range PM
    force), in a periodic box of side 4 with a 32^3 mesh.  Returns the
    simulation and, per top step, the binary's centre relative to the
    central mass and its separation vector (minimum image)."""
    L, nm = 4.0, 32
    rs = 1.25 * L / nm
    M, m, R, s = 1.0, 0.01, 1.0, 0.05
    c = np.array([2.0, 2.0, 2.0])
    vorb, vb = math.sqrt(M / R), math.sqrt(2 * m / s) / 2
    pos = np.array([c, c + [R, -s / 2, 0], c + [R, s / 2, 0]])
    mom = np.array([[0, -2 * m * vorb / M, 0], [vb, vorb, 0], [-vb, vorb, 0]])
    mass = np.array([M, m, m], np.float32)
    sim = kdk.Sim(pos, mom, mass, L, 1.0, 0.005, rs, 4.5 * rs, nm, dt, eta, max_level)
    hist = []
    for _ in range(steps):
        sim.top_step()
        cm = (sim.x[1] + sim.x[2]) / 2 - sim.x[0]
        sep = sim.x[1] - sim.x[2]
        hist.append(np.r_[cm - L * np.round(cm / L), sep - L * np.round(sep / L)])
    return sim, np.array(hist)


def test_three_body_split_orbit_is_bound_and_second_order():
    # a quarter of the outer orbit; the binary's steps are 1/16 of the top
    # step (level 4), then 1/32 and 1/64 of it in two finer runs (eta / 4,
    # eta / 16): the binary stays bound and the coarse run converges to the
    # fine one at second order (differences 16 : 4 : 1 -> ratio 5)
    a, ha = three_body(0.1, 0.05, 4, 16)
    b, hb = three_body(0.1, 0.05 / 4, 5, 16)
    c, hc = three_body(0.1, 0.05 / 16, 6, 16)
    assert list(a.level) == [0, 4, 4] and list(c.level) == [2, 6, 6]
    sep = np.linalg.norm(ha[:, 3:], axis=1)
    assert sep.min() > 0.9 * 0.05 and sep.max() < 1.1 * 0.05
    d_ac = np.abs(ha[-1] - hc[-1]).max()
    d_bc = np.abs(hb[-1] - hc[-1]).max()
    assert d_ac < 5e-3
    assert 3.5 < d_ac / d_bc < 7.0
