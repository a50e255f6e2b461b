"""The leaf-level tree part of the oracle (oracle/dtt.py) against what fixes
it: the two opening angles of Sec. 3.3 on box pairs computed by hand, the
acceptance of two clumps whose boxes are known exactly, theta = 0 and
one-particle leaves giving back the plain short-range sum, an accepted leaf
acting exactly as one body at its mass centre, and the error against the
plain sum growing with theta."""
import math

import numpy as np
import pytest

from oracle import dtt, force


def _clustered(n, seed, L=1.0, k=6, sigma=0.02):
    rng = np.random.default_rng(seed)
    cen = rng.uniform(0, L, (k, 3))
    pos = (cen[rng.integers(0, k, n)] + rng.normal(0, sigma, (n, 3))) % L
    return pos.astype(np.float32), np.full(n, 1.0 / n, np.float32)


RS = 1.25 / 32
RCUT = 4.5 * RS


def _exact(pos, mass):
    return force.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT).acc


def test_theta_zero_is_the_plain_sum():
    pos, mass = _clustered(1500, 1)
    r = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.0, leaf_max=16, T=12)
    a, n_acc = r.acc, r.n_accepted
    assert n_acc == 0 and r.n_ambiguous == 0
    ref = _exact(pos, mass)
    np.testing.assert_allclose(a, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_one_particle_leaves_are_exact_for_any_theta():
    pos, mass = _clustered(800, 2)
    r = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.5, leaf_max=1, group_size=8, T=12)
    a, n_acc = r.acc, r.n_accepted
    assert n_acc > 0
    ref = _exact(pos, mass)
    np.testing.assert_allclose(a, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_an_accepted_leaf_is_one_body_at_its_mass_centre():
    # a tight target clump and a tight source clump 0.1 apart (within rcut):
    # with theta 0.6 the source leaf is accepted and its pull on every target
    # is G M d f(r) / (r^2 + eps^2)^(3/2) towards its mass centre
    rng = np.random.default_rng(3)
    tgt = np.array([0.30, 0.30, 0.30]) + rng.normal(0, 1e-3, (8, 3))
    src = np.array([0.40, 0.30, 0.30]) + rng.normal(0, 1e-3, (8, 3))
    pos = np.vstack([tgt, src]).astype(np.float32)
    m_src = rng.uniform(0.5, 1.5, 8)
    mass = np.concatenate([np.full(8, 1e-15), m_src]).astype(np.float32)
    r = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.6, leaf_max=8, group_size=8, T=12)
    a, n_acc = r.acc, r.n_accepted
    assert n_acc >= 1
    ms = mass[8:].astype(np.float64)
    M = ms.sum()
    mc = (ms[:, None] * pos[8:].astype(np.float64)).sum(axis=0) / M
    d = mc[None, :] - pos[:8].astype(np.float64)
    r = np.linalg.norm(d, axis=1)
    want = M * d * (force.split_factor_np(r, RS) / (r * r + 1e-6) ** 1.5)[:, None]
    # the targets' own masses (1e-15) pull each other too, below the tolerance
    np.testing.assert_allclose(a[:8], want, rtol=1e-6)


def test_error_grows_with_theta():
    pos, mass = _clustered(3000, 4, sigma=0.01)
    ref = _exact(pos, mass)
    mag = np.linalg.norm(ref, axis=1)
    errs = []
    for th in (0.2, 0.4, 0.7):
        r = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, th, leaf_max=8, group_size=8, T=14)
        a, n_acc = r.acc, r.n_accepted
        assert n_acc > 0
        errs.append(np.percentile(np.linalg.norm(a - ref, axis=1) / mag, 90))
    assert errs[0] < errs[1] < errs[2]
    assert errs[0] < 1e-2


# Box pairs with their opening angles worked out by hand from Sec. 3.3:
# theta_1 = (A + B) / R, theta_2 = B / (R - A), A the target node's side
# width, B the source node's, R the distance of the centres.  Each row names
# the slip it would expose.
ANGLE_CASES = [
    # A,    B,    R,    theta_1,   theta_2,            theta, accepted
    (0.2, 0.2, 1.0, 0.4, 0.25, 0.3, False),              # half widths would give 0.2 and accept
    (0.2, 0.2, 1.0, 0.4, 0.25, 0.45, True),
    (0.3, 0.3, 2.0, 0.3, 0.3 / 1.7, 0.25, False),       # R^2 > (A+B)/theta would accept (4 > 2.4)
    (0.3, 0.3, 2.0, 0.3, 0.3 / 1.7, 0.35, True),
    (0.06, 0.06, 0.5, 0.24, 0.06 / 0.44, 0.3, True),    # R^2 > (A+B)/theta would reject (0.25 < 0.4)
    (1.0, 1.0, 1.5, 2.0 / 1.5, 2.0, 1.5, False),        # theta_2 decides: dropping it would accept
    (1.0, 1.0, 1.5, 2.0 / 1.5, 2.0, 2.1, True),
    (1.0, 0.2, 1.1, 1.2 / 1.1, 2.0, 1.2, False),        # A and B swapped would give theta_2 = 1/0.9 and accept
    (0.2, 1.0, 1.1, 1.2 / 1.1, 1.0 / 0.9, 1.2, True),
    (1.0, 0.1, 0.9, 1.1 / 0.9, math.inf, 10.0, False),  # R <= A: the source is never accepted
]


@pytest.mark.parametrize("A,B,R,th1,th2,theta,acc", ANGLE_CASES)
def test_opening_angles_by_hand(A, B, R, th1, th2, theta, acc):
    t1, t2 = dtt.opening_angles(A, B, R)
    assert t1 == pytest.approx(th1, rel=1e-15)
    assert t2 == pytest.approx(th2, rel=1e-15) if math.isfinite(th2) else t2 == math.inf
    assert dtt.accepted(A, B, R, theta) is acc
    # the flip distance sits between the accepted and rejected sides
    if math.isfinite(th2):
        Rt = dtt.threshold_distance(A, B, theta)
        assert (R > Rt) is acc


def test_side_width_is_the_largest_full_side():
    assert dtt.side_width(np.array([0.1, 0.05, 0.02])) == pytest.approx(0.2, rel=1e-15)
    assert dtt.side_width(np.array([0.01, 0.3, 0.02])) == pytest.approx(0.6, rel=1e-15)


def _two_cubes(c_t, a, c_s, b, m_s=1.0):
    """Eight particles on the corners of a cube of side a around c_t (tiny
    masses) and eight on the corners of a cube of side b around c_s."""
    corners = np.array([[i, j, k] for i in (-0.5, 0.5) for j in (-0.5, 0.5) for k in (-0.5, 0.5)])
    pos = np.vstack([np.asarray(c_t) + a * corners, np.asarray(c_s) + b * corners])
    mass = np.concatenate([np.full(8, 1e-15), np.full(8, m_s / 8)])
    return pos, mass


def test_acceptance_of_two_clumps_with_known_boxes():
    # target cube of side 0.02 around (0.28, 0.28, 0.28), source cube of side
    # 0.008 around (0.38, 0.28, 0.28): both lie inside cells of the key grid
    # that hold nothing else, so each clump is one leaf and one group.
    # Group 0 -> leaf 1: A = 0.02, B = 0.008, R = 0.1: theta_1 = 0.28,
    # theta_2 = 0.1; group 1 -> leaf 0: theta_1 = 0.28, theta_2 = 0.02/0.092.
    pos, mass = _two_cubes([0.28, 0.28, 0.28], 0.02, [0.38, 0.28, 0.28], 0.008)
    kw = dict(leaf_max=8, group_size=8, T=12)
    assert dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.29, **kw).n_accepted == 2
    assert dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.27, **kw).n_accepted == 0
    # near the threshold the pair is flagged ambiguous, with the difference
    # of the two treatments as its slack
    r = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.28 * (1 + 1e-9), band=1e-6, **kw)
    assert r.n_ambiguous == 2 and np.all(r.amb_abs > 0)


def test_theta_2_decides_when_the_boxes_are_close():
    # side 0.1 cubes around x = 0.305 and x = 0.435 (R = 0.13): theta_1 =
    # 0.2/0.13 = 1.54, theta_2 = 0.1/0.03 = 3.33: rejected at theta 2 (only
    # theta_2 forbids it), accepted at 3.5
    pos, mass = _two_cubes([0.305, 0.305, 0.305], 0.1, [0.435, 0.305, 0.305], 0.1)
    kw = dict(leaf_max=8, group_size=8, T=12)
    assert dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 2.0, **kw).n_accepted == 0
    assert dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 3.5, **kw).n_accepted == 2
