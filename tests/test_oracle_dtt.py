"""The leaf-level tree part of the oracle (oracle/dtt.py) against what fixes
it: theta = 0 and one-particle leaves give back the plain short-range sum, an
accepted leaf acts exactly as one body at its mass centre, and the error
against the plain sum grows with theta."""
import numpy as np

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
    a, n_acc = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.0, leaf_max=16, T=12)
    assert n_acc == 0
    ref = _exact(pos, mass)
    np.testing.assert_allclose(a, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_one_particle_leaves_are_exact_for_any_theta():
    pos, mass = _clustered(800, 2)
    a, n_acc = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.5, leaf_max=1, group_size=8, T=12)
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
    a, n_acc = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, 0.6, leaf_max=8, group_size=8, T=12)
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
        a, n_acc = dtt.accel(pos, mass, 1.0, 1.0, 1e-3, RS, RCUT, th, leaf_max=8, group_size=8, T=14)
        assert n_acc > 0
        errs.append(np.percentile(np.linalg.norm(a - ref, axis=1) / mag, 90))
    assert errs[0] < errs[1] < errs[2]
    assert errs[0] < 1e-2
