"""Pins of the learned-factor oracle: gradients against finite differences,
SiLU against its closed form, Adam's first step, the random streams."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_parameter_count():
    assert M.NPARAM == 321
    assert M.OFF["b3"] == (320, 321)


def test_silu_and_its_derivative():
    a = np.linspace(-8, 8, 101)
    np.testing.assert_allclose(M.silu(a), a / (1 + np.exp(-a)), rtol=1e-15)
    h = 1e-6
    num = (M.silu(a + h) - M.silu(a - h)) / (2 * h)
    np.testing.assert_allclose(M.silu_grad(a), num, rtol=1e-8, atol=1e-10)


def test_forward_matches_explicit_loops():
    rng = np.random.default_rng(0)
    th = rng.standard_normal(M.NPARAM) * 0.5
    z = rng.uniform(-1, 1, 5)
    y, _ = M.forward(th, z)
    W1, b1, W2, b2, W3, b3 = M.unpack(th)
    for n in range(5):
        h1 = [M.silu(W1[j] * z[n] + b1[j]) for j in range(16)]
        h2 = [M.silu(sum(W2[k, j] * h1[j] for j in range(16)) + b2[k]) for k in range(16)]
        assert abs(y[n] - (sum(W3[k] * h2[k] for k in range(16)) + b3)) < 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    th = rng.standard_normal(M.NPARAM) * 0.4
    z = rng.uniform(-1, 1, 64)
    tgt = rng.uniform(0.02, 1.0, 64)
    _, g = M.loss_and_grad(th, z, tgt)
    num = np.empty_like(g)
    h = 1e-6
    for i in range(M.NPARAM):
        e = np.zeros(M.NPARAM)
        e[i] = h
        num[i] = (M.loss_and_grad(th + e, z, tgt)[0] - M.loss_and_grad(th - e, z, tgt)[0]) / (2 * h)
    scale = np.abs(num).max()
    assert np.max(np.abs(g - num)) <= 1e-6 * scale


def test_adam_first_step_is_lr_times_sign():
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> delta = -lr g/(|g|+eps)
    opt = M.Adam(3)
    th = np.zeros(3)
    g = np.array([2.0, -0.5, 1e-3])
    th1 = opt.step(th, g, 0.1)
    np.testing.assert_allclose(th1, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_minimises_a_quadratic():
    opt = M.Adam(2)
    th = np.array([3.0, -2.0])
    for _ in range(3000):
        th = opt.step(th, 2 * (th - np.array([1.0, 0.5])), 0.01)
    np.testing.assert_allclose(th, [1.0, 0.5], atol=1e-3)


def test_splitmix64_reference_values():
    # splitmix64 seeded with 0: the published sequence starts 0xe220a8397b1dcdaf
    assert int(M.splitmix64(0, 0)) == 0xE220A8397B1DCDAF
    assert int(M.splitmix64(0, 1)) == 0x6E789E6AA1B965F4
    u = M.uniform24(7, np.arange(200000))
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 1e-3
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))


def test_training_replica_reduces_the_loss():
    th, losses = M.train(4.5, 20000, 512, 300, 1e-2, 1e-4, seed=3)
    assert losses[-1] < 0.1 * losses[0]


def test_c_factor_matches_numpy_forward():
    from oracle import force
    rng = np.random.default_rng(4)
    th = rng.standard_normal(M.NPARAM) * 0.5
    r = np.linspace(0, 0.17, 9)
    np.testing.assert_allclose(force.mlp_factor(th, r, 0.17578125), M.g_hat(th, r, 0.17578125), rtol=1e-13)


def test_force_with_network_equal_to_split_factor_limit():
    # a network whose output is the constant 1 gives the Newtonian (Plummer)
    # force inside rcut: same as the exact oracle with R_s -> infinity
    from oracle import force
    th = np.zeros(M.NPARAM)
    th[M.OFF["b3"][0]] = 1.0
    rng = np.random.default_rng(5)
    pos = rng.random((300, 3))
    m = rng.random(300)
    a = force.accel_mlp(pos, m, 1.0, 1.0, 1e-3, 0.17578125, th)
    b = force.accel(pos, m, 1.0, 1.0, 1e-3, 1e9, 0.17578125).acc
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10 * np.abs(b).max())
