"""Pins of the particle-mesh (long-range) oracle against what the mathematics
fixes: CIC identities, the discrete Poisson equation in real space, the
Gaussian form of the split filter, momentum conservation, and the periodic
Newtonian force of an Ewald sum for PM + PP together.

None of these re-types the oracle's formula: the Poisson check applies the
7-point stencil in real space, the filter check sums a Gaussian over the
mesh, and the Ewald sum below uses its own splitting parameter."""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import force, pm


# ---------------------------------------------------------------- Ewald sum
def ewald_accel(d, L, G=1.0, m=1.0, alpha=None, n_real=2, k_max=10):
    """Acceleration at the origin from a mass m at d and all its periodic
    images in a cube of side L, with a neutralising uniform background (the
    k = 0 term dropped).  Real-space part with erfc(alpha r), reciprocal part
    over |k_i| <= k_max * 2 pi / L."""
    if alpha is None:
        alpha = 5.0 / L
    d = np.asarray(d, np.float64)
    a = np.zeros(3)
    rng = np.arange(-n_real, n_real + 1)
    img = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3) * L
    dn = d[None, :] + img
    r = np.linalg.norm(dn, axis=1)
    w = erfc(alpha * r) + 2.0 * alpha * r / math.sqrt(math.pi) * np.exp(-(alpha * r) ** 2)
    a += G * m * (dn * (w / r ** 3)[:, None]).sum(0)
    ks = np.arange(-k_max, k_max + 1)
    K = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), -1).reshape(-1, 3)
    K = K[np.any(K != 0, axis=1)] * (2.0 * math.pi / L)
    k2 = (K ** 2).sum(1)
    a += G * m * 4.0 * math.pi / L ** 3 * (K * (np.exp(-k2 / (4 * alpha ** 2)) * np.sin(K @ d) / k2)[:, None]).sum(0)
    return a


def test_ewald_independent_of_alpha_and_newtonian_nearby():
    L = 1.0
    for d in ([0.1, 0.02, -0.03], [0.4, 0.3, 0.1], [0.01, 0.0, 0.0]):
        a1 = ewald_accel(d, L, alpha=4.0)
        a2 = ewald_accel(d, L, alpha=7.0)
        assert np.linalg.norm(a1 - a2) <= 1e-9 * np.linalg.norm(a1)
    d = np.array([0.01, 0.0, 0.0])
    newton = d / np.linalg.norm(d) ** 3
    # the periodic correction at r << L is O(r / L^3) (the images' tidal field)
    assert np.linalg.norm(ewald_accel(d, L) - newton) <= 1e-4 * np.linalg.norm(newton)
    # symmetry: a particle at the half-box point feels nothing
    assert np.linalg.norm(ewald_accel([0.5, 0.5, 0.5], L)) < 1e-9


# ---------------------------------------------------------------- CIC
def test_cic_conserves_mass_and_wraps():
    rng = np.random.default_rng(3)
    pos = rng.random((500, 3)) * 2.0 - 0.5        # outside [0, L) too
    m = rng.random(500)
    g = pm.cic_assign(pos, m, 1.0, 16)
    assert abs(g.sum() - m.sum()) < 1e-12 * m.sum()
    g2 = pm.cic_assign(pos + np.array([1.0, -2.0, 3.0]), m, 1.0, 16)
    assert np.max(np.abs(g2 - g)) < 1e-12


def test_cic_particle_on_node_goes_to_that_node():
    L, n = 1.0, 8
    pos = np.array([[3 / 8, 5 / 8, 0.0]])
    g = pm.cic_assign(pos, [2.0], L, n)
    assert g[3, 5, 0] == 2.0 and np.count_nonzero(g) == 1


def test_cic_interpolation_reproduces_linear_fields():
    # away from the periodic seam a linear field is interpolated exactly by
    # trilinear weights; swapping the two weights of an axis breaks this
    L, n = 1.0, 16
    idx = np.arange(n) * (L / n)
    X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
    field = 0.7 + 2.0 * X - 3.0 * Y + 0.5 * Z
    rng = np.random.default_rng(4)
    pos = 0.1 + 0.7 * rng.random((300, 3))
    got = pm.cic_interp(field, pos, L)
    ref = 0.7 + 2.0 * pos[:, 0] - 3.0 * pos[:, 1] + 0.5 * pos[:, 2]
    assert np.max(np.abs(got - ref)) < 1e-12


def test_cic_assignment_is_adjoint_of_interpolation():
    # sum_nodes M(node) f(node) = sum_p m_p (interp f)(x_p) for every f
    rng = np.random.default_rng(5)
    L, n = 2.0, 12
    pos = rng.random((400, 3)) * L
    m = rng.random(400)
    f = rng.normal(size=(n, n, n))
    lhs = float((pm.cic_assign(pos, m, L, n) * f).sum())
    rhs = float((m * pm.cic_interp(f, pos, L)).sum())
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


# ---------------------------------------------------------------- Poisson solve
def test_potential_solves_discrete_poisson_equation():
    # without the filter (R_s = 0) the potential satisfies the 7-point
    # Laplacian equation nabla^2 phi = 4 pi G (rho - mean rho) in real space
    rng = np.random.default_rng(6)
    L, n, G = 3.0, 16, 0.7
    grid = pm.cic_assign(rng.random((200, 3)) * L, rng.random(200), L, n)
    phi = pm.potential(grid, L, G, 0.0)
    dg = L / n
    lap = sum(np.roll(phi, 1, a) + np.roll(phi, -1, a) - 2 * phi for a in range(3)) / dg ** 2
    rho = grid / dg ** 3
    ref = 4 * math.pi * G * (rho - rho.mean())
    assert np.max(np.abs(lap - ref)) < 1e-10 * np.max(np.abs(ref))
    assert abs(phi.mean()) < 1e-12 * np.max(np.abs(phi))


def test_filter_is_gaussian_smoothing_of_variance_2rs2():
    # multiplying by exp(-k^2 R_s^2) equals convolving the density with a
    # 3-D Gaussian of per-axis variance 2 R_s^2 (the Gaussian whose enclosed
    # mass is 1 - f(s) of Eq. (split)); checked by summing the Gaussian
    # over the mesh (and its periodic images) in real space
    L, n, G = 1.0, 32, 1.0
    dg = L / n
    rs = 1.25 * dg
    grid = np.zeros((n, n, n))
    grid[0, 0, 0] = 1.0
    x = np.arange(n) * dg
    g1 = sum(np.exp(-((x + k * L) ** 2) / (4 * rs * rs)) for k in range(-3, 4))
    gauss = g1[:, None, None] * g1[None, :, None] * g1[None, None, :]
    gauss *= dg ** 3 / (4 * math.pi * rs * rs) ** 1.5      # mass per node
    got = pm.potential(grid, L, G, rs)
    ref = pm.potential(gauss, L, G, 0.0)
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    # a wrong width fails: the factor 2 in the variance is fixed
    wrong = pm.potential(grid, L, G, rs / math.sqrt(2.0))
    assert np.max(np.abs(wrong - ref)) > 1e-2 * np.max(np.abs(ref))


# ---------------------------------------------------------------- forces
def test_momentum_is_conserved():
    rng = np.random.default_rng(7)
    L, n = 1.0, 16
    pos = rng.random((300, 3)) * L
    m = rng.random(300)
    res = pm.accel(pos, m, L, 1.0, 1.25 * L / n, n)
    tot = (m[:, None] * res.acc).sum(0)
    assert np.linalg.norm(tot) < 1e-12 * (m[:, None] * np.abs(res.acc)).sum()


def test_translation_by_one_mesh_cell():
    rng = np.random.default_rng(8)
    L, n = 1.0, 16
    pos = rng.random((200, 3)) * L
    m = rng.random(200)
    a = pm.accel(pos, m, L, 1.0, 1.25 * L / n, n).acc
    b = pm.accel(pos + np.array([L / n, -2 * L / n, 0.0]), m, L, 1.0, 1.25 * L / n, n).acc
    assert np.max(np.abs(a - b)) < 1e-9 * np.max(np.abs(a))


# Plain PM (CIC both ways, 3-point Laplacian, central difference, no window
# deconvolution) at R_s = 1.25 mesh cells: the long-range part of a pair
# force is a few percent off within a few R_s (Sec. 3.1 notes that PM
# loses accuracy below a few mesh cells) and converges beyond.
@pytest.mark.parametrize("r_rs,tol", [(1.0, 0.03), (2.0, 0.09), (3.0, 0.09), (6.0, 0.035), (12.0, 0.012)])
def test_pm_plus_pp_matches_ewald_pair_force(r_rs, tol):
    L, n = 1.0, 32
    rs = 1.25 * L / n
    rcut = 4.5 * rs
    rng = np.random.default_rng(9 + int(r_rs))
    for _ in range(6):
        x0 = rng.random(3) * L
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x1 = x0 + u * r_rs * rs
        pos = np.array([x0, x1])
        mass = np.array([1e-12, 1.0])
        lr = pm.accel(pos, mass, L, 1.0, rs, n, targets=[0]).acc[0]
        sr = force.accel(pos, mass, L, 1.0, 0.0, rs, rcut, targets=np.array([0])).acc[0]
        ew = ewald_accel(x1 - x0, L)
        assert np.linalg.norm(lr + sr - ew) <= tol * np.linalg.norm(ew)


def test_pm_plus_pp_matches_ewald_many_bodies():
    # 64 particles: every pair at once, against the Ewald sum over all sources
    rng = np.random.default_rng(10)
    L, n = 1.0, 32
    rs = 1.25 * L / n
    pos = rng.random((64, 3)) * L
    m = rng.random(64) + 0.5
    lr = pm.accel(pos, m, L, 1.0, rs, n).acc
    sr = force.accel(pos, m, L, 1.0, 0.0, rs, 4.5 * rs).acc
    ref = np.zeros((64, 3))
    for i in range(64):
        for j in range(64):
            if i != j:
                ref[i] += ewald_accel(pos[j] - pos[i], L, m=m[j], n_real=1, k_max=8)
    # the pair errors above add up, and partly cancelling sums amplify them
    e = np.linalg.norm(lr + sr - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.median(e) < 0.035 and e.max() < 0.15
    # without the long-range part the sum is far off: the test discriminates
    e0 = np.linalg.norm(sr - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.median(e0) > 0.3


def test_pm_converges_with_the_mesh_at_second_order():
    # R_s fixed, mesh refined 32 -> 64 -> 128 (R_s = 1.25, 2.5, 5 cells): the
    # discretisation error of PM + PP against Ewald at r = 2 R_s falls about
    # fourfold per halving of the cell (CIC, the 3-point Laplacian and the
    # central difference are all second order)
    L = 1.0
    rs = 1.25 / 32
    rng = np.random.default_rng(12)
    pairs = []
    for _ in range(6):
        x0 = rng.random(3)
        u = rng.normal(size=3)
        pairs.append((x0, x0 + u / np.linalg.norm(u) * 2 * rs))
    med = []
    for n in (32, 64, 128):
        errs = []
        for x0, x1 in pairs:
            pos = np.array([x0, x1])
            mass = np.array([1e-12, 1.0])
            lr = pm.accel(pos, mass, L, 1.0, rs, n, targets=[0]).acc[0]
            sr = force.accel(pos, mass, L, 1.0, 0.0, rs, 4.5 * rs, targets=np.array([0])).acc[0]
            ew = ewald_accel(x1 - x0, L)
            errs.append(np.linalg.norm(lr + sr - ew) / np.linalg.norm(ew))
        med.append(np.median(errs))
    assert med[2] < 6e-3
    assert med[0] / med[1] > 2.5 and med[1] / med[2] > 3.0
