"""Seeded synthetic particle sets for the short-range PP force.

This module only draws inputs: positions, masses and the box/split
parameters of each workload.  It holds none of the force arithmetic, so both
the CUDA path and the FP64 oracle can be fed from it.

Workloads (all seeds fixed, ``numpy.random.default_rng(seed)``):

* ``uniform_small``  -- N=4096 uniform in the periodic unit box, m=1/N, G=1,
  eps=1e-3, rs=1.25/32, rcut=4.5 rs, leaf size <= 32.
* ``zeldovich_128``  -- 128^3 lattice in L=100 displaced by a Gaussian random
  field whose density spectrum is P(k) ~ k^-2 (Zel'dovich displacement
  psi_k = i k delta_k / k^2), rescaled so that the rms displacement is 0.3 of
  the lattice spacing.  rs = 1.25 L/128, rcut = 4.5 rs, eps = L/128/30.
  This stands in for the paper's 128^3, 100 Mpc/h 2LPTic run (Sec. 5), whose
  initial conditions are not available.
* ``nfw_mix_256``    -- 256^3 particles in L=200: 70% in 10^4 NFW haloes
  (c=10, dN/dM ~ M^-1.9 over three decades), 30% uniform background.
* ``batch_512``      -- 512 independent unit boxes, N per box log-uniform in
  [2048, 65536], each uniform or a single centred NFW halo (c=10,
  r200=0.2 L) with probability 1/2; rs = 1.25/32, rcut = 4.5 rs, eps=1e-3.

Every generator returns float32 positions in [0, L) and float32 masses.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "BoxParams", "ParticleSet", "uniform_box", "zeldovich_lattice",
    "nfw_halo_positions", "nfw_mixture", "batch_boxes", "workload",
    "WORKLOADS", "cubic_lattice",
]


@dataclasses.dataclass(frozen=True)
class BoxParams:
    """Box and split parameters of one periodic box.

    ``rcut`` is the hard cutoff radius, ``rs`` the split scale R_s of the
    short-range factor (Sec. 3.1), ``eps`` the Plummer softening length.
    """
    L: float
    G: float
    eps: float
    rs: float
    rcut: float
    leaf_max: int = 32


@dataclasses.dataclass
class ParticleSet:
    """Particles of one or more boxes, concatenated box after box."""
    pos: np.ndarray            # float32 [N, 3]
    mass: np.ndarray           # float32 [N]
    boxes: list                # list[BoxParams], one per box
    offsets: np.ndarray        # int64 [B+1], particle range of each box
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def box_slice(self, b: int) -> slice:
        return slice(int(self.offsets[b]), int(self.offsets[b + 1]))


def _single(pos, mass, params, name):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    mass = np.ascontiguousarray(mass, dtype=np.float32)
    return ParticleSet(pos, mass, [params], np.array([0, pos.shape[0]], np.int64), name)


def _wrap32(x, L):
    """Map float positions into [0, L) and store them as float32."""
    x = np.mod(np.asarray(x, np.float64), L)
    x32 = x.astype(np.float32)
    # float32 rounding can land exactly on L; fold it back to 0.
    x32[x32 >= np.float32(L)] = 0.0
    return x32


def uniform_box(n: int, params: BoxParams, seed: int, name: str = "uniform") -> ParticleSet:
    rng = np.random.default_rng(seed)
    pos = _wrap32(rng.random((n, 3)) * params.L, params.L)
    mass = np.full(n, 1.0 / n, np.float32)
    return _single(pos, mass, params, name)


def cubic_lattice(n_side: int, params: BoxParams, name: str = "lattice") -> ParticleSet:
    """Perfect cubic lattice of n_side^3 equal masses at cell centres."""
    a = params.L / n_side
    g = (np.arange(n_side) + 0.5) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    n = pos.shape[0]
    return _single(_wrap32(pos, params.L), np.full(n, 1.0 / n, np.float32), params, name)


def zeldovich_lattice(n_side: int, params: BoxParams, seed: int, rms_cells: float = 0.3,
                      name: str = "zeldovich") -> ParticleSet:
    """Lattice displaced by a Zel'dovich field with density spectrum P(k) ~ k^-2.

    A white-noise Gaussian field is filtered by sqrt(P(k)) = 1/k to give
    delta_k; the displacement is psi_k = i k delta_k / k^2 (so that
    div psi = -delta), and the field is rescaled so that the rms length of the
    displacement vector is ``rms_cells`` lattice spacings.
    """
    rng = np.random.default_rng(seed)
    L = params.L
    a = L / n_side
    white = rng.standard_normal((n_side, n_side, n_side))
    wk = np.fft.rfftn(white)
    k1 = np.fft.fftfreq(n_side, d=a) * 2 * np.pi
    kz = np.fft.rfftfreq(n_side, d=a) * 2 * np.pi
    KX, KY, KZ = np.meshgrid(k1, k1, kz, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    k2[0, 0, 0] = 1.0
    delta_k = wk / np.sqrt(k2)
    delta_k[0, 0, 0] = 0.0
    psi = []
    for K in (KX, KY, KZ):
        psi_k = 1j * K * delta_k / k2
        psi.append(np.fft.irfftn(psi_k, s=white.shape, axes=(0, 1, 2)))
    psi = np.stack([p.ravel() for p in psi], axis=1)
    rms = math.sqrt(float(np.mean(np.sum(psi * psi, axis=1))))
    psi *= rms_cells * a / rms
    g = (np.arange(n_side) + 0.5) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    pos = _wrap32(q + psi, L)
    n = pos.shape[0]
    return _single(pos, np.full(n, 1.0 / n, np.float32), params, name)


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def nfw_halo_positions(rng, n: int, centre, r200: float, c: float = 10.0):
    """n points drawn from an NFW profile truncated at r200 (concentration c).

    Radii invert the enclosed-mass fraction mu(x)/mu(c), x = r/r_s_nfw, by
    interpolation on a fine table; directions are isotropic.
    """
    xs = np.linspace(0.0, c, 20001)
    frac = _nfw_mu(xs) / _nfw_mu(c)
    u = rng.random(n)
    x = np.interp(u, frac, xs)
    r = x * (r200 / c)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.asarray(centre)[None, :] + r[:, None] * v


def nfw_mixture(n_side: int, params: BoxParams, seed: int, n_halo: int = 10_000,
                halo_frac: float = 0.7, c: float = 10.0, slope: float = -1.9,
                decades: float = 3.0, min_particles: int = 20,
                name: str = "nfw_mix") -> ParticleSet:
    """Halo mixture: ``halo_frac`` of the particles in NFW haloes, rest uniform.

    Halo masses follow dN/dM ~ M^slope over [M0, 10^decades M0], scaled so the
    haloes hold ``halo_frac`` of the mass; each halo gets round(M/m_p) particles
    (at least ``min_particles``), r200 = (3M / (4 pi 200 rho_bar))^(1/3).
    """
    rng = np.random.default_rng(seed)
    L = params.L
    n = n_side ** 3
    mp = 1.0 / n
    rho_bar = n * mp / L ** 3
    # inverse-CDF sampling of a power law on [1, 10^decades]
    a1 = slope + 1.0
    hi = 10.0 ** decades
    u = rng.random(n_halo)
    mrel = (1.0 + u * (hi ** a1 - 1.0)) ** (1.0 / a1)
    target = halo_frac * n
    counts = np.maximum(np.rint(mrel / mrel.sum() * target), min_particles).astype(np.int64)
    # trim the largest haloes until the total equals the target exactly
    excess = int(counts.sum() - round(target))
    order = np.argsort(-counts)
    k = 0
    while excess != 0:
        i = order[k % n_halo]
        step = 1 if excess > 0 else -1
        if counts[i] - step >= min_particles:
            counts[i] -= step
            excess -= step
        k += 1
    centres = rng.random((n_halo, 3)) * L
    parts = []
    for h in range(n_halo):
        m_h = counts[h] * mp
        r200 = (3.0 * m_h / (4.0 * math.pi * 200.0 * rho_bar)) ** (1.0 / 3.0)
        parts.append(nfw_halo_positions(rng, int(counts[h]), centres[h], r200, c))
    halo = np.concatenate(parts, axis=0)
    n_bg = n - halo.shape[0]
    bg = rng.random((n_bg, 3)) * L
    pos = np.concatenate([halo, bg], axis=0)
    perm = rng.permutation(n)
    pos = _wrap32(pos[perm], L)
    return _single(pos, np.full(n, mp, np.float32), params, name)


def batch_boxes(n_boxes: int, seed: int, n_min: int = 2048, n_max: int = 65536,
                p_nfw: float = 0.5, name: str = "batch") -> ParticleSet:
    """Many independent unit boxes of uneven size and structure."""
    rng = np.random.default_rng(seed)
    L = 1.0
    rs = 1.25 / 32
    params = BoxParams(L=L, G=1.0, eps=1e-3, rs=rs, rcut=4.5 * rs, leaf_max=32)
    ns = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_boxes))).astype(np.int64)
    kinds = rng.random(n_boxes) < p_nfw
    pos_list, mass_list = [], []
    for b in range(n_boxes):
        nb = int(ns[b])
        if kinds[b]:
            p = nfw_halo_positions(rng, nb, np.full(3, 0.5 * L), 0.2 * L, 10.0)
        else:
            p = rng.random((nb, 3)) * L
        pos_list.append(_wrap32(p, L))
        mass_list.append(np.full(nb, 1.0 / nb, np.float32))
    offsets = np.zeros(n_boxes + 1, np.int64)
    offsets[1:] = np.cumsum(ns)
    return ParticleSet(np.concatenate(pos_list), np.concatenate(mass_list),
                       [params] * n_boxes, offsets, name)


def _params_mesh(L, n_mesh, leaf_max=32, eps_div=30.0):
    rs = 1.25 * L / n_mesh
    return BoxParams(L=L, G=1.0, eps=L / n_mesh / eps_div, rs=rs, rcut=4.5 * rs, leaf_max=leaf_max)


WORKLOADS = ("uniform_small", "zeldovich_128", "nfw_mix_256", "batch_512")


def workload(name: str, scale: int | None = None) -> ParticleSet:
    """Build a named workload (seed = 1000 + its index in the list).

    ``scale`` shrinks the side count of the lattice workloads (e.g. 32 gives
    a 32^3 version with the same spacing-relative parameters) for tests.
    """
    if name == "uniform_small":
        rs = 1.25 / 32
        p = BoxParams(L=1.0, G=1.0, eps=1e-3, rs=rs, rcut=4.5 * rs, leaf_max=32)
        return uniform_box(4096 if scale is None else scale, p, seed=1001, name=name)
    if name == "zeldovich_128":
        ns = 128 if scale is None else scale
        L = 100.0 * ns / 128
        return zeldovich_lattice(ns, _params_mesh(L, ns), seed=1002, name=name)
    if name == "nfw_mix_256":
        ns = 256 if scale is None else scale
        L = 200.0 * ns / 256
        n_halo = 10_000 if scale is None else max(8, int(10_000 * (ns / 256) ** 3))
        return nfw_mixture(ns, _params_mesh(L, ns), seed=1003, n_halo=n_halo, name=name)
    if name == "batch_512":
        nb = 512 if scale is None else scale
        return batch_boxes(nb, seed=1004, name=name)
    raise KeyError(name)
