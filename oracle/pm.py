"""Long-range (particle-mesh) side of the force split, oracle side.

Test infrastructure only (see the package docstring).  Plain numpy in
float64, written from the PM description of Sec. 3.1 and taken in the
paper's order:

1. Assign the particle masses to a periodic N^3 mesh with the Cloud-in-Cell
   (CIC) scheme (Sec. 3.1: the conventional CIC assignment).
2. FFT the density.
3. Multiply by the Green's function of the 3-point difference Laplacian,
   g_k(l, m, n) = pi G Delta_g^2 / (sin^2(pi l/N) + sin^2(pi m/N) +
   sin^2(pi n/N))  (the equation of Sec. 3.1, with the sign of an attractive
   potential), and by the long-range filter exp(-k^2 R_s^2) that takes the
   short-range part out (Sec. 3.1; its real-space counterpart is the
   complement 1 - f(s) of Eq. (split)).
4. Inverse FFT: the potential on the mesh.
5. The acceleration of each particle interpolated from the potential mesh.

Readings taken here (the paper is silent or garbled on each):

* Sign and normalisation.  The printed g_k has no sign and a missing
  constant in the continuum form ("-/k^2").  phi_k = -pi G Delta_g^2 rho_k /
  S(l, m, n) with S = sum of the three sin^2 terms solves the discrete
  Poisson equation (7-point Laplacian) nabla^2 phi = 4 pi G (rho - rho_bar);
  rho is mass per cell volume Delta_g^3; the k = 0 mode is dropped (the
  periodic box has a neutralising mean density).
* Filter.  k^2 = (2 pi / L)^2 (l'^2 + m'^2 + n'^2) with l' the signed
  frequency in (-N/2, N/2]: the continuum wavenumber of the mode.
* Mesh.  Nodes at x = i Delta_g, Delta_g = L / N, i = 0..N-1, periodic.
* Gradient.  Sec. 3.1 only says that the accelerations are interpolated
  linearly from the potential mesh.  Here the mesh acceleration is the
  2-point central difference
  -(phi[i+1] - phi[i-1]) / (2 Delta_g), then CIC-interpolated to the
  particle with the assignment weights (so momentum is conserved).
* No deconvolution of the CIC window (the paper mentions none).
* The cell index of a particle is an integer decided by floating point: it
  is taken in FP64 with fixed operations (a coordinate in [0, L) is used
  as it is, any other becomes x - L floor(x / L); then u = x_w * (N / L),
  i0 = floor(u)), the same ones the CUDA path uses.
"""
from __future__ import annotations

import numpy as np


def cic_cells(pos, L, n_mesh):
    """Lower CIC node (int64 [P,3]) and fractional offset (float64 [P,3]).

    A coordinate already in [0, L) is kept; any other is wrapped as
    x - L floor(x / L) (a result equal to L maps to 0).  Then u = x * (N / L)
    in mesh units; node i0 = floor(u) mod N, fraction u - floor(u)."""
    x = np.asarray(pos, np.float64)
    inside = (x >= 0.0) & (x < L)
    xw = np.where(inside, x, x - L * np.floor(x / L))
    xw = np.where(xw >= L, 0.0, xw)
    u = xw * (n_mesh / L)
    fl = np.floor(u)
    f = u - fl
    i0 = fl.astype(np.int64) % n_mesh
    return i0, f


def cic_weights(f):
    """The 8 trilinear CIC weights per particle (w[:, a, b, c] for node
    offsets a, b, c in {0, 1} along x, y, z)."""
    w0 = 1.0 - f
    wx = np.stack([w0[:, 0], f[:, 0]], axis=1)
    wy = np.stack([w0[:, 1], f[:, 1]], axis=1)
    wz = np.stack([w0[:, 2], f[:, 2]], axis=1)
    return wx[:, :, None, None] * wy[:, None, :, None] * wz[:, None, None, :]


def cic_assign(pos, mass, L, n_mesh):
    """Mass on each mesh node [N,N,N] (indexed [ix, iy, iz]): every particle
    shares its mass between the 8 nodes of its cell with the CIC weights."""
    i0, f = cic_cells(pos, L, n_mesh)
    m = np.asarray(mass, np.float64)
    w = cic_weights(f) * m[:, None, None, None]
    grid = np.zeros((n_mesh,) * 3)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                ix = (i0[:, 0] + a) % n_mesh
                iy = (i0[:, 1] + b) % n_mesh
                iz = (i0[:, 2] + c) % n_mesh
                np.add.at(grid, (ix, iy, iz), w[:, a, b, c])
    return grid


def cic_interp(field, pos, L):
    """Value of a mesh field (shape [N,N,N] or [N,N,N,C]) at each particle,
    interpolated with the CIC weights."""
    n_mesh = field.shape[0]
    i0, f = cic_cells(pos, L, n_mesh)
    w = cic_weights(f)
    out = np.zeros((len(i0),) + field.shape[3:])
    for a in range(2):
        for b in range(2):
            for c in range(2):
                v = field[(i0[:, 0] + a) % n_mesh, (i0[:, 1] + b) % n_mesh, (i0[:, 2] + c) % n_mesh]
                wv = w[:, a, b, c]
                out += v * (wv if v.ndim == 1 else wv[:, None])
    return out


def signed_freq(n_mesh):
    """Signed frequencies l' in (-N/2, N/2] of the FFT bins 0..N-1."""
    l = np.arange(n_mesh)
    return np.where(l > n_mesh // 2, l - n_mesh, l)


def green_filtered(n_mesh, L, G, rs):
    """The multiplier of the density's FFT that gives the long-range
    potential: -pi G Delta_g^2 / S(l, m, n) * exp(-k^2 R_s^2), 0 at k = 0."""
    dg = L / n_mesh
    s2 = np.sin(np.pi * np.arange(n_mesh) / n_mesh) ** 2
    S = s2[:, None, None] + s2[None, :, None] + s2[None, None, :]
    kf = 2.0 * np.pi / L * signed_freq(n_mesh).astype(np.float64)
    k2 = kf[:, None, None] ** 2 + kf[None, :, None] ** 2 + kf[None, None, :] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        g = -np.pi * G * dg * dg / S * np.exp(-k2 * rs * rs)
    g[0, 0, 0] = 0.0
    return g


def potential(mass_grid, L, G, rs):
    """Long-range potential on the mesh from the node masses (steps 2-4)."""
    n_mesh = mass_grid.shape[0]
    dg = L / n_mesh
    rho = mass_grid / dg ** 3
    rho_k = np.fft.fftn(rho)
    return np.real(np.fft.ifftn(rho_k * green_filtered(n_mesh, L, G, rs)))


def mesh_accel(phi, L):
    """-grad phi on the mesh by the 2-point central difference, [N,N,N,3]."""
    n_mesh = phi.shape[0]
    dg = L / n_mesh
    acc = np.empty(phi.shape + (3,))
    for ax in range(3):
        acc[..., ax] = -(np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)) / (2.0 * dg)
    return acc


class PMResult:
    def __init__(self, acc, pot, mass_grid, phi):
        self.acc = acc            # [P,3] long-range acceleration
        self.pot = pot            # [P] long-range potential at the particle
        self.mass_grid = mass_grid
        self.phi = phi


def accel(pos, mass, L, G, rs, n_mesh, targets=None) -> PMResult:
    """Long-range acceleration and potential of every particle (or of the
    rows ``targets``) from all particles, through steps 1-5."""
    pos = np.asarray(pos, np.float64)
    grid = cic_assign(pos, mass, L, n_mesh)
    phi = potential(grid, L, G, rs)
    acc_mesh = mesh_accel(phi, L)
    q = pos if targets is None else pos[np.asarray(targets, np.int64)]
    return PMResult(cic_interp(acc_mesh, q, L), cic_interp(phi, q, L), grid, phi)
