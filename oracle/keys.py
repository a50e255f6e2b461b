"""Space-filling-curve keys of the ground grid + local octree (oracle side).

Test infrastructure only.  Written from the paper's description:

* Sec. 3.2: every particle is labelled with the index of its ``ground`` cell,
  (i * N_side + j) * N_side + k, with N_side a power of two, and particles are
  bucket-sorted by that index; inside a ground cell they are re-ordered by
  Morton key, whose order is the order of the octree, so every octree node is
  one contiguous run of particles.
* Sec. 4.1: the Peano-Hilbert curve gives the same octree property with only
  face-adjacent steps; it is offered here as the alternative local key.

Key layout (64-bit, MSB first):  box index | ground index | local key.
Per box the position is wrapped into [0, L) and quantised to 2^T cells per
axis (T key bits per axis); the top g bits of each axis give the ground cell
(N_side = 2^g, the largest power of two whose cell side L/N_side is at least
rcut, capped at 2^7), the low b = T - g bits the local coordinate.
Bit k of the local x, y, z coordinates lands on key bits 3k+2, 3k+1, 3k.
"""
from __future__ import annotations

import math

import numpy as np

G_MAX = 7


def key_bits_per_axis(n_boxes: int) -> int:
    """T: per-axis key bits, leaving room for the box index in 63 bits."""
    box_bits = 0 if n_boxes <= 1 else int(math.ceil(math.log2(n_boxes)))
    return (63 - box_bits) // 3


def ground_level(L: float, rcut: float) -> int:
    """Largest g <= G_MAX with L / 2^g >= rcut (ground cell no smaller than rcut)."""
    g = 0
    while g < G_MAX and L / float(2 ** (g + 1)) >= rcut:
        g += 1
    return g


def wrap(x, L):
    """Wrap coordinates into [0, L): x - L floor(x/L), in float64; values
    already in [0, L) are kept as they are."""
    x = np.asarray(x, np.float64)
    inside = (x >= 0.0) & (x < L)
    return np.where(inside, x, x - L * np.floor(x / L))


def quantise(xw, L, T):
    """Integer cell of a wrapped coordinate on a 2^T grid, clamped to range."""
    S = math.ldexp(1.0, T) / L
    q = np.floor(np.asarray(xw, np.float64) * S)
    q = np.clip(q, 0, 2 ** T - 1)
    return q.astype(np.int64)


def interleave3(x, y, z, bits):
    """Interleave the low ``bits`` bits of x, y, z (x most significant)."""
    x = np.asarray(x, np.uint64)
    y = np.asarray(y, np.uint64)
    z = np.asarray(z, np.uint64)
    out = np.zeros(np.broadcast(x, y, z).shape, np.uint64)
    for k in range(bits):
        one = np.uint64(1)
        kk = np.uint64(k)
        out |= ((x >> kk) & one) << np.uint64(3 * k + 2)
        out |= ((y >> kk) & one) << np.uint64(3 * k + 1)
        out |= ((z >> kk) & one) << np.uint64(3 * k)
    return out


def morton3(x, y, z, bits):
    return interleave3(x, y, z, bits)


def hilbert3(x, y, z, bits):
    """3-D Hilbert index of integer cell coordinates (``bits`` bits per axis).

    Follows J. Skilling, "Programming the Hilbert curve" (AIP Conf. Proc. 707,
    2004): the coordinates are turned into the "transposed" Hilbert index by
    undoing the per-level reflections/exchanges and Gray-coding, then the three
    transposed words are bit-interleaved like a Morton key.
    """
    X = [np.array(x, np.int64, copy=True), np.array(y, np.int64, copy=True),
         np.array(z, np.int64, copy=True)]
    if bits == 0:
        return np.zeros(X[0].shape, np.uint64)
    M = 1 << (bits - 1)
    Q = M
    while Q > 1:
        P = Q - 1
        for i in range(3):
            has = (X[i] & Q) != 0
            # where set: invert low bits of X[0]; else swap low bits of X[0], X[i]
            t = (X[0] ^ X[i]) & P
            X0_inv = X[0] ^ P
            X0_swp = X[0] ^ t
            Xi_swp = X[i] ^ t
            if i == 0:
                X[0] = np.where(has, X0_inv, X[0])  # swap with itself is a no-op
            else:
                new0 = np.where(has, X0_inv, X0_swp)
                X[i] = np.where(has, X[i], Xi_swp)
                X[0] = new0
        Q >>= 1
    for i in range(1, 3):
        X[i] = X[i] ^ X[i - 1]
    t = np.zeros_like(X[0])
    Q = M
    while Q > 1:
        t = np.where((X[2] & Q) != 0, t ^ (Q - 1), t)
        Q >>= 1
    for i in range(3):
        X[i] = X[i] ^ t
    return interleave3(X[0], X[1], X[2], bits)


def particle_keys(pos, L, rcut, T, key_kind=0, box_index=0):
    """Keys of one box's particles.  Returns (keys uint64, g, b)."""
    g = ground_level(L, rcut)
    b = T - g
    xw = wrap(pos, L)
    q = quantise(xw, L, T)
    gc = q >> b
    lc = q & ((1 << b) - 1)
    nside = 1 << g
    ground = (gc[:, 0] * nside + gc[:, 1]) * nside + gc[:, 2]
    if key_kind == 0:
        local = morton3(lc[:, 0], lc[:, 1], lc[:, 2], b)
    else:
        local = hilbert3(lc[:, 0], lc[:, 1], lc[:, 2], b)
    key = (np.uint64(box_index) << np.uint64(3 * T)) | (ground.astype(np.uint64) << np.uint64(3 * b)) | local
    return key, g, b
