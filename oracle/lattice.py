"""Lattice geometry for the oracle (test infrastructure, see ``oracle/__init__``).

Conventions (Sec. 6.2: X fastest, T slowest):
  * ``dims = (LX, LY, LZ, LT)``; direction mu = 0, 1, 2, 3 is x, y, z, t.
  * Natural arrays are indexed ``[t, z, y, x, ...]``.
  * Gauge field ``U[t, z, y, x, mu, a, b]`` is the SU(3) link from x to x + mu.
  * Parity of a site is (x + y + z + t) mod 2; even = 0 (Fig. 1: even-odd colouring).
  * Fermion hops that wrap around the t extent pick up a factor -1 per wrap when the
    time direction is antiperiodic. Gauge links are always periodic.
"""
import numpy as np


def all_coords(dims):
    """All site coordinates as an (V, 4) int array, ordered lexicographically with
    x fastest and t slowest (the natural-array order)."""
    LX, LY, LZ, LT = dims
    t, z, y, x = np.meshgrid(np.arange(LT), np.arange(LZ), np.arange(LY),
                             np.arange(LX), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


def parity_of(coords):
    return coords.sum(axis=1) % 2


def shift_coords(coords, dims, mu, n):
    """Coordinates of x + n*mu (wrapped) and the number of times the hop crossed the
    boundary of direction mu (signed: floor((x_mu + n) / L_mu))."""
    out = coords.copy()
    raw = coords[:, mu] + n
    out[:, mu] = np.mod(raw, dims[mu])
    wraps = np.floor_divide(raw, dims[mu])
    return out, wraps


def fermion_sign(wraps, mu, antiperiodic_t):
    """(-1)^(number of boundary crossings) for a hop in the antiperiodic t direction."""
    if mu == 3 and antiperiodic_t:
        return np.where(wraps % 2 == 0, 1.0, -1.0)
    return np.ones(wraps.shape)


def at(field, coords):
    """Gather ``field[t, z, y, x, ...]`` at an (N, 4) list of (x, y, z, t) coordinates."""
    return field[coords[:, 3], coords[:, 2], coords[:, 1], coords[:, 0]]


def site_index(coords, dims):
    """Lexicographic site index (x fastest)."""
    LX, LY, LZ, _ = dims
    return ((coords[:, 3] * LZ + coords[:, 2]) * LY + coords[:, 1]) * LX + coords[:, 0]


def dims_of(field):
    """(LX, LY, LZ, LT) of a natural-layout field."""
    return (field.shape[3], field.shape[2], field.shape[1], field.shape[0])
