"""Improved staggered (asqtad) operator for the oracle (test infrastructure; Eq. 3, Sec. 2.3).

Eq. 3 prints every hop with a "+" sign and no staggered phases, yet the text states
that the staggered matrix is anti-Hermitian (Sec. 3.1). The reading adopted is the
standard anti-Hermitian form with the phases eta_mu(x) = (-1)^(sum_{nu<mu} x_nu)
applied to stored (phase-free) links:
    D psi(x) = sum_mu eta_mu(x) [ Uf_mu(x) psi(x+mu)  - Uf_mu(x-mu)^dagger  psi(x-mu)
                                 + Ul_mu(x) psi(x+3mu) - Ul_mu(x-3mu)^dagger psi(x-3mu) ],
    M = m - D/2,      M^dagger = m + D/2,
with Uf the fat links and Ul the long links. A hop that wraps the antiperiodic t
extent is multiplied by -1 per crossing. On lattices with L <= 6 a 3-hop can land on
the same site as a 1-hop; such contributions simply add.
"""
import numpy as np

from .lattice import all_coords, at, dims_of, fermion_sign, shift_coords


def eta(coords, mu):
    """Staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})."""
    if mu == 0:
        return np.ones(len(coords))
    return np.where(coords[:, :mu].sum(axis=1) % 2 == 0, 1.0, -1.0)


def dslash(fat, long, psi, antiperiodic_t=True, sites=None):
    """Asqtad hopping term D at (N, 4) output sites (whole lattice if None).
    ``fat``/``long``: natural (T,Z,Y,X,4,3,3); ``psi``: natural (T,Z,Y,X,3)."""
    dims = dims_of(psi)
    xs = all_coords(dims) if sites is None else np.asarray(sites)
    out = np.zeros((len(xs), 3), dtype=np.complex128)
    for mu in range(4):
        e = eta(xs, mu)
        for links, n in ((fat, 1), (long, 3)):
            yf, wf = shift_coords(xs, dims, mu, +n)
            yb, wb = shift_coords(xs, dims, mu, -n)
            sf = fermion_sign(wf, mu, antiperiodic_t)
            sb = fermion_sign(wb, mu, antiperiodic_t)
            fwd = np.einsum("nab,nb->na", at(links, xs)[:, mu], at(psi, yf))
            bwd = np.einsum("nba,nb->na", at(links, yb)[:, mu].conj(), at(psi, yb))
            out += e[:, None] * (sf[:, None] * fwd - sb[:, None] * bwd)
    if sites is None:
        LX, LY, LZ, LT = dims
        return out.reshape(LT, LZ, LY, LX, 3)
    return out


def apply_M(fat, long, mass, psi, antiperiodic_t=True, sites=None, dagger=False):
    """M = m - D/2 (Eq. 3), or M^dagger = m + D/2."""
    dims = dims_of(psi)
    xs = all_coords(dims) if sites is None else np.asarray(sites)
    d = dslash(fat, long, psi, antiperiodic_t, xs)
    out = mass * at(psi, xs) + (0.5 if dagger else -0.5) * d
    if sites is None:
        LX, LY, LZ, LT = dims
        return out.reshape(LT, LZ, LY, LX, 3)
    return out


def apply_normal(fat, long, mass, psi, antiperiodic_t=True):
    """M^dagger M psi on the whole lattice, computed as two applications."""
    return apply_M(fat, long, mass, apply_M(fat, long, mass, psi, antiperiodic_t),
                   antiperiodic_t, dagger=True)


def parity_mask(dims, parity):
    """Natural-shaped boolean mask (T,Z,Y,X) of the sites with the given parity."""
    LX, LY, LZ, LT = dims
    t, z, y, x = np.meshgrid(np.arange(LT), np.arange(LZ), np.arange(LY),
                             np.arange(LX), indexing="ij")
    return (x + y + z + t) % 2 == parity
