"""Wilson-clover operator for the oracle (test infrastructure; Eq. 2, Sec. 2.2).

Eq. 2 in the paper's units reads
    M = -1/2 D + (4 + m + A_x),
    D psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                        + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ].
The kappa form used throughout (kappa = 1 / (2 (4 + m))) multiplies by 2 kappa:
    M_kappa = 2 kappa M = 1 + 2 kappa A - kappa D.
Solves are of M_kappa x = b; the paper-units solution is 2 kappa x.

The clover term is not spelled out in the paper beyond its structure (footnote to
Eq. 2: Hermitian diagonal blocks, 72 reals). Reading adopted:
    A(x)   = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
    F      = (Q - Q^dagger)/8 with its colour trace removed,
    Q_{mu nu}(x) = the four plaquette leaves around x, all in the mu->nu orientation.
"""
import numpy as np

from .gamma import P_MINUS, P_PLUS, PLANES, sigma, GAMMA5
from .lattice import all_coords, at, dims_of, fermion_sign, shift_coords


def _sites(dims, sites):
    return all_coords(dims) if sites is None else np.asarray(sites)


def _reshape_out(out, dims, sites):
    if sites is None:
        LX, LY, LZ, LT = dims
        return out.reshape((LT, LZ, LY, LX) + out.shape[1:])
    return out


def block_id(coords, block):
    """Index of the Schwarz block containing each site (blocks tile the lattice)."""
    b = [coords[:, mu] // block[mu] for mu in range(4)]
    return ((b[3] * 4096 + b[2]) * 4096 + b[1]) * 4096 + b[0]


def dslash(U, psi, antiperiodic_t=True, sites=None, dagger=False, block=None):
    """Hopping term D of Eq. 2 (or its adjoint, which swaps the two projectors) at the
    given (N, 4) output sites, or on the whole lattice when ``sites`` is None.

    With ``block = (bx, by, bz, bt)`` the hops whose (wrapped) target lies in another
    Schwarz block are dropped: the Dirichlet (zero) block boundary of Sec. 3.2 and
    Sec. 8.1 ("switch off the communications")."""
    dims = dims_of(psi)
    xs = _sites(dims, sites)
    out = np.zeros((len(xs), 4, 3), dtype=np.complex128)
    bx = None if block is None else block_id(xs, block)
    for mu in range(4):
        pf, pb = (P_PLUS[mu], P_MINUS[mu]) if dagger else (P_MINUS[mu], P_PLUS[mu])
        # forward: (1 -/+ gamma_mu) U_mu(x) psi(x + mu)
        yf, wf = shift_coords(xs, dims, mu, +1)
        sf = fermion_sign(wf, mu, antiperiodic_t)
        if bx is not None:
            sf = sf * (block_id(yf, block) == bx)
        Uf = at(U, xs)[:, mu]
        out += sf[:, None, None] * np.einsum("st,nab,ntb->nsa", pf, Uf, at(psi, yf))
        # backward: (1 +/- gamma_mu) U_mu(x - mu)^dagger psi(x - mu)
        yb, wb = shift_coords(xs, dims, mu, -1)
        sb = fermion_sign(wb, mu, antiperiodic_t)
        if bx is not None:
            sb = sb * (block_id(yb, block) == bx)
        Ub = at(U, yb)[:, mu]
        out += sb[:, None, None] * np.einsum("st,nba,ntb->nsa", pb, Ub.conj(), at(psi, yb))
    return _reshape_out(out, dims, sites)


def _shift(xs, dims, nu, n):
    return shift_coords(xs, dims, nu, n)[0]


def _dag(M):
    return np.swapaxes(M.conj(), -1, -2)


def plaquette_leaves(U, mu, nu, sites=None):
    """Sum Q_{mu nu}(x) of the four plaquette leaves with a corner at x, each traversed
    mu -> nu -> -mu -> -nu starting and ending at x (gauge links periodic)."""
    dims = dims_of(U)
    xs = _sites(dims, sites)
    s = lambda ys, d, n: _shift(ys, dims, d, n)
    Umu = lambda ys: at(U, ys)[:, mu]
    Unu = lambda ys: at(U, ys)[:, nu]
    xpm, xpn = s(xs, mu, 1), s(xs, nu, 1)
    xmm, xmn = s(xs, mu, -1), s(xs, nu, -1)
    xmm_pn = s(xmm, nu, 1)
    xmm_mn = s(xmm, nu, -1)
    xpm_mn = s(xpm, nu, -1)
    # leaf in the (+mu, +nu) quadrant
    q = Umu(xs) @ Unu(xpm) @ _dag(Umu(xpn)) @ _dag(Unu(xs))
    # (-mu, +nu)
    q = q + Unu(xs) @ _dag(Umu(xmm_pn)) @ _dag(Unu(xmm)) @ Umu(xmm)
    # (-mu, -nu)
    q = q + _dag(Umu(xmm)) @ _dag(Unu(xmm_mn)) @ Umu(xmm_mn) @ Unu(xmn)
    # (+mu, -nu)
    q = q + _dag(Unu(xmn)) @ Umu(xmn) @ Unu(xpm_mn) @ _dag(Umu(xs))
    return q


def field_strength(U, sites=None):
    """F_{mu nu}(x) = (Q - Q^dagger)/8 minus (1/3) tr, for the six planes mu < nu in
    the order of ``gamma.PLANES``. Shape (N, 6, 3, 3)."""
    dims = dims_of(U)
    xs = _sites(dims, sites)
    F = np.zeros((len(xs), 6, 3, 3), dtype=np.complex128)
    for p, (mu, nu) in enumerate(PLANES):
        q = plaquette_leaves(U, mu, nu, xs)
        f = (q - _dag(q)) / 8.0
        tr = np.trace(f, axis1=1, axis2=2) / 3.0
        F[:, p] = f - tr[:, None, None] * np.eye(3)
    return F


def clover(U, csw, sites=None):
    """Clover matrix A(x) = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x) as a
    12x12 matrix over (spin, colour) with index 3*spin + colour. Shape (N, 12, 12),
    or natural (T, Z, Y, X, 12, 12) when ``sites`` is None."""
    dims = dims_of(U)
    xs = _sites(dims, sites)
    F = field_strength(U, xs)
    A = np.zeros((len(xs), 12, 12), dtype=np.complex128)
    for p, (mu, nu) in enumerate(PLANES):
        A += np.einsum("st,nab->nsatb", sigma(mu, nu), F[:, p]).reshape(len(xs), 12, 12)
    A *= 0.5j * csw
    return _reshape_out(A, dims, sites)


def apply_clover(A, psi, sites=None):
    """A(x) psi(x). ``A`` is natural (T,Z,Y,X,12,12); ``psi`` natural (T,Z,Y,X,4,3)."""
    dims = dims_of(psi)
    xs = _sites(dims, sites)
    a = at(A, xs)
    v = at(psi, xs).reshape(len(xs), 12)
    out = np.einsum("nij,nj->ni", a, v).reshape(len(xs), 4, 3)
    return _reshape_out(out, dims, sites)


def apply_M(U, A, kappa, psi, antiperiodic_t=True, sites=None, dagger=False, block=None):
    """Kappa-form Wilson-clover operator M_kappa = 1 + 2 kappa A - kappa D (Eq. 2),
    or its adjoint M_kappa^dagger = 1 + 2 kappa A^dagger - kappa D^dagger.
    ``A`` may be None (no clover term). ``block`` restricts D to Schwarz blocks."""
    dims = dims_of(psi)
    xs = _sites(dims, sites)
    out = at(psi, xs).copy()
    if A is not None:
        a = at(A, xs)
        if dagger:
            a = _dag(a)
        out += 2.0 * kappa * np.einsum("nij,nj->ni", a,
                                       at(psi, xs).reshape(len(xs), 12)).reshape(len(xs), 4, 3)
    out -= kappa * dslash(U, psi, antiperiodic_t, xs, dagger=dagger, block=block)
    return _reshape_out(out, dims, sites)


def apply_gamma5(psi):
    return np.einsum("st,...tc->...sc", GAMMA5, psi)


def apply_M_sites(U, csw, kappa, psi, sites, antiperiodic_t=True, dagger=False, Ahat_codec=None):
    """M_kappa psi at the listed (N, 4) sites only, with the clover computed at those
    sites (for sampled checks on lattices too large for a whole-lattice clover array).
    ``Ahat_codec`` optionally maps Ahat = 1 + 2 kappa A to its stored-precision value."""
    xs = np.asarray(sites)
    A = clover(U, csw, xs) if csw else np.zeros((len(xs), 12, 12), dtype=np.complex128)
    Ahat = np.eye(12) + 2.0 * kappa * A
    if Ahat_codec is not None:
        Ahat = Ahat_codec(Ahat)
    if dagger:
        Ahat = _dag(Ahat)
    v = at(psi, xs).reshape(len(xs), 12)
    out = np.einsum("nij,nj->ni", Ahat, v).reshape(len(xs), 4, 3)
    return out - kappa * dslash(U, psi, antiperiodic_t, xs, dagger=dagger)


# ---------------------------------------------------------------------------
# Even-odd (Schur complement) form of the Wilson-clover operator (Sec. 3.1)
# ---------------------------------------------------------------------------

def clover_hat_inverse(A, kappa):
    """(1 + 2 kappa A)^-1 per site; A natural (T,Z,Y,X,12,12) or None (identity)."""
    if A is None:
        return None
    Ahat = np.eye(12) + 2.0 * kappa * A
    return np.linalg.inv(Ahat)


def _apply_site_matrix(Mx, psi):
    """psi(x) -> Mx(x) psi(x) for natural arrays (Mx None = identity)."""
    if Mx is None:
        return psi.copy()
    sh = psi.shape
    return np.einsum("...ij,...j->...i", Mx, psi.reshape(sh[:4] + (12,))).reshape(sh)


def _clover_hat(A, kappa, psi):
    return psi if A is None else psi + 2.0 * kappa * apply_clover(A, psi)


def parity_mask(dims, parity):
    LX, LY, LZ, LT = dims
    t, z, y, x = np.meshgrid(np.arange(LT), np.arange(LZ), np.arange(LY), np.arange(LX), indexing="ij")
    return ((x + y + z + t) % 2 == parity)[..., None, None]


def apply_schur(U, A, kappa, psi_e, antiperiodic_t=True, dagger=False):
    """Even-site Schur complement of M_kappa = [[Ahat_ee, -kappa D_eo], [-kappa D_oe, Ahat_oo]]:
        Mhat psi_e = Ahat_ee psi_e - kappa^2 D_eo Ahat_oo^-1 D_oe psi_e
    (adjoint: D replaced by D^dagger; Ahat is Hermitian). ``psi_e`` is a natural array
    whose odd sites are ignored; the result is zero on odd sites."""
    dims = dims_of(psi_e)
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    inv = clover_hat_inverse(A, kappa)
    t = dslash(U, psi_e * ev, antiperiodic_t, dagger=dagger) * od
    t = _apply_site_matrix(inv, t) * od
    u = dslash(U, t, antiperiodic_t, dagger=dagger) * ev
    return (_clover_hat(A, kappa, psi_e * ev) - kappa * kappa * u) * ev


def schur_source(U, A, kappa, b, antiperiodic_t=True):
    """bhat_e = b_e + kappa D_eo Ahat_oo^-1 b_o (zero on odd sites)."""
    dims = dims_of(b)
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    t = _apply_site_matrix(clover_hat_inverse(A, kappa), b * od) * od
    return (b + kappa * dslash(U, t, antiperiodic_t)) * ev


def schur_reconstruct(U, A, kappa, b, x_e, antiperiodic_t=True):
    """Full solution from the even one: x_o = Ahat_oo^-1 (b_o + kappa D_oe x_e)."""
    dims = dims_of(b)
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    u = (b + kappa * dslash(U, x_e * ev, antiperiodic_t)) * od
    return x_e * ev + _apply_site_matrix(clover_hat_inverse(A, kappa), u) * od
