"""Storage codecs for the oracle (test infrastructure; Sec. 5, strategies (a) and (c)).

Gauge compression (Sec. 5 (a)): an SU(3) matrix has 8 free parameters, so 18 stored
reals can be cut to 12 (two rows; the third is the complex conjugate of their cross
product) or to 8. The paper only cites the 8-parameter form; the reading here keeps
  a2, a3, b1 (three complex numbers) and the phases arg(a1), arg(c1),
for the matrix with rows a, b, c, and recovers the rest from unitarity and det = 1:
  |a1|^2 = 1 - |a2|^2 - |a3|^2,   |c1|^2 = 1 - |a1|^2 - |b1|^2,
  with N = |a2|^2 + |a3|^2 = 1 - |a1|^2:
  b2 = -(conj(a3) conj(c1) + a2 conj(a1) b1) / N
  b3 =  (conj(a2) conj(c1) - a3 conj(a1) b1) / N
  c2 =  (conj(a3) conj(b1) - a2 conj(a1) c1) / N
  c3 = -(conj(a2) conj(b1) + a3 conj(a1) c1) / N
which follow from conj(U_ij) = cofactor_ij (U^-1 = U^dagger and det U = 1) together
with the orthogonality of row a to rows b and c. Degenerate when N -> 0.

Half precision (Sec. 5 (c)): the paper's 16-bit fixed-point format is read as IEEE
binary16 values scaled by a per-site FP32 norm (max |real| over the site), with
round-to-nearest-even on encode.
"""
import numpy as np


def pack12(U):
    """First two rows of each 3x3 matrix (..., 2, 3)."""
    return U[..., :2, :].copy()


def unpack12(R):
    """Rebuild (..., 3, 3) from two rows: row 3 = conj(row1 x row2)."""
    a, b = R[..., 0, :], R[..., 1, :]
    c = np.conj(np.cross(a, b))
    return np.stack([a, b, c], axis=-2)


def pack8(U):
    """(..., 8) reals: Re/Im a2, a3, b1, then arg(a1), arg(c1)."""
    a2, a3, b1 = U[..., 0, 1], U[..., 0, 2], U[..., 1, 0]
    out = np.stack([a2.real, a2.imag, a3.real, a3.imag, b1.real, b1.imag,
                    np.angle(U[..., 0, 0]), np.angle(U[..., 2, 0])], axis=-1)
    return out


def unpack8(P):
    a2 = P[..., 0] + 1j * P[..., 1]
    a3 = P[..., 2] + 1j * P[..., 3]
    b1 = P[..., 4] + 1j * P[..., 5]
    N = np.abs(a2) ** 2 + np.abs(a3) ** 2
    a1 = np.sqrt(np.maximum(1.0 - N, 0.0)) * np.exp(1j * P[..., 6])
    c1 = np.sqrt(np.maximum(1.0 - np.abs(a1) ** 2 - np.abs(b1) ** 2, 0.0)) * np.exp(1j * P[..., 7])
    ca1, ca2, ca3, cb1, cc1 = np.conj(a1), np.conj(a2), np.conj(a3), np.conj(b1), np.conj(c1)
    b2 = -(ca3 * cc1 + a2 * ca1 * b1) / N
    b3 = (ca2 * cc1 - a3 * ca1 * b1) / N
    c2 = (ca3 * cb1 - a2 * ca1 * c1) / N
    c3 = -(ca2 * cb1 + a3 * ca1 * c1) / N
    rows = [np.stack([a1, a2, a3], -1), np.stack([b1, b2, b3], -1), np.stack([c1, c2, c3], -1)]
    return np.stack(rows, axis=-2)


def _to_reals(z):
    return np.stack([z.real, z.imag], axis=-1)


def _from_reals(r):
    return r[..., 0] + 1j * r[..., 1]


def half_roundtrip_site(field, site_axes):
    """Encode/decode a natural complex field with one FP32 norm per site.
    ``site_axes``: number of trailing (internal) complex axes per site."""
    r = _to_reals(field)
    axes = tuple(range(r.ndim - site_axes - 1, r.ndim))
    norm = np.max(np.abs(r), axis=axes, keepdims=True).astype(np.float32)
    safe = np.where(norm > 0, norm, np.float32(1.0))
    q = (r.astype(np.float32) / safe).astype(np.float16).astype(np.float32) * safe
    q = np.where(norm > 0, q, np.float32(0.0))
    return _from_reals(q.astype(np.float64))


def spinor_half(psi):
    """Wilson (..., 4, 3) or staggered (..., 3) spinor -> decoded FP16+norm values."""
    return half_roundtrip_site(psi, 2 if psi.shape[-2:] == (4, 3) else 1)


def spinor_single(psi):
    return psi.astype(np.complex64).astype(np.complex128)


def links_half(U):
    """Links stored directly as binary16 (entries of SU(3) lie in [-1, 1])."""
    return _from_reals(_to_reals(U).astype(np.float16).astype(np.float64))


def links_single(U):
    return U.astype(np.complex64).astype(np.complex128)


def clover_packed_reals(Ahat):
    """The 72 stored reals of a chirally block-diagonal 12x12 matrix: for each of the
    two 6x6 Hermitian blocks, its 6 real diagonal entries and the 15 complex entries
    below the diagonal. Shape (..., 72)."""
    parts = []
    for b in range(2):
        blk = Ahat[..., 6 * b:6 * b + 6, 6 * b:6 * b + 6]
        parts.append(np.real(np.diagonal(blk, axis1=-2, axis2=-1)))
        il = np.tril_indices(6, -1)
        low = blk[..., il[0], il[1]]
        parts.append(low.real)
        parts.append(low.imag)
    return np.concatenate(parts, axis=-1)


def clover_from_packed_reals(R):
    out = np.zeros(R.shape[:-1] + (12, 12), dtype=np.complex128)
    il = np.tril_indices(6, -1)
    o = 0
    for b in range(2):
        d = R[..., o:o + 6]; o += 6
        re = R[..., o:o + 15]; o += 15
        im = R[..., o:o + 15]; o += 15
        blk = np.zeros(R.shape[:-1] + (6, 6), dtype=np.complex128)
        idx = np.arange(6)
        blk[..., idx, idx] = d
        blk[..., il[0], il[1]] = re + 1j * im
        blk[..., il[1], il[0]] = re - 1j * im
        out[..., 6 * b:6 * b + 6, 6 * b:6 * b + 6] = blk
    return out


def clover_half(Ahat):
    """Block-diagonal Hermitian clover matrix stored as binary16 values scaled by one
    FP32 per-site norm (max |stored real|), decoded back to complex128."""
    R = clover_packed_reals(Ahat)
    norm = np.max(np.abs(R), axis=-1, keepdims=True).astype(np.float32)
    safe = np.where(norm > 0, norm, np.float32(1.0))
    q = (R.astype(np.float32) / safe).astype(np.float16).astype(np.float32) * safe
    return clover_from_packed_reals(q.astype(np.float64))


def clover_single(Ahat):
    R = clover_packed_reals(Ahat).astype(np.float32).astype(np.float64)
    return clover_from_packed_reals(R)
