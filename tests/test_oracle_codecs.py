"""Pins of the oracle's storage codecs (Sec. 5 (a), (c)). CPU only."""
import numpy as np

from oracle import codecs
from paper_1109_2935_gb300 import synth


def _haar(n, seed):
    return synth.haar_su3((n,), synth._gen(seed, "cpu"), "cpu").numpy()


def test_recon12_roundtrip():
    U = _haar(20000, 1)
    assert np.max(np.abs(codecs.unpack12(codecs.pack12(U)) - U)) < 1e-14


def test_recon8_roundtrip():
    """The 8-real form divides by N = |a2|^2 + |a3|^2 = 1 - |a1|^2 and recovers |a1|
    and |c1| as square roots of differences, so its rounding error grows like
    eps (1/N + 1/|a1| + 1/|c1|): exact to rounding, degenerate as N, |a1| or |c1| -> 0."""
    U = _haar(20000, 2)
    P = codecs.pack8(U)
    assert P.shape == (20000, 8)
    err = np.max(np.abs(codecs.unpack8(P) - U), axis=(1, 2))
    N = np.abs(U[:, 0, 1]) ** 2 + np.abs(U[:, 0, 2]) ** 2
    bound = 2.2e-16 * (1 / N + 1 / np.abs(U[:, 0, 0]) + 1 / np.abs(U[:, 2, 0])) + 1e-15
    assert np.all(err < 8 * bound)
    assert np.median(err) < 1e-15


def test_recon8_rows_unitary_and_det_one():
    U = codecs.unpack8(codecs.pack8(_haar(1000, 3)))
    eye = np.einsum("nij,nkj->nik", U, U.conj())
    assert np.max(np.abs(eye - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-13


def test_half_spinor_error_bound():
    psi = synth.wilson_spinor((4, 4, 4, 4), 9).numpy() * 37.0
    q = codecs.spinor_half(psi)
    r = np.stack([psi.real, psi.imag], -1)
    norm = np.max(np.abs(r), axis=(-3, -2, -1))
    err = np.max(np.abs(np.stack([(q - psi).real, (q - psi).imag], -1)), axis=(-3, -2, -1))
    # binary16 has an 11-bit significand: relative rounding error <= 2^-11 of the norm
    assert np.all(err <= 2.0 ** -11 * norm * (1 + 1e-6))
    assert np.all(err > 0)
    # the maximal component is represented exactly (it encodes as +/-1)
    z = np.zeros_like(psi)
    assert np.array_equal(codecs.spinor_half(z), z)


def test_clover_packing_is_lossless():
    rng = np.random.default_rng(0)
    A = np.zeros((5, 12, 12), dtype=complex)
    for b in range(2):
        h = rng.normal(size=(5, 6, 6)) + 1j * rng.normal(size=(5, 6, 6))
        A[:, 6 * b:6 * b + 6, 6 * b:6 * b + 6] = h + np.swapaxes(h.conj(), -1, -2)
    R = codecs.clover_packed_reals(A)
    assert R.shape == (5, 72)
    assert np.array_equal(codecs.clover_from_packed_reals(R), A)
    q = codecs.clover_half(A)
    assert np.max(np.abs(q - A)) <= 2.0 ** -11 * np.max(np.abs(R)) * 1.01


def test_single_precision_rounding():
    """FP32 storage (reading of the single-precision fields): round to nearest, so each
    real component moves by at most half an FP32 unit (2^-24 relative for normal
    values); the rounding is idempotent and leaves short dyadic values unchanged."""
    rng = np.random.default_rng(5)
    z = (rng.normal(size=(4000, 4, 3)) + 1j * rng.normal(size=(4000, 4, 3))) * 10.0 ** rng.integers(-3, 4, (4000, 1, 1))
    for f in (codecs.spinor_single, codecs.links_single):
        q = f(z)
        for part in (np.real, np.imag):
            assert np.all(np.abs(part(q) - part(z)) <= 2.0 ** -24 * np.abs(part(z)))
        assert np.array_equal(f(q), q)
    d = (rng.integers(-4096, 4096, size=(100, 3, 3)) + 1j * rng.integers(-4096, 4096, size=(100, 3, 3))) / 1024.0
    assert np.array_equal(codecs.links_single(d), d)


def test_half_links_round_to_nearest_even():
    """FP16 links are binary16 entries (reading of the 16-bit format): an error of at most
    2^-11 relative in the normal range, ties to the even significand, idempotent."""
    U = _haar(5000, 6)
    q = codecs.links_half(U)
    for part in (np.real, np.imag):
        a, b = part(U), part(q)
        normal = np.abs(a) >= 2.0 ** -14
        assert np.all(np.abs(b - a)[normal] <= 2.0 ** -11 * np.abs(a)[normal])
        assert np.all(np.abs(b - a)[~normal] <= 2.0 ** -25)
    assert np.array_equal(codecs.links_half(q), q)
    # 1 + 2^-11 lies halfway between 1 and 1 + 2^-10: the even neighbour is 1;
    # 1 + 3 * 2^-11 lies halfway between 1 + 2^-10 and 1 + 2^-9: the even one is 1 + 2^-9
    t = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 2.0 ** -11)], dtype=complex)
    assert np.array_equal(codecs.links_half(t).real, [1.0, 1 + 2.0 ** -9, -1.0])


def test_half_site_norm_scaling():
    """The per-site norm is the largest |real| of the site: that component decodes exactly,
    a site scaled by a power of two decodes to the scaled values, and a zero site stays
    zero while its neighbours are encoded on their own scale."""
    psi = synth.wilson_spinor((2, 2, 2, 2), 11).numpy()
    q = codecs.spinor_half(psi)
    r, rq = np.stack([psi.real, psi.imag], -1), np.stack([q.real, q.imag], -1)
    flat, flatq = r.reshape(16, 24), rq.reshape(16, 24)
    k = np.argmax(np.abs(flat), axis=1)
    assert np.array_equal(flat[np.arange(16), k].astype(np.float32), flatq[np.arange(16), k])
    assert np.array_equal(codecs.spinor_half(psi * 2.0 ** 7), q * 2.0 ** 7)
    psi2 = psi.copy()
    psi2[0, 0, 0, 0] = 0
    q2 = codecs.spinor_half(psi2)
    assert np.all(q2[0, 0, 0, 0] == 0)
    assert np.array_equal(q2[1], q[1])


def test_clover_storage_bounds():
    """FP16 clover: binary16 of the 72 stored reals over one FP32 per-site scale, so every
    entry is within 2^-11 of that scale; FP32 clover within 2^-24 relative per real."""
    rng = np.random.default_rng(8)
    A = np.zeros((50, 12, 12), dtype=complex)
    for b in range(2):
        h = rng.normal(size=(50, 6, 6)) + 1j * rng.normal(size=(50, 6, 6))
        A[:, 6 * b:6 * b + 6, 6 * b:6 * b + 6] = (h + np.swapaxes(h.conj(), -1, -2)) * 10.0 ** rng.integers(-2, 3, (50, 1, 1))
    R = codecs.clover_packed_reals(A)
    scale = np.max(np.abs(R), axis=-1)
    Rh = codecs.clover_packed_reals(codecs.clover_half(A))
    assert np.all(np.max(np.abs(Rh - R), axis=-1) <= 2.0 ** -11 * scale * (1 + 1e-6))
    Rs = codecs.clover_packed_reals(codecs.clover_single(A))
    assert np.all(np.abs(Rs - R) <= 2.0 ** -24 * np.abs(R))
    # the decoded matrices stay Hermitian and chirally block-diagonal
    for f in (codecs.clover_half, codecs.clover_single):
        D = f(A)
        assert np.array_equal(D, np.swapaxes(D.conj(), -1, -2))
        assert np.all(D[:, :6, 6:] == 0) and np.all(D[:, 6:, :6] == 0)
