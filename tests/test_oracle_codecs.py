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
