"""Pins of the oracle's spin basis: Clifford algebra, hermiticity, diagonal gamma5."""
import numpy as np

from oracle.gamma import GAMMA, GAMMA5, P_MINUS, P_PLUS, sigma, PLANES


def test_clifford_algebra():
    for m in range(4):
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2.0 * np.eye(4) * (m == n), atol=0)


def test_hermitian_and_gamma5_diagonal():
    for g in GAMMA:
        assert np.array_equal(g, g.conj().T)
    assert np.array_equal(GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))


def test_projectors_unnormalised():
    # P^{-/+mu} = 1 -/+ gamma_mu: (P/2) is an idempotent rank-2 projector.
    for pm, pp in zip(P_MINUS, P_PLUS):
        assert np.allclose((pm / 2) @ (pm / 2), pm / 2)
        assert np.linalg.matrix_rank(pm) == 2
        assert np.allclose(pm + pp, 2 * np.eye(4))


def test_sigma_commutes_with_gamma5_and_is_hermitian():
    for mu, nu in PLANES:
        s = sigma(mu, nu)
        assert np.allclose(s, s.conj().T)
        assert np.allclose(s @ GAMMA5, GAMMA5 @ s)
