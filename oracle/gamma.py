"""Euclidean Dirac matrices for the oracle (test infrastructure).

The paper leaves the spin basis open ("similarity transforms to increase the sparsity
of the Dirac matrices", Sec. 5). The reading adopted here is a chiral basis in which
gamma5 = gamma1 gamma2 gamma3 gamma4 is diagonal, diag(1, 1, -1, -1), so that the
clover term, which commutes with gamma5, is block diagonal with two Hermitian 6x6
blocks (the 72-real structure of the footnote to Eq. 2).

Each gamma_mu has the off-diagonal form [[0, B_mu], [B_mu^dagger, 0]] with a 2x2
unitary B_mu. ``tests/test_oracle_gamma.py`` checks the Clifford algebra, hermiticity
and the diagonal gamma5.
"""
import numpy as np

_i = 1j
_B = [
    np.array([[0, _i], [_i, 0]], dtype=np.complex128),   # x
    np.array([[0, -1], [1, 0]], dtype=np.complex128),    # y
    np.array([[_i, 0], [0, -_i]], dtype=np.complex128),  # z
    np.array([[1, 0], [0, 1]], dtype=np.complex128),     # t
]
_Z = np.zeros((2, 2), dtype=np.complex128)

GAMMA = [np.block([[_Z, b], [b.conj().T, _Z]]) for b in _B]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)

# Eq. 2 projectors P^{-mu} = 1 - gamma_mu (forward hop) and P^{+mu} = 1 + gamma_mu
# (backward hop). They are unnormalised: for unit links the diagonal 4 of Eq. 2
# equals 1/2 * sum_mu (1 + 1), which fixes P = 1 -/+ gamma, not (1 -/+ gamma)/2.
P_MINUS = [ID4 - g for g in GAMMA]
P_PLUS = [ID4 + g for g in GAMMA]


def sigma(mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] (Hermitian)."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
