"""Pins of the oracle's lattice geometry, boundary signs and clover inverse, and of the
direction of the learned preconditioner's transports (CPU only).

Boundary condition (the paper leaves it to the configuration; read as antiperiodic time
for fermion hops): a hop in t picks up (-1) for every time it crosses the t boundary, and a
3-hop on a short lattice may cross it twice. The values below are counted by hand from
that rule."""
import numpy as np

from oracle import lattice, ptc, wilson
from paper_1109_2935_gb300 import synth


def test_boundary_crossings_and_signs_by_hand():
    dims = (4, 4, 4, 3)
    xs = np.array([[0, 0, 0, t] for t in range(3)])
    # (t, hop) -> (target t, crossings) on T = 3
    expect = {(0, +1): (1, 0), (2, +1): (0, 1), (0, -1): (2, -1), (1, -1): (0, 0),
              (0, +3): (0, 1), (2, +3): (2, 1), (0, -3): (0, -1), (2, -3): (2, -1)}
    for (t, n), (tt, w) in expect.items():
        ys, wraps = lattice.shift_coords(xs[t:t + 1], dims, 3, n)
        assert ys[0, 3] == tt and wraps[0] == w
        s = lattice.fermion_sign(wraps, 3, True)[0]
        assert s == (-1.0 if w % 2 else 1.0)
        assert lattice.fermion_sign(wraps, 3, False)[0] == 1.0
        assert lattice.fermion_sign(wraps, 2, True)[0] == 1.0
    # T = 2: a 3-hop from t = 1 forward crosses twice (sign +1), from t = 0 once (sign -1)
    d2 = (4, 4, 4, 2)
    for t, n, w in ((0, 3, 1), (1, 3, 2), (0, -3, -2), (1, -3, -1)):
        _, wraps = lattice.shift_coords(np.array([[0, 0, 0, t]]), d2, 3, n)
        assert wraps[0] == w
        assert lattice.fermion_sign(wraps, 3, True)[0] == (-1.0 if w % 2 else 1.0)


def test_site_index_and_parity():
    dims = (4, 6, 2, 8)
    xs = lattice.all_coords(dims)
    idx = lattice.site_index(xs, dims)
    assert np.array_equal(np.sort(idx), np.arange(4 * 6 * 2 * 8))
    x = np.array([[3, 5, 1, 7]])
    assert lattice.site_index(x, dims)[0] == ((7 * 2 + 1) * 6 + 5) * 4 + 3
    assert lattice.parity_of(x)[0] == (3 + 5 + 1 + 7) % 2


def test_clover_hat_inverse_is_the_inverse():
    dims = (4, 4, 4, 4)
    U = synth.wilson_gauge(dims, 0.5, 1, 77).numpy()
    A = wilson.clover(U, 1.0)
    kappa = 0.13
    inv = wilson.clover_hat_inverse(A, kappa)
    Ahat = np.eye(12) + 2 * kappa * A
    assert np.max(np.abs(np.einsum("...ij,...jk->...ik", Ahat, inv) - np.eye(12))) < 1e-13
    # block-diagonal in chirality like Ahat itself
    assert np.max(np.abs(inv[..., :6, 6:])) < 1e-15 and np.max(np.abs(inv[..., 6:, :6])) < 1e-15
    assert wilson.clover_hat_inverse(None, kappa) is None


def test_transport_with_unit_links_is_a_shift():
    """With U = 1, T_{+mu} psi (x) = psi(x + mu) and T_{-mu} psi (x) = psi(x - mu), with the
    antiperiodic sign on the t hops that cross the boundary."""
    dims = (4, 6, 2, 8)
    psi = synth.wilson_spinor(dims, 5).numpy()
    U = np.broadcast_to(np.eye(3, dtype=complex), (8, 2, 6, 4, 4, 3, 3)).copy()
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    for mu in range(4):
        fwd = np.roll(psi, -1, axis=axis[mu])
        bwd = np.roll(psi, +1, axis=axis[mu])
        if mu == 3:
            fwd[-1] *= -1   # t = T-1 reads t = 0 across the boundary
            bwd[0] *= -1    # t = 0 reads t = T-1
        assert np.array_equal(ptc.transport(U, psi, 1 + 2 * mu), fwd)
        assert np.array_equal(ptc.transport(U, psi, 2 + 2 * mu), bwd)
        if mu == 3:
            assert np.array_equal(ptc.transport(U, psi, 1 + 2 * mu, antiperiodic_t=False),
                                  np.roll(psi, -1, axis=0))
    assert np.array_equal(ptc.transport(U, psi, 0), psi)
