"""Pins of the oracle's asqtad operator (Eq. 3, read as the anti-Hermitian staggered
form with eta phases) against closed forms and symmetries. CPU only."""
import numpy as np
import pytest
import torch

from oracle import staggered
from oracle.lattice import all_coords
from paper_1109_2935_gb300 import synth


def _const_links(dims, c):
    return synth.unit_gauge(dims).numpy() * c


def _plane_wave(dims, n, col, apbc):
    p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)])
    if apbc:
        p[3] = (2 * n[3] + 1) * np.pi / dims[3]
    c = all_coords(dims)
    ph = np.exp(1j * (c @ p))
    LX, LY, LZ, LT = dims
    return (ph[:, None] * col[None]).reshape(LT, LZ, LY, LX, 3), p, ph, c


@pytest.mark.parametrize("dims,n,apbc", [
    ((4, 4, 4, 4), (1, 0, 1, 0), True),     # L = 4: x+3mu = x-mu, 1-hop and 3-hop add
    ((6, 4, 8, 6), (1, 1, 3, 2), True),
    ((8, 6, 4, 4), (3, 1, 0, 1), False),
    ((2, 2, 2, 2), (1, 0, 1, 0), True),
])
def test_free_field_closed_forms(dims, n, apbc, rng):
    """Constant fat = c1, long = c3 links:
    D e^{ipx} v = sum_mu eta_mu(x) 2i (c1 sin p_mu + c3 sin 3p_mu) e^{ipx} v and
    M^dagger M e^{ipx} v = [m^2 + sum_mu (c1 sin p_mu + c3 sin 3 p_mu)^2] e^{ipx} v."""
    c1, c3, m = 0.7, -0.2, 0.05
    col = rng.normal(size=3) + 1j * rng.normal(size=3)
    psi, p, ph, c = _plane_wave(dims, n, col, apbc)
    fat, lng = _const_links(dims, c1), _const_links(dims, c3)
    D = staggered.dslash(fat, lng, psi, apbc).reshape(-1, 3)
    w = 2j * (c1 * np.sin(p) + c3 * np.sin(3 * p))
    fac = sum(staggered.eta(c, mu) * w[mu] for mu in range(4))
    assert np.max(np.abs(D - (fac * ph)[:, None] * col[None])) < 1e-13
    MdM = staggered.apply_normal(fat, lng, m, psi, apbc)
    lam = m * m + np.sum((c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2)
    assert np.max(np.abs(MdM - lam * psi)) < 1e-13


def _fields(dims):
    fat, lng = synth.asqtad_links(dims, 31, 32)
    return fat.numpy(), lng.numpy()


def test_anti_hermitian_and_adjoint():
    dims = (4, 6, 4, 8)
    fat, lng = _fields(dims)
    x = synth.staggered_spinor(dims, 1).numpy()
    y = synth.staggered_spinor(dims, 2).numpy()
    Dx = staggered.dslash(fat, lng, x)
    Dy = staggered.dslash(fat, lng, y)
    assert abs(np.vdot(y, Dx) + np.vdot(Dy, x)) < 1e-12 * abs(np.vdot(y, Dx))
    m = 0.01
    Mx = staggered.apply_M(fat, lng, m, x)
    Mdy = staggered.apply_M(fat, lng, m, y, dagger=True)
    assert abs(np.vdot(y, Mx) - np.vdot(Mdy, x)) < 1e-12 * abs(np.vdot(y, Mx))


def test_epsilon_hermiticity_and_parity():
    dims = (4, 4, 4, 6)
    fat, lng = _fields(dims)
    x = synth.staggered_spinor(dims, 3).numpy()
    eps = np.where(staggered.parity_mask(dims, 0), 1.0, -1.0)[..., None]
    # eps D eps = -D (D joins sites of opposite parity only)
    lhs = eps * staggered.dslash(fat, lng, eps * x)
    assert np.max(np.abs(lhs + staggered.dslash(fat, lng, x))) < 1e-13
    even = staggered.parity_mask(dims, 0)[..., None]
    out = staggered.dslash(fat, lng, x * even)
    assert np.max(np.abs(out * even)) == 0.0


def test_normal_operator_decouples_parities():
    dims = (4, 4, 4, 4)
    fat, lng = _fields(dims)
    m = 0.03
    even = staggered.parity_mask(dims, 0)[..., None]
    x = synth.staggered_spinor(dims, 4, parity=0).numpy()
    out = staggered.apply_normal(fat, lng, m, x)
    assert np.max(np.abs(out * (~even))) < 1e-14
    # (M^dagger M)_ee = m^2 - 1/4 D_eo D_oe
    D = lambda v: staggered.dslash(fat, lng, v)
    alt = m * m * x - 0.25 * D(D(x))
    assert np.max(np.abs((out - alt) * even)) < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 6, 8)
    fat, lng = synth.asqtad_links(dims, 5, 6)
    LX, LY, LZ, LT = dims
    G = synth.haar_su3((LT, LZ, LY, LX), synth._gen(77, "cpu"), "cpu")
    fat_t = synth.gauge_transform(fat, G, hop=1).numpy()
    lng_t = synth.gauge_transform(lng, G, hop=3).numpy()
    G = G.numpy()
    psi = synth.staggered_spinor(dims, 8).numpy()
    lhs = staggered.dslash(fat_t, lng_t, np.einsum("...ab,...b->...a", G, psi))
    rhs = np.einsum("...ab,...b->...a", G, staggered.dslash(fat.numpy(), lng.numpy(), psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-13
