"""Pins of the oracle's Wilson-clover operator (Eq. 2) against closed forms,
symmetries and hand expansions. CPU only."""
import numpy as np
import pytest
import torch

from oracle import wilson
from oracle.gamma import GAMMA, GAMMA5, PLANES, sigma
from oracle.lattice import all_coords
from paper_1109_2935_gb300 import synth


def _plane_wave(dims, n, s, antiperiodic_t):
    """psi(x) = exp(i p.x) s with p_mu = 2 pi n_mu / L_mu (x, y, z) and, for an
    antiperiodic t, p_t = (2 n_t + 1) pi / L_t."""
    p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)], dtype=float)
    if antiperiodic_t:
        p[3] = (2 * n[3] + 1) * np.pi / dims[3]
    c = all_coords(dims)
    ph = np.exp(1j * (c @ p))
    LX, LY, LZ, LT = dims
    return (ph[:, None, None] * s[None]).reshape(LT, LZ, LY, LX, 4, 3), p, ph


@pytest.mark.parametrize("dims,n,apbc", [
    ((4, 4, 4, 4), (1, 0, 2, 0), True),
    ((4, 6, 4, 8), (1, 2, 3, 1), True),
    ((4, 4, 6, 4), (0, 1, 1, 2), False),
    ((2, 2, 2, 2), (1, 0, 1, 0), True),   # L = 2: x+mu and x-mu coincide, hops add
])
@pytest.mark.parametrize("dagger", [False, True])
def test_free_field_plane_wave(dims, n, apbc, dagger, rng):
    """Unit links: M_kappa psi = e^{ipx} [1 - 2 kappa sum cos p + (+/-) 2 i kappa sum gamma sin p] s."""
    kappa = 0.11
    s = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi, p, ph = _plane_wave(dims, n, s, apbc)
    U = synth.unit_gauge(dims).numpy()
    out = wilson.apply_M(U, None, kappa, psi, apbc, dagger=dagger)
    sgn = -1.0 if dagger else 1.0
    K = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) \
        + sgn * 2j * kappa * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    expect = (ph[:, None, None] * (K @ s)[None]).reshape(psi.shape)
    assert np.max(np.abs(out - expect)) < 1e-13


def _random_fields(dims, seed=7, csw=1.0):
    U = synth.wilson_gauge(dims, 0.5, 1, seed).numpy()
    A = wilson.clover(U, csw)
    return U, A


def test_gamma5_hermiticity_and_adjoint(rng):
    dims = (4, 4, 4, 6)
    U, A = _random_fields(dims)
    kappa = 0.13
    x = synth.wilson_spinor(dims, 11).numpy()
    y = synth.wilson_spinor(dims, 12).numpy()
    Mx = wilson.apply_M(U, A, kappa, x)
    Mdy = wilson.apply_M(U, A, kappa, y, dagger=True)
    # (y, M x) = (M^dagger y, x)
    lhs, rhs = np.vdot(y, Mx), np.vdot(Mdy, x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # M^dagger = gamma5 M gamma5
    g5Mg5 = wilson.apply_gamma5(wilson.apply_M(U, A, kappa, wilson.apply_gamma5(y)))
    assert np.max(np.abs(g5Mg5 - Mdy)) < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 6, 4)
    U, A = _random_fields(dims)
    kappa = 0.125
    LX, LY, LZ, LT = dims
    G = synth.haar_su3((LT, LZ, LY, LX), synth._gen(99, "cpu"), "cpu")
    Ut = synth.gauge_transform(torch.from_numpy(U), G).numpy()
    G = G.numpy()
    At = wilson.clover(Ut, 1.0)
    psi = synth.wilson_spinor(dims, 5).numpy()
    Gpsi = np.einsum("...ab,...sb->...sa", G, psi)
    lhs = wilson.apply_M(Ut, At, kappa, Gpsi)
    rhs = np.einsum("...ab,...sb->...sa", G, wilson.apply_M(U, A, kappa, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    # clover transforms as G A G^dagger (G acting on colour)
    G12 = np.einsum("st,...ab->...satb", np.eye(4), G).reshape(G.shape[:4] + (12, 12))
    At2 = G12 @ A @ np.swapaxes(G12.conj(), -1, -2)
    assert np.max(np.abs(At - At2)) < 1e-13


def test_clover_structure():
    dims = (4, 4, 4, 4)
    U, A = _random_fields(dims)
    assert np.max(np.abs(A - np.swapaxes(A.conj(), -1, -2))) < 1e-15      # Hermitian
    G5 = np.kron(GAMMA5, np.eye(3))
    assert np.max(np.abs(A @ G5 - G5 @ A)) < 1e-15                        # [A, gamma5] = 0
    assert np.max(np.abs(np.trace(A, axis1=-2, axis2=-1))) < 1e-14        # traceless
    F = wilson.field_strength(U)
    assert np.max(np.abs(F + np.swapaxes(F.conj(), -1, -2))) < 1e-15      # anti-Hermitian
    assert np.max(np.abs(np.trace(F, axis1=-2, axis2=-1))) < 1e-15


def test_unit_links_have_no_clover():
    dims = (4, 4, 4, 4)
    A = wilson.clover(synth.unit_gauge(dims).numpy(), 1.3)
    assert np.max(np.abs(A)) == 0.0


@pytest.mark.parametrize("nflux", [1, 3])
def test_clover_constant_abelian_field(nflux):
    """Uniform abelian field in the x-y plane: every (x,y) plaquette equals exp(i b Lambda)
    with Lambda = diag(1, -1, 0), b = 2 pi n / (LX LY). Then F_xy = i sin(b) Lambda, all
    other F vanish, and A = -(c_sw/2) sin(b) sigma_xy (x) Lambda exactly."""
    dims = (4, 6, 4, 4)
    LX, LY, LZ, LT = dims
    b = 2 * np.pi * nflux / (LX * LY)
    lam = np.array([1.0, -1.0, 0.0])
    U = synth.unit_gauge(dims).numpy()
    for x in range(LX):
        U[:, :, :, x, 1] = np.diag(np.exp(1j * b * x * lam))
    for y in range(LY):
        U[:, :, y, LX - 1, 0] = np.diag(np.exp(-1j * b * LX * y * lam))
    csw = 1.7
    A = wilson.clover(U, csw)
    expect = -(csw / 2) * np.sin(b) * np.kron(sigma(0, 1), np.diag(lam))
    assert np.max(np.abs(A - expect)) < 1e-14
    F = wilson.field_strength(U)
    assert np.max(np.abs(F[:, 0] - 1j * np.sin(b) * np.diag(lam))) < 1e-15
    assert np.max(np.abs(F[:, 1:])) < 1e-15


def test_clover_single_excited_link():
    """Only U_x(0) = W differs from 1 on a 4^4 lattice. For nu = y, z, t the four
    leaves of Q_{x nu} at a site are W, W^dagger or 1: Q = 2 + W + W^dagger at 0 and
    x-hat (so F = 0 there), Q = 3 + W at nu-hat and x-hat + nu-hat, Q = 3 + W^dagger at
    -nu-hat and x-hat - nu-hat. Planes without x and all other sites have F = 0."""
    dims = (4, 4, 4, 4)
    U = synth.unit_gauge(dims).numpy()
    W = synth.haar_su3((), synth._gen(3, "cpu"), "cpu").numpy()
    U[0, 0, 0, 0, 0] = W
    T = (W - W.conj().T) / 8
    T = T - np.trace(T) / 3 * np.eye(3)
    F = wilson.field_strength(U)
    c = all_coords(dims)
    expect = np.zeros_like(F)
    for p, (mu, nu) in enumerate(PLANES):
        if mu != 0:
            continue
        for sign_site, val in ((+1, T), (-1, -T)):
            for base in (0, 1):
                site = np.zeros(4, int)
                site[0] = base
                site[nu] = sign_site % dims[nu]
                idx = np.where((c == site).all(axis=1))[0][0]
                expect[idx, p] = val
    assert np.max(np.abs(F - expect)) < 1e-15


def test_site_subset_matches_whole_lattice():
    dims = (4, 4, 4, 6)
    U, A = _random_fields(dims)
    psi = synth.wilson_spinor(dims, 3).numpy()
    full = wilson.apply_M(U, A, 0.12, psi).reshape(-1, 4, 3)
    sel = np.array([0, 5, 17, 200, 383])
    sub = wilson.apply_M(U, A, 0.12, psi, sites=all_coords(dims)[sel])
    assert np.array_equal(full[sel], sub)


def test_dslash_couples_opposite_parity_only():
    dims = (4, 4, 4, 4)
    U, _ = _random_fields(dims)
    psi = synth.wilson_spinor(dims, 3).numpy()
    c = all_coords(dims)
    par = (c.sum(1) % 2).reshape(4, 4, 4, 4)
    psi_even = psi * (par == 0)[..., None, None]
    out = wilson.dslash(U, psi_even)
    assert np.max(np.abs(out[par == 0])) == 0.0
    assert np.max(np.abs(out[par == 1])) > 0.1


def test_schur_complement_equals_dense_block_schur():
    """The even-site Schur operator equals M_ee - M_eo M_oo^-1 M_oe of the assembled
    dense matrix of M_kappa (index sets by parity), and the even-odd solve
    reconstructs the solution of the full system."""
    dims = (2, 2, 2, 4)
    U, A = _random_fields(dims, seed=9)
    kappa = 0.12
    M = lambda v: wilson.apply_M(U, A, kappa, v)
    shape = dims[::-1] + (4, 3)
    n = int(np.prod(shape))
    D = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        D[:, j] = M(e.reshape(shape)).ravel()
    par = np.repeat((all_coords(dims).sum(1) % 2), 12)
    E, O = np.where(par == 0)[0], np.where(par == 1)[0]
    S = D[np.ix_(E, E)] - D[np.ix_(E, O)] @ np.linalg.solve(D[np.ix_(O, O)], D[np.ix_(O, E)])
    psi = synth.wilson_spinor(dims, 4).numpy()
    got = wilson.apply_schur(U, A, kappa, psi).ravel()[E]
    assert np.max(np.abs(got - S @ psi.ravel()[E])) < 1e-13
    gotd = wilson.apply_schur(U, A, kappa, psi, dagger=True).ravel()[E]
    assert np.max(np.abs(gotd - S.conj().T @ psi.ravel()[E])) < 1e-13
    # solve through the Schur system
    b = synth.wilson_spinor(dims, 5).numpy()
    bhat = wilson.schur_source(U, A, kappa, b).ravel()[E]
    xe = np.linalg.solve(S, bhat)
    xfull = np.zeros(n, dtype=complex)
    xfull[E] = xe
    x = wilson.schur_reconstruct(U, A, kappa, b, xfull.reshape(shape))
    assert np.linalg.norm(M(x) - b) / np.linalg.norm(b) < 1e-13


def _sample_sites(dims, n, seed):
    """A site sample that always contains both t edges (where antiperiodic hops wrap),
    a repeated site and an unsorted order."""
    r = np.random.default_rng(seed)
    c = all_coords(dims)
    idx = r.choice(len(c), size=min(n, len(c)), replace=False)
    edge = np.where((c[:, 3] == 0) | (c[:, 3] == dims[3] - 1))[0][:3]
    idx = np.concatenate([idx, edge, idx[:1]])
    return idx, c[idx]


@pytest.mark.parametrize("dims,apbc", [((4, 4, 4, 6), True), ((2, 2, 2, 2), True),
                                       ((2, 4, 2, 4), False)])
def test_site_subset_clover_matches_whole_lattice(dims, apbc):
    """clover(U, csw, sites) is the whole-lattice clover field read at those sites."""
    U, A = _random_fields(dims, seed=21, csw=1.3)
    idx, xs = _sample_sites(dims, 40, 3)
    sub = wilson.clover(U, 1.3, xs)
    whole = A.reshape(-1, 12, 12)[idx]
    assert np.max(np.abs(sub - whole)) <= 1e-13 * np.max(np.abs(whole))


def _codec_half(Ahat):
    from oracle import codecs
    return codecs.clover_half(Ahat)


def _codec_single(Ahat):
    from oracle import codecs
    return codecs.clover_single(Ahat)


@pytest.mark.parametrize("dims,apbc", [((4, 4, 4, 6), True), ((2, 2, 2, 2), True),
                                       ((2, 4, 2, 4), False)])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("codec", [None, _codec_half, _codec_single])
def test_apply_M_sites_matches_whole_lattice(dims, apbc, dagger, codec):
    """apply_M_sites (the checker of every sampled full-size GPU result) equals the
    whole-lattice M_kappa of Eq. 2 at the sampled sites. With a storage codec the
    whole-lattice operator is given the clover A' = (codec(1 + 2 kappa A) - 1) / (2 kappa),
    so that its own 1 + 2 kappa A' is the stored Ahat."""
    kappa, csw = 0.127, 1.3
    U, A = _random_fields(dims, seed=22, csw=csw)
    psi = synth.wilson_spinor(dims, 23).numpy()
    idx, xs = _sample_sites(dims, 50, 4)
    got = wilson.apply_M_sites(U, csw, kappa, psi, xs, apbc, dagger, Ahat_codec=codec)
    if codec is None:
        Aw = A
    else:
        Aw = (codec(np.eye(12) + 2.0 * kappa * A) - np.eye(12)) / (2.0 * kappa)
    whole = wilson.apply_M(U, Aw, kappa, psi, apbc, dagger=dagger).reshape(-1, 4, 3)[idx]
    err = np.max(np.abs(got - whole)) / np.max(np.abs(whole))
    assert err <= 1e-13, err
    # a dropped clover or hopping term would be far outside this bound
    assert np.max(np.abs(whole - psi.reshape(-1, 4, 3)[idx])) > 1e-2


def test_apply_M_sites_without_clover_is_wilson():
    """csw = 0: apply_M_sites is the plain Wilson operator 1 - kappa D."""
    dims = (4, 4, 2, 4)
    U, _ = _random_fields(dims, seed=24)
    psi = synth.wilson_spinor(dims, 25).numpy()
    idx, xs = _sample_sites(dims, 20, 5)
    got = wilson.apply_M_sites(U, 0.0, 0.11, psi, xs, True, False)
    whole = wilson.apply_M(U, None, 0.11, psi, True).reshape(-1, 4, 3)[idx]
    assert np.max(np.abs(got - whole)) <= 1e-13 * np.max(np.abs(whole))
