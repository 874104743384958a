"""GPU parity of the Wilson-clover operator (Eq. 2) against the FP64 oracle, through
the C ABI: full M and M^dagger with the clover term, the parity hopping blocks
D_eo / D_oe and their adjoints, in FP64 / FP32 / FP16 storage with 18-, 12- and
8-real links, on lattices whose half-volume leaves a ragged last thread block."""
import numpy as np
import pytest
import torch

from helpers import F16, F32, F64, check, dec_clover_hat, dec_links, dec_spinor, parity_mask
from oracle import wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), 1), ((6, 6, 6, 10), 3), ((2, 2, 2, 2), 1), ((8, 4, 6, 4), 3)]


def _setup(dirac, dims, smear, prec, recon, csw=1.0, kappa=0.13, apbc=True):
    U = synth.wilson_gauge(dims, 0.5, smear, 100 + sum(dims))
    psi = synth.wilson_spinor(dims, 200 + sum(dims))
    rc = (recon, recon, recon)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=csw, t_antiperiodic=apbc,
                        block=(2, 2, 2, 2), recon=rc)
    lat.load_gauge(U)
    Un = U.numpy()
    A = wilson.clover(Un, csw) if csw else None
    Ahat = np.eye(12) + 2 * kappa * A if csw else None
    Ud = dec_links(Un, prec)
    if csw:
        Ad = (dec_clover_hat(Ahat, prec) - np.eye(12)) / (2 * kappa)
    else:
        Ad = None
    return lat, U, psi, Ud, Ad


@pytest.mark.parametrize("dims,smear", CASES)
@pytest.mark.parametrize("prec,recon", [(F64, 18), (F64, 12), (F32, 18), (F32, 12), (F32, 8),
                                        (F16, 18), (F16, 12), (F16, 8)])
@pytest.mark.parametrize("dagger", [False, True])
def test_full_operator(dirac, dims, smear, prec, recon, dagger):
    lat, U, psi, Ud, Ad = _setup(dirac, dims, smear, prec, recon)
    x = lat.to_device(psi.cuda(), prec)
    y = lat.new_field(prec)
    (lat.apply_dagger if dagger else lat.apply)(y, x, dirac.PARITY_FULL, prec)
    got = lat.to_natural(y, prec, device="cpu").numpy()
    ref = wilson.apply_M(Ud, Ad, 0.13, dec_spinor(psi.numpy(), prec), True, dagger=dagger)
    check(got, ref, prec, 24, f"M dims={dims} prec={prec} recon={recon} dag={dagger}")


@pytest.mark.parametrize("dims,smear", CASES[:2])
@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_parity_dslash(dirac, dims, smear, prec, parity, dagger):
    lat, U, psi, Ud, _ = _setup(dirac, dims, smear, prec, 12)
    src = lat.to_device(psi.cuda(), prec, 1 - parity)
    out = lat.new_field(prec, parity)
    (lat.apply_dagger if dagger else lat.apply)(out, src, parity, prec)
    got = lat.to_natural(out, prec, parity, device="cpu").numpy()
    m_out = parity_mask(dims, parity)
    m_in = parity_mask(dims, 1 - parity)
    ref = wilson.dslash(Ud, dec_spinor(psi.numpy(), prec) * m_in[..., None, None], True, dagger=dagger)
    check(got[m_out], ref[m_out], prec, 24, f"D parity={parity} prec={prec}")


@pytest.mark.parametrize("apbc", [True, False])
def test_plain_wilson_no_clover(dirac, apbc):
    """c_sw = 0 (the 4^4, kappa = 0.12, sigma = 0.3 configuration): M = 1 - kappa D."""
    dims = (4, 4, 4, 4)
    U = synth.wilson_gauge(dims, 0.3, 0, 1001)
    psi = synth.wilson_spinor(dims, 1002)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=0.0, t_antiperiodic=apbc,
                        recon=(18, 12, 12))
    lat.load_gauge(U)
    x = lat.to_device(psi.cuda(), F64)
    y = lat.new_field(F64)
    lat.apply(y, x, dirac.PARITY_FULL, F64)
    got = lat.to_natural(y, F64, device="cpu").numpy()
    ref = wilson.apply_M(U.numpy(), None, 0.12, psi.numpy(), apbc)
    check(got, ref, F64, 24, "plain Wilson")


def test_free_field_eigenvalue_on_gpu(dirac):
    """Unit links, plane wave: the GPU operator reproduces the closed form exactly."""
    dims = (4, 4, 4, 8)
    from oracle.gamma import GAMMA
    from oracle.lattice import all_coords
    rng = np.random.default_rng(0)
    s = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    n = (1, 2, 0, 1)
    p = np.array([2 * np.pi * n[m] / dims[m] for m in range(4)])
    p[3] = (2 * n[3] + 1) * np.pi / dims[3]
    ph = np.exp(1j * (all_coords(dims) @ p))
    psi = torch.from_numpy((ph[:, None, None] * s[None]).reshape(8, 4, 4, 4, 4, 3))
    kappa = 0.1
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, recon=(18, 12, 12))
    lat.load_gauge(synth.unit_gauge(dims))
    x = lat.to_device(psi.cuda(), F64)
    y = lat.new_field(F64)
    lat.apply(y, x, dirac.PARITY_FULL, F64)
    got = lat.to_natural(y, F64, device="cpu").numpy().reshape(-1, 4, 3)
    K = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    expect = ph[:, None, None] * (K @ s)[None]
    assert np.max(np.abs(got - expect)) < 1e-13


def test_gamma5_hermiticity_on_gpu(dirac):
    dims = (4, 4, 6, 4)
    U = synth.wilson_gauge(dims, 0.5, 1, 7)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.13, csw=1.2, recon=(18, 12, 12))
    lat.load_gauge(U)
    xs = [synth.wilson_spinor(dims, s) for s in (1, 2)]
    f = [lat.to_device(v.cuda(), F64) for v in xs]
    Mx, Mdy = lat.new_field(F64), lat.new_field(F64)
    lat.apply(Mx, f[0], dirac.PARITY_FULL, F64)
    lat.apply_dagger(Mdy, f[1], dirac.PARITY_FULL, F64)
    a = lat.cdot(f[1], Mx, F64)
    b = lat.cdot(Mdy, f[0], F64)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_operator(dirac, prec, dagger):
    """Even-odd Schur complement Ahat_ee - kappa^2 D_eo Ahat_oo^-1 D_oe (Sec. 3.1)."""
    dims = (6, 6, 6, 10)
    kappa = 0.13
    lat, U, psi, Ud, Ad = _setup(dirac, dims, 3, prec, 12, kappa=kappa)
    x = lat.to_device(psi.cuda(), prec, 0)
    y = lat.new_field(prec, 0)
    lat.apply_eo(y, x, prec, dagger)
    got = lat.to_natural(y, prec, 0, device="cpu").numpy()
    ev = parity_mask(dims, 0)
    ref = wilson.apply_schur(Ud, Ad, kappa, dec_spinor(psi.numpy(), prec) * ev[..., None, None], True, dagger)
    check(got[ev], ref[ev], prec, 24, f"Schur prec={prec} dag={dagger}")
