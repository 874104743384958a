"""GPU parity of the asqtad operator (Eq. 3, anti-Hermitian reading with eta phases)
against the FP64 oracle through the C ABI: parity hopping blocks, the full operator
and its adjoint, and the even-site normal operator, in FP64 / FP32 / FP16 storage
with 18-, 12- and 8-real long links. 4^4 lattices make the 3-hop alias a 1-hop."""
import numpy as np
import pytest

from helpers import F16, F32, F64, check, dec_links, dec_spinor, parity_mask
from oracle import staggered
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [(4, 4, 4, 4), (6, 4, 6, 10), (8, 6, 4, 6)]
MASS = 0.01


def _setup(dirac, dims, prec, recon, apbc=True):
    fat, lng = synth.asqtad_links(dims, 3001 + dims[0], 3002 + dims[1])
    psi = synth.staggered_spinor(dims, 3003 + dims[3])
    lat = dirac.Lattice(dims, dirac.ASQTAD, mass=MASS, t_antiperiodic=apbc, recon=(recon,) * 3)
    lat.load_gauge(fat, 1)
    lat.load_gauge(lng, 2)
    return lat, dec_links(fat.numpy(), prec), dec_links(lng.numpy(), prec), psi


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("prec,recon", [(F64, 18), (F64, 12), (F32, 18), (F32, 12), (F32, 8),
                                        (F16, 18), (F16, 12), (F16, 8)])
@pytest.mark.parametrize("parity", [0, 1])
def test_parity_dslash(dirac, dims, prec, recon, parity):
    lat, fat, lng, psi = _setup(dirac, dims, prec, recon)
    src = lat.to_device(psi.cuda(), prec, 1 - parity)
    out = lat.new_field(prec, parity)
    lat.apply(out, src, parity, prec)
    got = lat.to_natural(out, prec, parity, device="cpu").numpy()
    m_out, m_in = parity_mask(dims, parity), parity_mask(dims, 1 - parity)
    ref = staggered.dslash(fat, lng, dec_spinor(psi.numpy(), prec) * m_in[..., None])
    check(got[m_out], ref[m_out], prec, 6, f"asqtad D dims={dims} prec={prec} recon={recon}")


@pytest.mark.parametrize("dims", CASES[:2])
@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("apbc", [True, False])
def test_full_operator(dirac, dims, prec, dagger, apbc):
    lat, fat, lng, psi = _setup(dirac, dims, prec, 12, apbc)
    x = lat.to_device(psi.cuda(), prec)
    y = lat.new_field(prec)
    (lat.apply_dagger if dagger else lat.apply)(y, x, dirac.PARITY_FULL, prec)
    got = lat.to_natural(y, prec, device="cpu").numpy()
    ref = staggered.apply_M(fat, lng, MASS, dec_spinor(psi.numpy(), prec), apbc, dagger=dagger)
    check(got, ref, prec, 6, f"asqtad M prec={prec} dag={dagger}")


@pytest.mark.parametrize("dims", CASES[:2])
@pytest.mark.parametrize("prec", [F64, F32])
def test_even_normal_operator(dirac, dims, prec):
    """(M^dagger M)_ee = m^2 - 1/4 D_eo D_oe on a half-field."""
    lat, fat, lng, psi = _setup(dirac, dims, prec, 12)
    even = parity_mask(dims, 0)
    x = lat.to_device(psi.cuda(), prec, 0)
    y = lat.new_field(prec, 0)
    lat.apply_normal(y, x, 0, prec)
    got = lat.to_natural(y, prec, 0, device="cpu").numpy()
    ref = staggered.apply_normal(fat, lng, MASS, dec_spinor(psi.numpy(), prec) * even[..., None])
    check(got[even], ref[even], prec, 6, f"asqtad normal prec={prec}")


def test_anti_hermiticity_on_gpu(dirac):
    dims = (6, 4, 6, 10)
    lat, fat, lng, _ = _setup(dirac, dims, F64, 18)
    xe = lat.to_device(synth.staggered_spinor(dims, 5).cuda(), F64, 0)
    yo = lat.to_device(synth.staggered_spinor(dims, 6).cuda(), F64, 1)
    Dx = lat.new_field(F64, 1)
    Dy = lat.new_field(F64, 0)
    lat.apply(Dx, xe, 1, F64)   # D_oe x_e
    lat.apply(Dy, yo, 0, F64)   # D_eo y_o
    a = lat.cdot(yo, Dx, F64, 1)
    b = lat.cdot(Dy, xe, F64, 0)
    assert abs(a + b) < 1e-12 * abs(a)
