"""GPU parity of the BLAS-1 / reduction entry points (FP64 accumulation) against
numpy on the exported fields, plus precision conversion round trips."""
import numpy as np
import pytest

from helpers import F16, F32, F64, dec_spinor
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,dims", [(0, (6, 6, 6, 10)), (1, (8, 6, 4, 6)), (0, (2, 2, 2, 2))])
@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("parity", [-1, 0, 1])
def test_reductions(dirac, kind, dims, prec, parity):
    lat = dirac.Lattice(dims, kind, kappa=0.1, mass=0.1)
    gen = synth.wilson_spinor if kind == 0 else synth.staggered_spinor
    a, b = gen(dims, 1), gen(dims, 2)
    fa = lat.to_device(a.cuda(), prec, parity)
    fb = lat.to_device(b.cuda(), prec, parity)
    na = lat.to_natural(fa, prec, parity, device="cpu").numpy()
    nb = lat.to_natural(fb, prec, parity, device="cpu").numpy()
    # FP64 fields: FP64 arithmetic. FP32/FP16 fields: FP32 products summed per site, then
    # FP64 accumulation across sites, so a few FP32 ulps relative.
    tol = 1e-13 if prec == F64 else 1e-6
    assert abs(lat.norm2(fa, prec, parity) - np.vdot(na, na).real) <= tol * np.vdot(na, na).real
    d = lat.cdot(fa, fb, prec, parity)
    assert abs(d - np.vdot(na, nb)) <= tol * np.sqrt(np.vdot(na, na).real * np.vdot(nb, nb).real)
    alpha = 0.3 - 0.7j
    r = lat.caxpy_norm(alpha, fa, fb, prec, parity)
    nb2 = lat.to_natural(fb, prec, parity, device="cpu").numpy()
    expect = nb + alpha * na
    rel = 1e-14 if prec == F64 else (1e-6 if prec == F32 else 2e-3)
    assert np.linalg.norm(nb2 - expect) <= rel * np.linalg.norm(expect) * 4
    assert abs(r - np.vdot(nb2, nb2).real) <= tol * np.vdot(nb2, nb2).real


@pytest.mark.parametrize("src,dst", [(F64, F32), (F64, F16), (F32, F16), (F16, F64), (F32, F64)])
def test_convert(dirac, src, dst):
    dims = (6, 4, 4, 8)
    lat = dirac.Lattice(dims, 0)
    psi = synth.wilson_spinor(dims, 9)
    fs = lat.to_device(psi.cuda(), src)
    fd = lat.new_field(dst)
    lat.convert(fd, dst, fs, src)
    got = lat.to_natural(fd, dst, device="cpu").numpy()
    ref = dec_spinor(dec_spinor(psi.numpy(), src), dst)
    tol = {F64: 1e-15, F32: 2e-7, F16: 2e-3}[max(src, dst)]
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref) * 4


def test_import_export_roundtrip_exact_f64(dirac):
    dims = (6, 6, 4, 10)
    lat = dirac.Lattice(dims, 0)
    psi = synth.wilson_spinor(dims, 11)
    f = lat.to_device(psi.cuda(), F64)
    back = lat.to_natural(f, F64, device="cpu")
    assert np.array_equal(back.numpy(), psi.numpy())
    # a half-field export leaves the other parity of the destination untouched
    import torch
    dst = torch.full(lat.natural_shape(), 5.0 + 0j, dtype=torch.complex128)
    fe = lat.to_device(psi.cuda(), F64, 0)
    lat.export_spinor(fe, F64, 0, dst)
    from helpers import parity_mask
    m = parity_mask(dims, 0)
    assert np.array_equal(dst.numpy()[m], psi.numpy()[m])
    assert np.all(dst.numpy()[~m] == 5.0)
