"""C-ABI argument checking and error reporting (no kernel is given a bad input)."""
import ctypes

import pytest

from helpers import F16, F32, F64
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _params(dirac, dims=(4, 4, 4, 4), kind=0, block=(2, 2, 2, 2)):
    p = dirac.DiracParams()
    p.dims[:] = list(dims)
    p.kind = kind
    p.kappa = 0.1
    p.block[:] = list(block)
    p.mr_steps = 2
    p.recon[:] = [18, 12, 12]
    return p


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 3), (1, 1, 1, 1)), ((0, 4, 4, 4), (1, 1, 1, 1)),
                                        ((4, 4, 4, 4), (3, 1, 1, 1)), ((8, 8, 8, 8), (8, 8, 8, 1))])
def test_create_rejects_bad_geometry(dirac, dims, block):
    h = ctypes.c_void_p()
    p = _params(dirac, dims, 0, block)
    assert dirac.dirac_create(ctypes.byref(p), ctypes.byref(h)) == dirac.ERR_ARG
    assert not h.value


def test_state_and_argument_errors(dirac):
    lat = dirac.Lattice((4, 4, 4, 4), dirac.WILSON_CLOVER, kappa=0.1, csw=1.0, block=(2, 2, 2, 2))
    x = lat.new_field(dirac.F64)
    y = lat.new_field(dirac.F64)
    rc = dirac.dirac_apply(lat.ctx, y.data_ptr(), x.data_ptr(), -1, 0, None)
    assert rc == dirac.ERR_STATE
    assert b"gauge" in dirac.dirac_last_error(lat.ctx)
    lat.load_gauge(synth.wilson_gauge((4, 4, 4, 4), 0.5, 0, 1))
    assert dirac.dirac_apply(lat.ctx, x.data_ptr(), x.data_ptr(), -1, 0, None) == dirac.ERR_ARG
    assert dirac.dirac_apply(lat.ctx, y.data_ptr(), x.data_ptr(), -1, 7, None) == dirac.ERR_ARG
    assert dirac.dirac_apply_normal(lat.ctx, y.data_ptr(), x.data_ptr(), 0, 0, None) == dirac.ERR_UNSUPPORTED


def test_asqtad_rejects_schwarz_and_wrong_links(dirac):
    lat = dirac.Lattice((4, 4, 4, 4), dirac.ASQTAD, mass=0.1)
    U = synth.unit_gauge((4, 4, 4, 4))
    with pytest.raises(dirac.DiracError):
        lat.load_gauge(U, 0)
    lat.load_gauge(U, 1)
    lat.load_gauge(U, 2)
    x, y = lat.new_field(dirac.F32), lat.new_field(dirac.F32)
    assert dirac.schwarz_precondition(lat.ctx, y.data_ptr(), x.data_ptr(), 1, None) == dirac.ERR_UNSUPPORTED


def test_precision_outside_mask(dirac):
    lat = dirac.Lattice((4, 4, 4, 4), dirac.WILSON_CLOVER, kappa=0.1, prec_mask=1)
    lat.load_gauge(synth.unit_gauge((4, 4, 4, 4)))
    x, y = lat.new_field(dirac.F16), lat.new_field(dirac.F16)
    assert dirac.dirac_apply(lat.ctx, y.data_ptr(), x.data_ptr(), -1, 2, None) == dirac.ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("parity", [-1, 0, 1])
def test_host_array_paths_agree(dirac, prec, parity):
    """A natural array in device memory, in page-locked host memory (read and written in
    place by the conversion kernels for FP64/FP32) and in pageable host memory gives the
    same device field and the same exported array, bit for bit; an export of one parity
    leaves the other parity's sites of the host array untouched."""
    import torch
    from paper_1109_2935_gb300 import synth
    dims = (6, 4, 4, 8)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12)
    psi = synth.wilson_spinor(dims, 5)
    fields = []
    for src in (psi.cuda(), psi.clone().pin_memory(), psi.clone()):
        f = lat.new_field(prec, parity)
        lat.import_spinor(f, prec, parity, src)
        fields.append(f)
    assert torch.equal(fields[0], fields[1]) and torch.equal(fields[0], fields[2])
    marker = torch.full_like(psi, 7.0 + 0.0j)
    outs = []
    for dst in (marker.cuda(), marker.clone().pin_memory(), marker.clone()):
        lat.export_spinor(fields[0], prec, parity, dst)
        torch.cuda.synchronize()
        outs.append(dst.cpu())
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    if parity >= 0:
        LX, LY, LZ, LT = dims
        t, z, y, x = torch.meshgrid(torch.arange(LT), torch.arange(LZ), torch.arange(LY), torch.arange(LX),
                                    indexing="ij")
        other = ((t + z + y + x) % 2) != parity
        assert torch.all(outs[1][other] == 7.0)
