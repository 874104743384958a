"""C-ABI argument checking and error reporting (no kernel is given a bad input)."""
import ctypes

import pytest

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
