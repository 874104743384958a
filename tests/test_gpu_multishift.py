"""Multi-shift solves of Eq. 4 (Sec. 8.2 strategy: sloppy multi-shift CG, then mixed
precision refinement per shift), checked by the FP64 oracle: every x_j must satisfy
||b - (M^dagger M + sigma_j) x_j|| / ||b|| <= 1e-10."""
import ctypes

import numpy as np
import pytest

from helpers import F32, F64
from oracle import solvers as osolv
from oracle import staggered, wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _asqtad(dirac, dims, m):
    fat, lng = synth.asqtad_links(dims, 3001, 3002)
    b = synth.staggered_spinor(dims, 3003, parity=0)
    lat = dirac.Lattice(dims, dirac.ASQTAD, mass=m, recon=(18, 12, 12))
    lat.load_gauge(fat, 1)
    lat.load_gauge(lng, 2)
    fn, ln = fat.numpy(), lng.numpy()
    even = staggered.parity_mask(dims, 0)[..., None]
    N = lambda v: staggered.apply_normal(fn, ln, m, v * even) * even
    return lat, b, N, even


@pytest.mark.parametrize("sloppy", [F32, F64])
def test_asqtad_multishift_each_shift_to_1e10(dirac, sloppy):
    dims = (8, 8, 8, 8)
    lat, b, N, even = _asqtad(dirac, dims, 0.05)
    shifts = [0.1, 0.0, 1.0, 0.01]
    fb = lat.to_device(b.cuda(), F64, 0)
    xs = [lat.new_field(F64, 0) for _ in shifts]
    st = lat.solve_multishift(xs, fb, shifts, dirac.CG_EVEN_NORMAL, tol=1e-10, max_iter=5000,
                              delta=0.1, prec_sloppy=sloppy)
    bn = b.numpy()
    for sgm, fx, rst in zip(shifts, xs, st["refine"]):
        x = lat.to_natural(fx, F64, 0, device="cpu").numpy() * even
        res = np.linalg.norm(bn - N(x) - sgm * x) / np.linalg.norm(bn)
        assert res <= 1e-10, (sgm, res, st)
        assert abs(rst["true_rel_resid"] - res) < 1e-12
    assert st["multishift"]["iters"] > 0


def test_multishift_fp64_stage_matches_oracle(dirac):
    """All-FP64 multi-shift stage: the same Krylov recurrences as the oracle's, so the
    solutions agree and the iteration count matches (one extra step at most, the
    stop being read one iteration behind)."""
    dims = (4, 4, 4, 8)
    m = 0.1
    lat, b, N, even = _asqtad(dirac, dims, m)
    shifts = [0.0, 0.05, 0.5]
    fb = lat.to_device(b.cuda(), F64, 0)
    xs = [lat.new_field(F64, 0) for _ in shifts]
    st = lat.solve_multishift(xs, fb, shifts, dirac.CG_EVEN_NORMAL, tol=1e-9, max_iter=2000,
                              delta=0.0, prec_sloppy=F64)
    xo, info = osolv.multishift_cg(N, b.numpy(), shifts, 1e-9, 2000)
    for j, fx in enumerate(xs):
        x = lat.to_natural(fx, F64, 0, device="cpu").numpy() * even
        assert np.linalg.norm(x - xo[j]) / np.linalg.norm(xo[j]) < 1e-9, j
    assert abs(st["multishift"]["iters"] - info["iters"]) <= 1


def test_wilson_normal_multishift(dirac):
    dims = (4, 4, 4, 4)
    U = synth.wilson_gauge(dims, 0.3, 0, 1001)
    b = synth.wilson_spinor(dims, 1002)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=1.0, recon=(18, 12, 12))
    lat.load_gauge(U)
    shifts = [0.05, 0.5]
    fb = lat.to_device(b.cuda(), F64)
    xs = [lat.new_field(F64) for _ in shifts]
    lat.solve_multishift(xs, fb, shifts, dirac.CG_NORMAL, tol=1e-10, max_iter=3000, prec_sloppy=F32)
    Un = U.numpy()
    A = wilson.clover(Un, 1.0)
    Nn = lambda v: wilson.apply_M(Un, A, 0.12, wilson.apply_M(Un, A, 0.12, v), dagger=True)
    for sgm, fx in zip(shifts, xs):
        x = lat.to_natural(fx, F64, device="cpu").numpy()
        bn = b.numpy()
        assert np.linalg.norm(bn - Nn(x) - sgm * x) / np.linalg.norm(bn) <= 1e-10


def test_multishift_argument_checks(dirac):
    dims = (4, 4, 4, 4)
    lat, b, N, even = _asqtad(dirac, dims, 0.1)
    fb = lat.to_device(b.cuda(), F64, 0)
    x = lat.new_field(F64, 0)
    sp = dirac.SolverParams(dirac.CG_EVEN_NORMAL, 1e-10, 100, 16, 0.1, 1, F32, F32)
    ptr = (ctypes.c_void_p * 1)(x.data_ptr())
    neg = (ctypes.c_double * 1)(-0.5)
    assert dirac.solve_multishift(lat.ctx, ptr, fb.data_ptr(), neg, 1, ctypes.byref(sp), None, None) == dirac.ERR_ARG
    zero = (ctypes.c_double * 1)(0.0)
    assert dirac.solve_multishift(lat.ctx, ptr, fb.data_ptr(), zero, 0, ctypes.byref(sp), None, None) == dirac.ERR_ARG
    sp.alg = dirac.BICGSTAB
    assert dirac.solve_multishift(lat.ctx, ptr, fb.data_ptr(), zero, 1, ctypes.byref(sp), None, None) == dirac.ERR_UNSUPPORTED
