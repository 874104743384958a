"""The double-single Wilson-clover operator (FP64 storage, float-float arithmetic) used for
the solvers' true residuals: it must agree with the FP64 operator to 1e-13 relative (and
the FP64 oracle to the same), and solves that use it must still reach the oracle's FP64
true residual of 1e-10."""
import numpy as np
import pytest
import torch

from helpers import F16, F64
from oracle import wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,csw,apbc", [((4, 4, 4, 4), 1.0, True), ((6, 6, 6, 10), 1.0, True),
                                           ((2, 2, 2, 2), 1.3, True), ((8, 4, 4, 6), 0.0, False)])
@pytest.mark.parametrize("dagger", [False, True])
def test_ds_operator_matches_fp64(dirac, dims, csw, apbc, dagger):
    kappa = 0.127
    U = synth.wilson_gauge(dims, 0.5, 1, 71)
    psi = synth.wilson_spinor(dims, 72)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=csw, t_antiperiodic=apbc)
    lat.load_gauge(U)
    x = lat.to_device(psi.cuda(), F64)
    y64, yds = lat.new_field(F64), lat.new_field(F64)
    (lat.apply_dagger if dagger else lat.apply)(y64, x, dirac.PARITY_FULL, F64)
    lat.apply_ds(yds, x, dagger)
    a = lat.to_natural(y64, F64, device="cpu").numpy()
    b = lat.to_natural(yds, F64, device="cpu").numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(a) <= 1e-13
    A = wilson.clover(U.numpy(), csw) if csw else None
    ref = wilson.apply_M(U.numpy(), A, kappa, psi.numpy(), apbc, dagger=dagger)
    assert np.linalg.norm(b - ref) / np.linalg.norm(ref) <= 1e-13
    lat.close()


def test_ds_operator_rejections(dirac):
    lat = dirac.Lattice((4, 4, 4, 4), dirac.ASQTAD, mass=0.1)
    f = lat.new_field(F64)
    assert dirac.dirac_apply_ds(lat.ctx, f.data_ptr(), lat.new_field(F64).data_ptr(), 0, None) in (
        dirac.ERR_UNSUPPORTED, dirac.ERR_STATE)
    lw = dirac.Lattice((4, 4, 4, 4), dirac.WILSON_CLOVER, kappa=0.12, recon=(12, 12, 12))
    lw.load_gauge(synth.wilson_gauge((4, 4, 4, 4), 0.5, 1, 3))
    g = lw.new_field(F64)
    assert dirac.dirac_apply_ds(lw.ctx, g.data_ptr(), lw.new_field(F64).data_ptr(), 0, None) == dirac.ERR_UNSUPPORTED


@pytest.mark.parametrize("alg", ["BICGSTAB", "GCR_DD", "CG_NORMAL"])
def test_solves_with_ds_residuals_reach_1e10(dirac, alg):
    """Mixed solves whose restarts / reliable updates use the double-single residual; the
    oracle recomputes the FP64 true residual of the returned x."""
    dims, kappa = (8, 8, 8, 8), 0.124
    U = synth.wilson_gauge(dims, 0.5, 3, 73)
    b = synth.wilson_spinor(dims, 74)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, block=(4, 4, 4, 4), mr_steps=6)
    lat.load_gauge(U)
    fb = lat.to_device(b.cuda(), F64)
    res = {}
    for ds in (True, False):
        lat.set_ds_residual(ds)
        fx = lat.new_field(F64)
        st = lat.solve(fx, fb, getattr(dirac, alg), tol=1e-10, max_iter=4000, delta=0.1,
                       prec_sloppy=F16 if alg != "CG_NORMAL" else dirac.F32, prec_precond=F16)
        assert st["true_rel_resid"] <= 1e-10
        x = lat.to_natural(fx, F64, device="cpu").numpy()
        A = wilson.clover(U.numpy(), 1.0)
        Mx = wilson.apply_M(U.numpy(), A, kappa, x)
        if alg == "CG_NORMAL":
            Mx = wilson.apply_M(U.numpy(), A, kappa, Mx, dagger=True)
        e = np.linalg.norm(b.numpy() - Mx) / np.linalg.norm(b.numpy())
        assert e <= 1e-10, (ds, e)
        res[ds] = st["iters"]
    # the residual arithmetic does not make the solve take meaningfully longer (BiCGstab's
    # iteration counts move by rounding either way)
    assert res[True] <= 1.25 * res[False] + 8, res
    lat.close()
