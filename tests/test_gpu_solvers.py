"""GPU solves (CG, BiCGstab, GCR, GCR-DD of Algorithm 1) checked by the FP64 oracle:
the oracle recomputes ||b - A x|| / ||b|| from the exported solution, which must be
<= the requested tolerance (1e-10), in pure FP64 and in mixed precision."""
import numpy as np
import pytest
import torch

from helpers import F16, F32, F64
from oracle import staggered, wilson
from oracle import solvers as osolv
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _oracle_resid(A, x, b):
    r = b - A(x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("sloppy,delta", [(F64, 0.0), (F32, 0.1), (F16, 0.1)])
def test_cg_normal_4444(dirac, sloppy, delta):
    """4^4 plain Wilson (kappa = 0.12, sigma = 0.3, antiperiodic t): CG on
    M^dagger M x = b to 1e-10, and the same solution as the oracle's CG."""
    dims = (4, 4, 4, 4)
    U = synth.wilson_gauge(dims, 0.3, 0, 1001)
    b = synth.wilson_spinor(dims, 1002)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=0.0, recon=(18, 12, 12))
    lat.load_gauge(U)
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, dirac.CG_NORMAL, tol=1e-10, max_iter=2000, delta=delta, prec_sloppy=sloppy)
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    Un = U.numpy()
    N = lambda v: wilson.apply_M(Un, None, 0.12, wilson.apply_M(Un, None, 0.12, v), dagger=True)
    assert _oracle_resid(N, x, b.numpy()) <= 1e-10
    assert abs(st["true_rel_resid"] - _oracle_resid(N, x, b.numpy())) < 1e-12
    xo, _ = osolv.cg(N, b.numpy(), 1e-12, 2000)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-8


def _wc_problem(dirac, dims, kappa, block=(4, 4, 4, 4), steps=6, seed=2001):
    U = synth.wilson_gauge(dims, 0.5, 3, seed)
    b = synth.wilson_spinor(dims, seed + 1)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, block=block,
                        mr_steps=steps, recon=(18, 12, 12))
    lat.load_gauge(U)
    Un = U.numpy()
    A = wilson.clover(Un, 1.0)
    M = lambda v: wilson.apply_M(Un, A, kappa, v)
    return lat, b, M


@pytest.mark.parametrize("alg,sloppy,precond,delta", [
    ("BICGSTAB", F64, F64, 0.0), ("BICGSTAB", F32, F32, 0.1), ("BICGSTAB", F16, F16, 0.1),
    ("GCR", F64, F64, 0.0),
    ("GCR_DD", F64, F64, 0.0), ("GCR_DD", F32, F16, 1e-3), ("GCR_DD", F16, F16, 0.1),
])
def test_wilson_clover_solvers(dirac, alg, sloppy, precond, delta):
    dims = (8, 8, 8, 8)
    lat, b, M = _wc_problem(dirac, dims, 0.124)
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, getattr(dirac, alg), tol=1e-10, max_iter=4000, k_max=16, delta=delta,
                   prec_sloppy=sloppy, prec_precond=precond)
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    res = _oracle_resid(M, x, b.numpy())
    assert res <= 1e-10, (alg, st)
    assert abs(st["true_rel_resid"] - res) < 1e-12


@pytest.mark.parametrize("alg,sloppy,delta", [("BICGSTAB_EO", F64, 0.0), ("BICGSTAB_EO", F16, 0.1),
                                               ("GCR_EO", F64, 0.0), ("GCR_EO", F32, 1e-3)])
def test_even_odd_solvers(dirac, alg, sloppy, delta):
    """Even-odd preconditioned solves (Sec. 3.1): the Schur system on even sites, then
    x_o rebuilt; the FP64 oracle checks the full system M x = b, and the Schur system
    needs fewer iterations than the unpreconditioned one."""
    dims = (8, 8, 8, 8)
    lat, b, M = _wc_problem(dirac, dims, 0.124)
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, getattr(dirac, alg), tol=1e-10, max_iter=4000, k_max=16, delta=delta,
                   prec_sloppy=sloppy, prec_precond=sloppy)
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    res = _oracle_resid(M, x, b.numpy())
    assert res <= 1e-10, (alg, st)
    assert abs(st["true_rel_resid"] - res) < 1e-12
    fx2 = lat.new_field(F64)
    base = "BICGSTAB" if alg.startswith("BICG") else "GCR"
    st0 = lat.solve(fx2, fb, getattr(dirac, base), tol=1e-10, max_iter=4000, k_max=16, delta=delta,
                    prec_sloppy=sloppy, prec_precond=sloppy)
    assert st["iters"] < st0["iters"], (st, st0)


def test_gcr_dd_first_cycle_matches_oracle(dirac):
    """FP64 GCR-DD: after one restart cycle the GPU iterate equals the oracle's
    Algorithm 1 with the oracle's Schwarz preconditioner (same k_max, same steps)."""
    dims = (8, 4, 4, 8)
    lat, b, M = _wc_problem(dirac, dims, 0.124, block=(4, 4, 4, 4), steps=4, seed=77)
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, dirac.GCR_DD, tol=1e-10, max_iter=5, k_max=5, delta=0.0,
                   prec_sloppy=F64, prec_precond=F64, raise_on_error=False)
    assert st["iters"] == 5 and st["restarts"] == 1
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    U = synth.wilson_gauge(dims, 0.5, 3, 77).numpy()
    A = wilson.clover(U, 1.0)
    K = lambda r: osolv.schwarz_mr(U, A, 0.124, r, (4, 4, 4, 4), 4)
    xo, info = osolv.gcr(M, K, b.numpy(), 1e-10, 5, 5, 0.0)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-11


@pytest.mark.parametrize("sloppy,delta", [(F64, 0.0), (F32, 0.1), (F16, 0.1)])
def test_staggered_even_cg(dirac, sloppy, delta):
    dims = (8, 8, 8, 8)
    m = 0.05
    fat, lng = synth.asqtad_links(dims, 3001, 3002)
    b = synth.staggered_spinor(dims, 3003, parity=0)
    lat = dirac.Lattice(dims, dirac.ASQTAD, mass=m, recon=(18, 12, 12))
    lat.load_gauge(fat, 1)
    lat.load_gauge(lng, 2)
    fb = lat.to_device(b.cuda(), F64, 0)
    fx = lat.new_field(F64, 0)
    st = lat.solve(fx, fb, dirac.CG_EVEN_NORMAL, tol=1e-10, max_iter=5000, delta=delta,
                   prec_sloppy=sloppy)
    x = lat.to_natural(fx, F64, 0, device="cpu").numpy()
    fn, ln = fat.numpy(), lng.numpy()
    even = staggered.parity_mask(dims, 0)[..., None]
    N = lambda v: staggered.apply_normal(fn, ln, m, v * even) * even
    assert _oracle_resid(N, x * even, b.numpy()) <= 1e-10, st


def test_zero_source_gives_zero(dirac):
    dims = (4, 4, 4, 4)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=1.0, recon=(18, 12, 12))
    lat.load_gauge(synth.wilson_gauge(dims, 0.5, 1, 1))
    fb = lat.new_field(F64)
    fx = lat.new_field(F64)
    fx.fill_(3)
    st = lat.solve(fx, fb, dirac.BICGSTAB, tol=1e-10)
    assert lat.norm2(fx, F64) == 0.0 and st["iters"] == 0


def test_not_converged_status(dirac):
    dims = (8, 8, 8, 8)
    lat, b, M = _wc_problem(dirac, dims, 0.124)
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, dirac.BICGSTAB, tol=1e-10, max_iter=3, raise_on_error=False)
    assert st["status"] == "ERR_NOT_CONVERGED" and st["iters"] == 3
    assert 0 < st["true_rel_resid"] < 1


@pytest.mark.parametrize("alg", ["BICGSTAB", "GCR_DD", "CG_NORMAL", "BICGSTAB_EO"])
def test_nonfinite_source_is_reported(dirac, alg):
    """A NaN in the source is detected from the device-side scalars and reported as
    DIRAC_ERR_NONFINITE (failure injected on the host side, in the data)."""
    dims = (4, 4, 4, 4)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=1.0, block=(2, 2, 2, 2),
                        recon=(18, 12, 12))
    lat.load_gauge(synth.wilson_gauge(dims, 0.5, 1, 1))
    b = synth.wilson_spinor(dims, 2)
    b[1, 2, 3, 0, 1, 2] = float("nan")
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, getattr(dirac, alg), tol=1e-10, max_iter=50, prec_sloppy=F32,
                   prec_precond=F32, raise_on_error=False)
    assert st["status"] == "ERR_NONFINITE", st


@pytest.mark.parametrize("alg", ["CG_NORMAL", "BICGSTAB", "GCR"])
def test_singular_operator_is_reported(dirac, alg):
    """Free Wilson operator, periodic in t, kappa = 1/8: the constant spinor is an exact
    zero mode (M 1 = (1 - 8 kappa) 1 = 0), so M x = b has no solution for a generic b.
    Every solver stops within its budget with a status (not converged or breakdown)
    instead of returning OK or running on."""
    dims = (4, 4, 4, 4)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.125, csw=0.0, t_antiperiodic=False)
    lat.load_gauge(synth.unit_gauge(dims))
    # the zero mode exists on the device too
    one = torch.zeros(dims[::-1] + (4, 3), dtype=torch.complex128)
    one[..., 0, 0] = 1.0
    f1 = lat.to_device(one.cuda(), F64)
    m1 = lat.new_field(F64)
    lat.apply(m1, f1, dirac.PARITY_FULL, F64)
    assert lat.norm2(m1, F64) < 1e-28
    fb = lat.to_device(synth.wilson_spinor(dims, 5).cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, getattr(dirac, alg), tol=1e-10, max_iter=300, raise_on_error=False)
    assert st["status"] in ("ERR_NOT_CONVERGED", "ERR_BREAKDOWN"), st
    assert st["iters"] <= 300
