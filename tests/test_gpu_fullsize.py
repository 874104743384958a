"""Parity at the full workload sizes, in the launch configurations the benchmark
times: the 24^3x128 Wilson-clover operator (FP64-18, FP32-12, FP16-12; full M, M^dagger
and the parity dslash) and the 48^3x144 asqtad parity dslash. The oracle evaluates the
operators one site at a time at a random sample of output sites."""
import numpy as np
import pytest
import torch

from helpers import F16, F32, F64, check, dec_clover_hat, dec_spinor
from oracle import staggered, wilson
from oracle.lattice import all_coords
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _sample(dims, n, parity=None, seed=0):
    c = all_coords(dims)
    if parity is not None:
        c = c[c.sum(1) % 2 == parity]
    rng = np.random.default_rng(seed)
    s = c[rng.choice(len(c), n, replace=False)]
    # always include the lattice corners (wrapping hops in every direction)
    corners = np.array([[0, 0, 0, 0], [dims[0] - 1, dims[1] - 1, dims[2] - 1, dims[3] - 1]])
    if parity is not None:
        corners = corners[corners.sum(1) % 2 == parity]
    return np.concatenate([s, corners])


def _at(nat, s):
    return nat[s[:, 3], s[:, 2], s[:, 1], s[:, 0]]


@pytest.fixture(scope="module")
def wilson_full(dirac):
    dims = (24, 24, 24, 128)
    kappa, csw = 0.1350, 1.0
    U = synth.wilson_gauge(dims, 0.5, 3, 2001, device="cuda")
    psi = synth.wilson_spinor(dims, 2002, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=csw, block=(4, 4, 4, 4),
                        mr_steps=6, recon=(18, 12, 12))
    lat.load_gauge(U)
    yield lat, U.cpu().numpy(), psi, kappa, csw
    lat.close()


@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("dagger", [False, True])
def test_wilson_clover_24x128(dirac, wilson_full, prec, dagger):
    lat, Un, psi, kappa, csw = wilson_full
    dims = lat.dims
    x = lat.to_device(psi, prec)
    y = lat.new_field(prec)
    (lat.apply_dagger if dagger else lat.apply)(y, x, dirac.PARITY_FULL, prec)
    got = lat.to_natural(y, prec, device="cpu").numpy()
    s = _sample(dims, 384, seed=prec + 10 * dagger)
    psi_d = dec_spinor(psi.cpu().numpy(), prec)
    # F32/F16 links: the oracle takes the FP64 links; the kernel's link rounding is
    # within the FP32 bound, and within the FP16 per-site bound
    ref = wilson.apply_M_sites(Un, csw, kappa, psi_d, s, True, dagger,
                               Ahat_codec=lambda A: dec_clover_hat(A, prec))
    check(_at(got, s), ref, prec, 24, f"24^3x128 M prec={prec} dag={dagger}")


@pytest.mark.parametrize("parity", [0, 1])
def test_wilson_dslash_24x128_f32(dirac, wilson_full, parity):
    lat, Un, psi, kappa, csw = wilson_full
    dims = lat.dims
    src = lat.to_device(psi, F32, 1 - parity)
    out = lat.new_field(F32, parity)
    lat.apply(out, src, parity, F32)
    got = lat.to_natural(out, F32, parity, device="cpu").numpy()
    s = _sample(dims, 384, parity, seed=3 + parity)
    m = ((np.indices(psi.shape[:4]).sum(0)) % 2 == 1 - parity)
    psi_d = dec_spinor(psi.cpu().numpy(), F32) * m[..., None, None]
    ref = wilson.dslash(Un, psi_d, True, s)
    check(_at(got, s), ref, F32, 24, f"24^3x128 D_{parity}")


def _sampled_residual(Un, csw, kappa, b, x, dims, n=512, seed=9):
    """||b - M x|| / ||b|| over a random sample of sites (plus the corners), the oracle
    evaluating M one site at a time: an estimate of the true residual that does not use
    the library's own FP64 residual."""
    s = _sample(dims, n, seed=seed)
    mx = wilson.apply_M_sites(Un, csw, kappa, x, s, True, False)
    bs = _at(b, s)
    return np.linalg.norm(bs - mx) / np.linalg.norm(bs)


@pytest.mark.parametrize("alg,sloppy,precond,kappa", [
    ("BICGSTAB_EO", F16, F16, 0.124),
    ("GCR_DD", F16, F16, 0.124),
])
def test_solves_24x128_reach_1e10(dirac, alg, sloppy, precond, kappa):
    """Mixed-precision solves of the 24^3x128 workload as the benchmark runs them: the
    library's FP64 true residual <= 1e-10, and the oracle's sampled residual agrees."""
    dims = (24, 24, 24, 128)
    U = synth.wilson_gauge(dims, 0.5, 3, 2001, device="cuda")
    b = synth.wilson_spinor(dims, 2002, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, block=(4, 4, 4, 4), mr_steps=6,
                        recon=(18, 12, 12))
    lat.load_gauge(U)
    fb = lat.to_device(b, F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, getattr(dirac, alg), tol=1e-10, max_iter=4000, k_max=16, delta=0.1,
                   prec_sloppy=sloppy, prec_precond=precond)
    assert st["true_rel_resid"] <= 1e-10
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    est = _sampled_residual(U.cpu().numpy(), 1.0, kappa, b.cpu().numpy(), x, dims)
    assert est < 1e-9, est
    lat.close()


def test_learned_preconditioner_solve_24x128_kappa_0135(dirac):
    """At kappa 0.1350 (the workload as configured), GCR with a PTC network trained on a
    16^4 field at the same kappa and applied unchanged to 24^3x128 reaches 1e-10; the
    oracle's sampled residual agrees."""
    import bench
    dims = (24, 24, 24, 128)
    kappa = 0.135
    plat, pnet, _, _, _ = bench.train_ptc(dirac, synth, torch.device("cuda"), kappa)
    w = pnet.get_weights()
    plat.close()
    U = synth.wilson_gauge(dims, 0.5, 3, 2001, device="cuda")
    b = synth.wilson_spinor(dims, 2002, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, block=(4, 4, 4, 4), mr_steps=6,
                        recon=(18, 12, 12))
    lat.load_gauge(U)
    net = dirac.Ptc(lat, bench.PTC_CHANNELS)
    net.set_weights(w)
    net.attach(force=True)
    fb = lat.to_device(b, F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, dirac.GCR_PTC, tol=1e-10, max_iter=2000, k_max=16, delta=0.1,
                   prec_sloppy=F32, prec_precond=F32)
    assert st["true_rel_resid"] <= 1e-10 and st["precond"] == "ptc"
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    est = _sampled_residual(U.cpu().numpy(), 1.0, kappa, b.cpu().numpy(), x, dims)
    assert est < 1e-9, est
    lat.close()


def test_asqtad_48x144(dirac):
    dims = (48, 48, 48, 144)
    fat, lng = synth.asqtad_links(dims, 3001, 3002, device="cuda")
    psi = synth.staggered_spinor(dims, 3003, device="cuda")
    lat = dirac.Lattice(dims, dirac.ASQTAD, mass=0.01, recon=(18, 12, 12))
    lat.load_gauge(fat, 1)
    lat.load_gauge(lng, 2)
    fat_n, lng_n, psi_n = fat.cpu().numpy(), lng.cpu().numpy(), psi.cpu().numpy()
    del fat, lng
    torch.cuda.empty_cache()
    for prec in (F64, F32, F16):
        for parity in (0, 1):
            src = lat.to_device(psi, prec, 1 - parity)
            out = lat.new_field(prec, parity)
            lat.apply(out, src, parity, prec)
            got = lat.to_natural(out, prec, parity, device="cpu").numpy()
            s = _sample(dims, 256, parity, seed=7 * prec + parity)
            m = ((np.indices(psi_n.shape[:4]).sum(0)) % 2 == 1 - parity)
            ref = staggered.dslash(fat_n, lng_n, dec_spinor(psi_n, prec) * m[..., None], True, s)
            check(_at(got, s), ref, prec, 6, f"48^3x144 asqtad D_{parity} prec={prec}")
            del src, out
    lat.close()


def _staggered_sampled_residual(fat_n, lng_n, mass, shift, b, x, dims, n=256, seed=11):
    """||b - ((M^dagger M)_ee + shift) x|| / ||b|| over a random sample of even sites
    (plus the origin), the oracle evaluating (M^dagger M)_ee = m^2 - 1/4 D_eo D_oe
    (Sec. 3.1, Eq. 3) one site at a time: D x at the odd sites the sample's hops reach
    (1- and 3-hops in every direction), then D of that at the sample."""
    s = _sample(dims, n, parity=0, seed=seed)
    neigh = []
    for mu in range(4):
        for h in (1, -1, 3, -3):
            y = s.copy()
            y[:, mu] = (y[:, mu] + h) % dims[mu]
            neigh.append(y)
    neigh = np.unique(np.concatenate(neigh), axis=0)
    x_e = x * staggered.parity_mask(dims, 0)[..., None]
    dx = staggered.dslash(fat_n, lng_n, x_e, True, neigh)
    Y = np.zeros_like(x)
    Y[neigh[:, 3], neigh[:, 2], neigh[:, 1], neigh[:, 0]] = dx
    ddx = staggered.dslash(fat_n, lng_n, Y, True, s)
    ax = (mass * mass + shift) * _at(x, s) - 0.25 * ddx
    bs = _at(b, s)
    return np.linalg.norm(bs - ax) / np.linalg.norm(bs)


def test_asqtad_solves_48x144_oracle_gated(dirac):
    """The asqtad solves of the benchmark at 48^3x144, m = 0.01: mixed FP64/FP32 CG on
    (M^dagger M)_ee and the 4-shift multi-shift solve (Eq. 4, Sec. 8.2). The library's
    FP64 true residual <= 1e-10 for every system, and the oracle's sampled residual
    agrees (<= 1e-9)."""
    dims, mass = (48, 48, 48, 144), 0.01
    fat, lng = synth.asqtad_links(dims, 3001, 3002, device="cuda")
    src = synth.staggered_spinor(dims, 3003, device="cuda", parity=0)
    lat = dirac.Lattice(dims, dirac.ASQTAD, mass=mass, recon=(18, 12, 12))
    lat.load_gauge(fat, 1)
    lat.load_gauge(lng, 2)
    fat_n, lng_n = fat.cpu().numpy(), lng.cpu().numpy()
    del fat, lng
    torch.cuda.empty_cache()
    b_n = src.cpu().numpy()
    b = lat.to_device(src, F64, 0)
    x = lat.new_field(F64, 0)
    st = lat.solve(x, b, dirac.CG_EVEN_NORMAL, tol=1e-10, max_iter=6000, delta=0.1, prec_sloppy=F32)
    assert st["true_rel_resid"] <= 1e-10
    xn = lat.to_natural(x, F64, 0, device="cpu").numpy()
    est = _staggered_sampled_residual(fat_n, lng_n, mass, 0.0, b_n, xn, dims)
    assert est < 1e-9, est
    shifts = [0.0, 0.0005, 0.005, 0.05]
    xs = [lat.new_field(F64, 0) for _ in shifts]
    r = lat.solve_multishift(xs, b, shifts, dirac.CG_EVEN_NORMAL, tol=1e-10, max_iter=6000,
                             delta=0.1, prec_sloppy=F32)
    for j, (sg, xj) in enumerate(zip(shifts, xs)):
        assert r["refine"][j]["true_rel_resid"] <= 1e-10, (j, r["refine"][j])
        xjn = lat.to_natural(xj, F64, 0, device="cpu").numpy()
        est = _staggered_sampled_residual(fat_n, lng_n, mass, sg, b_n, xjn, dims, seed=20 + j)
        assert est < 1e-9, (j, est)
    lat.close()


def test_learned_preconditioner_adaptive_choice_24x128(dirac):
    """GCR_PTC without forcing the network, on the 24^3x128 workload with a network trained
    on 16^4 at kappa 0.135 and applied unchanged: at kappa 0.124 (where the Schwarz
    preconditioner converges faster per second) the solve ends on Schwarz and takes at most
    a quarter longer than GCR-DD with the same precisions; at kappa 0.1350 (where GCR-DD
    stalls) it ends on the network and converges. Both solutions pass the oracle's sampled
    residual."""
    import bench
    dims = (24, 24, 24, 128)
    plat, pnet, _, _, _ = bench.train_ptc(dirac, synth, torch.device("cuda"), 0.135)
    w = pnet.get_weights()
    plat.close()
    U = synth.wilson_gauge(dims, 0.5, 3, 2001, device="cuda")
    b = synth.wilson_spinor(dims, 2002, device="cuda")
    for kappa, expect in ((0.124, "schwarz"), (0.135, "ptc")):
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, block=(4, 4, 4, 4), mr_steps=6,
                            recon=(18, 12, 12))
        lat.load_gauge(U)
        net = dirac.Ptc(lat, bench.PTC_CHANNELS)
        net.set_weights(w)
        net.attach(force=False)
        fb = lat.to_device(b, F64)
        fx = lat.new_field(F64)
        st = lat.solve(fx, fb, dirac.GCR_PTC, tol=1e-10, max_iter=3000, k_max=16, delta=0.1,
                       prec_sloppy=F16, prec_precond=F16)
        info = {k: st[k] for k in ("iters", "seconds", "precond", "precond_rate", "precond_switches",
                                   "precond_reduction", "true_rel_resid")}
        assert st["true_rel_resid"] <= 1e-10, info
        assert st["precond_rate"][0] != -1 and st["precond_rate"][1] != -1, info  # both were measured
        if kappa == 0.124:
            fy = lat.new_field(F64)
            ref = lat.solve(fy, fb, dirac.GCR_DD, tol=1e-10, max_iter=3000, k_max=16, delta=0.1,
                            prec_sloppy=F16, prec_precond=F16)
            assert st["seconds"] <= 1.25 * ref["seconds"], (info, ref["seconds"])
        else:
            assert st["precond"] == expect, info
        x = lat.to_natural(fx, F64, device="cpu").numpy()
        est = _sampled_residual(U.cpu().numpy(), 1.0, kappa, b.cpu().numpy(), x, dims)
        assert est < 1e-9, est
        net.close()
        lat.close()
