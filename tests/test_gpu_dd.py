"""Domain decomposition (Sec. 6) emulated on one GPU (dirac_dd_*): the Wilson-clover
operator over P virtual ranks (t-slabs, or a grid cutting any of the four dimensions) with spin-projected face exchange into ghost zones must
equal the single-domain operator bit for bit in FP64 and FP32, for every link format, M
and M^dagger, with and without the clover term, and at the antiperiodic t edge. With
FP16 storage the two kernels contract the decode product (half x site norm) into
different fused multiply-adds, so the FP32 arithmetic differs by rounding and the
re-encoded outputs agree to one FP16 unit in the last place per site."""
import numpy as np
import pytest
import torch

from helpers import F16, F32, F64
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _same(lat, out, ref, prec):
    if prec != F16:
        return torch.equal(out, ref)
    a = lat.to_natural(out, prec, device="cpu").numpy().reshape(-1, 12)
    b = lat.to_natural(ref, prec, device="cpu").numpy().reshape(-1, 12)
    site = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    return bool(np.max(site) <= 2.0 ** -10)


def _setup(dirac, dims, csw=1.0, recon=(18, 12, 12), apbc=True, seed=4001):
    U = synth.wilson_gauge(dims, 0.5, 1, seed)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.13, csw=csw, recon=recon, t_antiperiodic=apbc)
    lat.load_gauge(U)
    return lat


@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("nranks", [1, 2, 4, 8])
@pytest.mark.parametrize("dagger", [False, True])
def test_dd_equals_single_domain_bitwise(dirac, prec, nranks, dagger):
    dims = (6, 4, 8, 16)
    lat = _setup(dirac, dims)
    src = lat.to_device(synth.wilson_spinor(dims, 7).cuda(), prec)
    ref = lat.new_field(prec)
    if dagger:
        lat.apply_dagger(ref, src, prec=prec)
    else:
        lat.apply(ref, src, prec=prec)
    dd = dirac.DomainDecomposition(lat, nranks, prec)
    assert dd.info()["local_dims"] == (6, 4, 8, 16 // nranks)
    out = torch.zeros_like(ref)
    dd.scatter(src)
    dd.apply(dagger=dagger)
    dd.gather(out)
    torch.cuda.synchronize()
    assert _same(lat, out, ref, prec)
    dd.close()


@pytest.mark.parametrize("recon", [(18, 18, 18), (18, 8, 8)])
@pytest.mark.parametrize("csw,apbc", [(0.0, True), (1.0, False)])
def test_dd_link_formats_no_clover_periodic(dirac, recon, csw, apbc):
    dims = (4, 6, 4, 12)
    lat = _setup(dirac, dims, csw=csw, recon=recon, apbc=apbc)
    for prec in (F64, F32, F16):
        src = lat.to_device(synth.wilson_spinor(dims, 9).cuda(), prec)
        ref = lat.new_field(prec)
        lat.apply(ref, src, prec=prec)
        dd = dirac.DomainDecomposition(lat, 3 if dims[3] % 6 == 0 else 2, prec)
        out = torch.zeros_like(ref)
        dd.scatter(src)
        dd.apply()
        dd.gather(out)
        torch.cuda.synchronize()
        assert _same(lat, out, ref, prec), prec
        dd.close()


def test_dd_repeated_applications_and_bad_partition(dirac):
    """Applying twice in a row (send buffers reused) still matches; an odd local extent
    is rejected."""
    dims = (4, 4, 4, 8)
    lat = _setup(dirac, dims)
    src = lat.to_device(synth.wilson_spinor(dims, 3).cuda(), F32)
    ref1, ref2 = lat.new_field(F32), lat.new_field(F32)
    lat.apply(ref1, src, prec=F32)
    lat.apply(ref2, ref1, prec=F32)
    dd = dirac.DomainDecomposition(lat, 2, F32)
    mid, out = torch.zeros_like(ref1), torch.zeros_like(ref1)
    dd.scatter(src)
    dd.apply()
    dd.gather(mid)
    dd.scatter(mid)
    dd.apply()
    dd.gather(out)
    torch.cuda.synchronize()
    assert torch.equal(mid, ref1) and torch.equal(out, ref2)
    dd.close()
    with pytest.raises(dirac.DiracError):
        dirac.DomainDecomposition(lat, 8, F32)   # LT / 8 = 1 slice
    with pytest.raises(dirac.DiracError):
        dirac.DomainDecomposition(lat, 3, F32)   # 8 / 3 not an integer


@pytest.mark.parametrize("prec,nranks", [(F32, 2), (F32, 8), (F64, 4)])
def test_dd_full_size(dirac, prec, nranks):
    """24^3x128 (the benchmark lattice): the decomposed operator equals the single-domain
    one bit for bit."""
    dims = (24, 24, 24, 128)
    U = synth.wilson_gauge(dims, 0.5, 3, 2001, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.135, csw=1.0, recon=(18, 12, 12))
    lat.load_gauge(U)
    src = lat.to_device(synth.wilson_spinor(dims, 2002, device="cuda"), prec)
    ref = lat.new_field(prec)
    lat.apply(ref, src, prec=prec)
    dd = dirac.DomainDecomposition(lat, nranks, prec)
    out = torch.zeros_like(ref)
    dd.scatter(src)
    dd.apply()
    dd.gather(out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    dd.close()
    lat.close()


GRIDS = [(2, 1, 1, 1), (1, 2, 1, 1), (1, 1, 2, 1), (2, 2, 1, 2), (2, 2, 2, 2), (4, 1, 2, 1)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("dagger", [False, True])
def test_dd_grid_equals_single_domain(dirac, grid, prec, dagger):
    """Cuts in x, y, z and t (alone and together, local extents down to 2): ghost zones in
    every cut dimension, bit-identical to the single-domain operator in FP64 / FP32."""
    dims = (8, 4, 8, 8)
    lat = _setup(dirac, dims)
    src = lat.to_device(synth.wilson_spinor(dims, 11).cuda(), prec)
    ref = lat.new_field(prec)
    if dagger:
        lat.apply_dagger(ref, src, prec=prec)
    else:
        lat.apply(ref, src, prec=prec)
    dd = dirac.DomainDecomposition(lat, grid, prec)
    info = dd.info()
    assert info["local_dims"] == tuple(d // g for d, g in zip(dims, grid))
    fsite = 96 if prec == F64 else 48
    vloc = np.prod(info["local_dims"])
    assert info["face_bytes"] == sum(2 * vloc // info["local_dims"][m] * fsite for m in range(4) if grid[m] > 1)
    out = torch.zeros_like(ref)
    dd.scatter(src)
    dd.apply(dagger=dagger)
    dd.gather(out)
    torch.cuda.synchronize()
    assert _same(lat, out, ref, prec)
    dd.close()


@pytest.mark.parametrize("recon", [(18, 18, 18), (18, 8, 8)])
def test_dd_grid_link_formats_periodic_no_clover(dirac, recon):
    dims = (4, 4, 8, 4)
    lat = _setup(dirac, dims, csw=0.0, recon=recon, apbc=False)
    for prec in (F64, F32, F16):
        src = lat.to_device(synth.wilson_spinor(dims, 13).cuda(), prec)
        ref = lat.new_field(prec)
        lat.apply(ref, src, prec=prec)
        dd = dirac.DomainDecomposition(lat, (2, 2, 2, 2), prec)
        out = torch.zeros_like(ref)
        dd.scatter(src)
        dd.apply()
        dd.gather(out)
        torch.cuda.synchronize()
        assert _same(lat, out, ref, prec), prec
        dd.close()


def test_dd_bad_grids(dirac):
    lat = _setup(dirac, (4, 4, 4, 8))
    for grid in ((3, 1, 1, 1), (4, 1, 1, 1), (1, 1, 1, 0), (2, 2, 2, 8)):
        with pytest.raises(dirac.DiracError):
            dirac.DomainDecomposition(lat, grid, F32)


def test_dd_grid_full_size(dirac):
    """24^3x128 cut 2 x 2 x 2 x 2 (16 ranks, every dimension): bit for bit in FP32."""
    dims = (24, 24, 24, 128)
    U = synth.wilson_gauge(dims, 0.5, 3, 2001, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.135, csw=1.0, recon=(18, 12, 12))
    lat.load_gauge(U)
    src = lat.to_device(synth.wilson_spinor(dims, 2002, device="cuda"), F32)
    ref = lat.new_field(F32)
    lat.apply(ref, src, prec=F32)
    dd = dirac.DomainDecomposition(lat, (2, 2, 2, 2), F32)
    out = torch.zeros_like(ref)
    dd.scatter(src)
    dd.apply()
    dd.gather(out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    dd.close()
    lat.close()
