"""Tensor-core multi-right-hand-side Wilson-clover operator (FP16 storage): per site
the link-times-spinor products of all right-hand sides as one dense contraction (Eq. 2,
rows = right-hand sides, K = spin-projected hops x colours), the clover blocks as one
more k-tile. Every right-hand side must match the FP64 oracle within the FP16 per-site
bound, with the oracle given the decoded FP16 inputs, links and clover."""
import numpy as np
import pytest
import torch

from helpers import F16, check, dec_clover_hat, dec_links
from oracle import wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(dirac, specs, recon=12, csw=1.0, point=False):
    lats, ins, outs, refs = [], [], [], []
    for k, (dims, kappa, n) in enumerate(specs):
        U = synth.wilson_gauge(dims, 0.5, 2, 30 + k)
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=csw, recon=(18, recon, recon))
        lat.load_gauge(U)
        fb = lat.field_bytes(F16)
        xin = torch.zeros(n * fb, dtype=torch.uint8, device="cuda")
        Un = U.numpy()
        A = wilson.clover(Un, csw) if csw else None
        Ahat = np.eye(12) + 2 * kappa * A if csw else None
        Ad = (dec_clover_hat(Ahat, F16) - np.eye(12)) / (2 * kappa) if csw else None
        rr = []
        for r in range(n):
            psi = synth.wilson_spinor(dims, 300 + 13 * k + r)
            if point and r % 2 == 0:
                # a point source: one non-zero site, so most rows have zero norms
                keep = torch.zeros_like(psi)
                keep[0, 0, 0, r % dims[0]] = psi[0, 0, 0, r % dims[0]]
                psi = keep
            lat.import_spinor(xin[r * fb:(r + 1) * fb], F16, -1, psi.cuda())
            dec = lat.to_natural(xin[r * fb:(r + 1) * fb], F16, device="cpu").numpy()
            rr.append(wilson.apply_M(dec_links(Un, F16), Ad, kappa, dec))
        lats.append(lat)
        ins.append(xin)
        outs.append(torch.zeros_like(xin))
        refs.append(rr)
    return lats, ins, outs, refs


def _check_all(lats, outs, refs, what):
    for lat, out, rr in zip(lats, outs, refs):
        fb = lat.field_bytes(F16)
        for r, ref in enumerate(rr):
            got = lat.to_natural(out[r * fb:(r + 1) * fb], F16, device="cpu").numpy()
            if not np.any(ref):
                assert not np.any(got), (what, lat.dims, r)
                continue
            check(got, ref, F16, 24, f"{what} {lat.dims} rhs {r}")


@pytest.mark.parametrize("recon", [12, 18])
@pytest.mark.parametrize("nrhs", [1, 5, 12, 16, 17])
def test_tensor_core_batch_matches_oracle(dirac, recon, nrhs):
    specs = [((4, 4, 4, 4), 0.130, nrhs), ((6, 6, 6, 10), 0.133, max(1, nrhs - 3)), ((2, 2, 2, 2), 0.125, 3)]
    lats, ins, outs, refs = _setup(dirac, specs, recon)
    b = dirac.Batch(lats, outs, ins, [s[2] for s in specs], F16)
    b.set_tensor_cores(True)
    assert b.kernel_info()["tensor_cores"]
    b.apply()
    torch.cuda.synchronize()
    _check_all(lats, outs, refs, f"tensor cores recon {recon}")
    # replayed from a CUDA graph: the same outputs
    first = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    b.capture(2)
    b.apply()
    torch.cuda.synchronize()
    for o, f in zip(outs, first):
        assert torch.equal(o, f)
    b.close()


def test_tensor_core_no_clover_and_point_sources(dirac):
    """c_sw = 0 (Ahat = 1) and point sources (rows whose neighbours are all zero: the row
    scale is 0 and the output must be exactly zero there)."""
    specs = [((4, 4, 4, 6), 0.12, 6), ((4, 4, 2, 4), 0.12, 4)]
    lats, ins, outs, refs = _setup(dirac, specs, 12, csw=0.0, point=True)
    b = dirac.Batch(lats, outs, ins, [s[2] for s in specs], F16)
    b.set_tensor_cores(True)
    b.apply()
    torch.cuda.synchronize()
    _check_all(lats, outs, refs, "tensor cores, no clover, point sources")
    b.close()


def test_tensor_core_unsupported_for_fp32(dirac):
    specs = [((4, 4, 4, 4), 0.13, 2)]
    U = synth.wilson_gauge((4, 4, 4, 4), 0.5, 1, 3)
    lat = dirac.Lattice((4, 4, 4, 4), dirac.WILSON_CLOVER, kappa=0.13, csw=1.0)
    lat.load_gauge(U)
    fb = lat.field_bytes(dirac.F32)
    x = torch.zeros(2 * fb, dtype=torch.uint8, device="cuda")
    b = dirac.Batch([lat], [torch.zeros_like(x)], [x], [2], dirac.F32)
    assert not b.kernel_info()["tensor_cores"] and b.kernel_info()["tensor_core_ms"] < 0
    with pytest.raises(dirac.DiracError):
        b.set_tensor_cores(True)
    b.close()
