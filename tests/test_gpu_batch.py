"""Batched Wilson-clover operator: many right-hand sides per lattice and several
lattices of different sizes per launch (persistent kernel, autotuned tile shape,
CUDA-graph replay). Each output must be bitwise identical to the single-RHS kernel
(same per-site code) and match the FP64 oracle."""
import numpy as np
import pytest
import torch

from helpers import F16, F32, F64, check, dec_clover_hat, dec_links, dec_spinor
from oracle import wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _lattice(dirac, dims, kappa, seed, recon=12):
    U = synth.wilson_gauge(dims, 0.5, 2, seed)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, recon=(18, recon, recon))
    lat.load_gauge(U)
    return lat, U


def _rhs(lat, prec, n, seed):
    fb = lat.field_bytes(prec)
    buf = torch.zeros(n * fb, dtype=torch.uint8, device="cuda")
    nat = []
    for r in range(n):
        psi = synth.wilson_spinor(lat.dims, seed + r)
        lat.import_spinor(buf[r * fb:(r + 1) * fb], prec, -1, psi.cuda())
        nat.append(psi)
    return buf, nat


@pytest.mark.parametrize("prec", [F64, F32, F16])
@pytest.mark.parametrize("nrhs", [1, 5, 12, 17])
def test_apply_multi_equals_single(dirac, prec, nrhs):
    dims = (6, 6, 6, 10)
    lat, U = _lattice(dirac, dims, 0.13, 11)
    fb = lat.field_bytes(prec)
    xin, nat = _rhs(lat, prec, nrhs, 100)
    yout = torch.zeros_like(xin)
    lat.apply_multi(yout, xin, nrhs, prec)
    for r in range(nrhs):
        ref = lat.new_field(prec)
        lat.apply(ref, xin[r * fb:(r + 1) * fb], dirac.PARITY_FULL, prec)
        assert torch.equal(yout[r * fb:(r + 1) * fb], ref), r
    # one right-hand side against the oracle
    Un = U.numpy()
    Ahat = np.eye(12) + 2 * 0.13 * wilson.clover(Un, 1.0)
    Ad = (dec_clover_hat(Ahat, prec) - np.eye(12)) / (2 * 0.13)
    got = lat.to_natural(yout[(nrhs - 1) * fb:nrhs * fb], prec, device="cpu").numpy()
    ref = wilson.apply_M(dec_links(Un, prec), Ad, 0.13, dec_spinor(nat[-1].numpy(), prec))
    check(got, ref, prec, 24, "multi-RHS")


@pytest.mark.parametrize("prec", [F32, F16])
def test_batch_uneven_lattices_graph(dirac, prec):
    specs = [((4, 4, 4, 4), 0.130, 3), ((6, 6, 6, 10), 0.133, 5), ((8, 8, 4, 4), 0.136, 2)]
    lats, ins, outs, nats = [], [], [], []
    for k, (dims, kappa, n) in enumerate(specs):
        lat, U = _lattice(dirac, dims, kappa, 20 + k)
        xin, nat = _rhs(lat, prec, n, 200 + 10 * k)
        lats.append(lat)
        ins.append(xin)
        outs.append(torch.zeros_like(xin))
        nats.append(nat)
    b = dirac.Batch(lats, outs, ins, [s[2] for s in specs], prec)
    info = b.info()
    assert info["rhs_per_cta"] in (1, 2, 4, 8, 16) and info["grid"] >= 1
    for k in range(len(outs)):
        outs[k].zero_()
    b.apply()
    torch.cuda.synchronize()
    ref_outs = []
    for lat, xin, out, (dims, kappa, n) in zip(lats, ins, outs, specs):
        fb = lat.field_bytes(prec)
        refs = []
        for r in range(n):
            ref = lat.new_field(prec)
            lat.apply(ref, xin[r * fb:(r + 1) * fb], dirac.PARITY_FULL, prec)
            assert torch.equal(out[r * fb:(r + 1) * fb], ref), (dims, r)
            refs.append(ref)
        ref_outs.append(refs)
    # graph replay of 3 batched launches gives the same outputs (M in, three times)
    for k in range(len(outs)):
        outs[k].zero_()
    b.capture(3)
    b.apply()
    torch.cuda.synchronize()
    for lat, out, refs in zip(lats, outs, ref_outs):
        fb = lat.field_bytes(prec)
        for r, ref in enumerate(refs):
            assert torch.equal(out[r * fb:(r + 1) * fb], ref)
    b.close()


def test_batch_argument_checks(dirac):
    l1, _ = _lattice(dirac, (4, 4, 4, 4), 0.13, 1, recon=12)
    l2, _ = _lattice(dirac, (4, 4, 4, 6), 0.13, 2, recon=18)
    x1, _ = _rhs(l1, F32, 2, 5)
    x2, _ = _rhs(l2, F32, 2, 7)
    with pytest.raises(dirac.DiracError):
        dirac.Batch([l1, l2], [torch.zeros_like(x1), torch.zeros_like(x2)], [x1, x2], [2, 2], F32)
    # in and out overlapping
    assert dirac.dirac_apply_multi(l1.ctx, x1.data_ptr(), x1.data_ptr(), 2, F32, None) == dirac.ERR_ARG
