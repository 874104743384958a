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
    if prec == F16:
        b.set_tensor_cores(False)  # the CUDA-core kernel: bitwise equal to single-RHS
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


def test_batch_at_the_configured_sizes(dirac):
    """The benchmark's batched workload: 16^3x32, 24^3x64 and 32^3x64 with 12 right-hand
    sides each (kappa 0.130 / 0.133 / 0.136, FP16 storage) in one persistent launch: every
    output equals the single-RHS kernel's bit for bit, and one right-hand side of the
    largest lattice matches the oracle on sampled sites."""
    from oracle.lattice import all_coords
    specs = [((16, 16, 16, 32), 0.130, 4001), ((24, 24, 24, 64), 0.133, 4003), ((32, 32, 32, 64), 0.136, 4005)]
    nrhs, prec = 12, F16
    lats, ins, outs, Us = [], [], [], []
    for dims, kappa, seed in specs:
        U = synth.wilson_gauge(dims, 0.5, 3, seed, device="cuda")
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, recon=(18, 12, 12))
        lat.load_gauge(U)
        fb = lat.field_bytes(prec)
        xin = torch.zeros(nrhs * fb, dtype=torch.uint8, device="cuda")
        for r in range(nrhs):
            lat.import_spinor(xin[r * fb:(r + 1) * fb], prec, -1, synth.wilson_spinor(dims, seed + 1 + 17 * r,
                                                                                        device="cuda"))
        lats.append(lat)
        ins.append(xin)
        outs.append(torch.zeros_like(xin))
        Us.append(U)
    b = dirac.Batch(lats, outs, ins, [nrhs] * 3, prec)
    b.set_tensor_cores(False)
    b.apply()
    torch.cuda.synchronize()
    for lat, xin, out in zip(lats, ins, outs):
        fb = lat.field_bytes(prec)
        for r in range(nrhs):
            ref = lat.new_field(prec)
            lat.apply(ref, xin[r * fb:(r + 1) * fb], dirac.PARITY_FULL, prec)
            assert torch.equal(out[r * fb:(r + 1) * fb], ref), (lat.dims, r)
    # the tensor-core kernel on the same plan: every output site within the FP16 per-site
    # bound of the CUDA-core result (checked on the first and last right-hand side)
    cc = [o.clone() for o in outs]
    b.set_tensor_cores(True)
    for o in outs:
        o.zero_()
    b.apply()
    torch.cuda.synchronize()
    for lat, o, c in zip(lats, outs, cc):
        fb = lat.field_bytes(prec)
        for r in (0, nrhs - 1):
            got = lat.to_natural(o[r * fb:(r + 1) * fb], prec, device="cpu").numpy()
            ref = lat.to_natural(c[r * fb:(r + 1) * fb], prec, device="cpu").numpy()
            check(got, ref, F16, 24, f"tensor-core vs CUDA-core {lat.dims} rhs {r}")
    # the oracle on sampled sites of the last right-hand side of 32^3x64
    lat, xin, out, U = lats[-1], ins[-1], outs[-1], Us[-1]
    dims, kappa = specs[-1][0], specs[-1][1]
    fb = lat.field_bytes(prec)
    psi = lat.to_natural(xin[(nrhs - 1) * fb:], prec, device="cpu").numpy()   # decoded FP16 input
    got = lat.to_natural(out[(nrhs - 1) * fb:], prec, device="cpu").numpy()
    rng = np.random.default_rng(1)
    c = all_coords(dims)
    s = c[rng.choice(len(c), 256, replace=False)]
    ref = wilson.apply_M_sites(dec_links(U.cpu().numpy(), prec), 1.0, kappa, psi, s, True, False,
                               Ahat_codec=lambda A: dec_clover_hat(A, prec))
    check(got[s[:, 3], s[:, 2], s[:, 1], s[:, 0]], ref, prec, 24, "batched 32^3x64 sampled")
