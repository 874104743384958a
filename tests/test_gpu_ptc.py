"""GPU parity of the parallel-transport convolution (PTC) network (dirac_ptc_*) against
the FP64 oracle (oracle/ptc.py): forward, loss and weight gradients, one Adam step,
training, and its use as the preconditioner of flexible GCR checked by the oracle's
true residual. FP32 arithmetic: 1e-5 relative."""
import numpy as np
import pytest
import torch

from helpers import F32, F64
from oracle import ptc as optc
from oracle import wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _lattice(dirac, dims, kappa=0.12, recon=(18, 12, 12), seed=5001, sigma=0.5, smooth=3):
    U = synth.wilson_gauge(dims, sigma, smooth, seed)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, recon=recon)
    lat.load_gauge(U)
    return lat, U.numpy()


def _weights(channels, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return [scale * (rng.normal(size=(9, channels[l + 1], channels[l], 4, 4))
                     + 1j * rng.normal(size=(9, channels[l + 1], channels[l], 4, 4)))
            for l in range(len(channels) - 1)]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims,channels,recon", [
    ((4, 4, 4, 6), (1, 2, 1), (18, 18, 12)),
    ((6, 4, 4, 8), (1, 4, 2, 1), (18, 12, 12)),
    ((4, 6, 4, 4), (1, 1), (18, 8, 12)),
    ((4, 4, 4, 4), (1, 4, 4, 1), (18, 12, 12)),
    ((2, 2, 2, 4), (1, 2, 4, 2, 1), (18, 18, 12)),
])
def test_forward_matches_oracle(dirac, dims, channels, recon):
    lat, U = _lattice(dirac, dims, recon=recon)
    net = dirac.Ptc(lat, channels)
    net.tensor_cores(False)
    Ws = _weights(channels, 7)
    net.set_weights(Ws)
    # weights round to FP32 on the device; the oracle uses the same rounded values
    Wr = net.get_weights()
    for w, wr in zip(Ws, Wr):
        assert np.max(np.abs(w - wr)) < 1e-6 * np.max(np.abs(w))
    r = synth.wilson_spinor(dims, 11)
    out = lat.new_field(F32)
    net.apply(out, lat.to_device(r.cuda(), F32))
    got = lat.to_natural(out, F32, device="cpu").numpy()
    rd = lat.to_natural(lat.to_device(r.cuda(), F32), F32, device="cpu").numpy()
    expect, _ = optc.net_forward(U, Wr, rd)
    assert _rel(got, expect) < 1e-5
    site = np.linalg.norm((got - expect).reshape(-1, 12), axis=1) / np.linalg.norm(expect.reshape(-1, 12), axis=1)
    assert np.max(site) < 1e-4


@pytest.mark.parametrize("channels", [(1, 2, 1), (1, 4, 2, 1), (1, 1)])
def test_gradient_matches_oracle(dirac, channels):
    dims = (4, 4, 4, 6)
    lat, U = _lattice(dirac, dims)
    net = dirac.Ptc(lat, channels)
    net.set_weights(_weights(channels, 3, 0.2))
    Wr = net.get_weights()
    r = synth.wilson_spinor(dims, 21)
    v = synth.wilson_spinor(dims, 22)
    fr, fv = lat.to_device(r.cuda(), F32), lat.to_device(v.cuda(), F32)
    loss, grads = net.gradient(fr, fv)
    rd = lat.to_natural(fr, F32, device="cpu").numpy()
    vd = lat.to_natural(fv, F32, device="cpu").numpy()
    L, og = optc.loss_and_grad(U, Wr, rd, vd)
    assert abs(loss - L) < 1e-5 * L
    for g, o in zip(grads, og):
        assert _rel(g, o) < 1e-5


def test_gradient_ragged_lattice_and_antiperiodic_edge(dirac):
    """6^3x10 (sites not a multiple of the block size; 10 t-slices cross the antiperiodic
    edge) with recon-8 FP32 links."""
    dims = (6, 6, 6, 10)
    lat, U = _lattice(dirac, dims, recon=(18, 8, 12))
    net = dirac.Ptc(lat, (1, 2, 1))
    net.set_weights(_weights((1, 2, 1), 5, 0.2))
    Wr = net.get_weights()
    r, v = synth.wilson_spinor(dims, 31), synth.wilson_spinor(dims, 32)
    fr, fv = lat.to_device(r.cuda(), F32), lat.to_device(v.cuda(), F32)
    loss, grads = net.gradient(fr, fv)
    rd = lat.to_natural(fr, F32, device="cpu").numpy()
    vd = lat.to_natural(fv, F32, device="cpu").numpy()
    L, og = optc.loss_and_grad(U, Wr, rd, vd)
    assert abs(loss - L) < 1e-5 * L
    for g, o in zip(grads, og):
        assert _rel(g, o) < 1e-5


def test_gauge_equivariance_full_size(dirac):
    """16^4 (the PTC workload size): K_{U^G}(G r) = G K_U(r) for a random gauge
    transformation G, and the forward pass equals the oracle's."""
    dims = (16, 16, 16, 16)
    U = synth.wilson_gauge(dims, 0.5, 3, 5001)
    LX, LY, LZ, LT = dims
    G = synth.haar_su3((LT, LZ, LY, LX), synth._gen(77, "cpu"), "cpu")
    Ut = synth.gauge_transform(U, G)
    r = synth.wilson_spinor(dims, 5002)
    Gr = torch.einsum("tzyxab,tzyxsb->tzyxsa", G, r)
    Ws = _weights((1, 2, 1), 9, 0.2)
    outs = []
    for links, src in ((U, r), (Ut, Gr)):
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.1355, csw=1.0)
        lat.load_gauge(links)
        net = dirac.Ptc(lat, (1, 2, 1))
        net.tensor_cores(False)
        net.set_weights(Ws)
        out = lat.new_field(F32)
        net.apply(out, lat.to_device(src.cuda(), F32))
        outs.append(lat.to_natural(out, F32, device="cpu").numpy())
        Wr = net.get_weights()
        if links is U:
            rd = lat.to_natural(lat.to_device(r.cuda(), F32), F32, device="cpu").numpy()
            expect, _ = optc.net_forward(U.numpy(), Wr, rd)
            assert _rel(outs[0], expect) < 1e-5
        lat.close()
    Gk = np.einsum("tzyxab,tzyxsb->tzyxsa", G.numpy(), outs[0])
    assert _rel(outs[1], Gk) < 1e-5


@pytest.mark.parametrize("dims,channels,recon", [
    ((4, 4, 4, 6), (1, 2, 1), (18, 18, 12)),
    ((6, 6, 6, 10), (1, 4, 4, 1), (18, 12, 12)),     # 2160 sites: a ragged last tile of 128
    ((4, 6, 4, 4), (1, 1), (18, 8, 12)),
    ((4, 4, 4, 4), (1, 4, 2, 1), (18, 12, 12)),
    ((2, 2, 2, 4), (1, 2, 4, 2, 1), (18, 18, 12)),
    ((8, 8, 8, 8), (1, 4, 4, 1), (18, 12, 12)),
])
def test_tensor_core_forward_matches_oracle(dirac, dims, channels, recon):
    """tcgen05 layers (BF16 operands, FP32 accumulation) against the FP64 oracle with the
    device's FP32 weights: the error is the BF16 rounding of the transported inputs and
    of the weights, ~2^-9 relative per operand."""
    lat, U = _lattice(dirac, dims, recon=recon)
    net = dirac.Ptc(lat, channels)
    net.tensor_cores(True)
    net.set_weights(_weights(channels, 17))
    Wr = net.get_weights()
    r = synth.wilson_spinor(dims, 19)
    fin = lat.to_device(r.cuda(), F32)
    out = lat.new_field(F32)
    net.apply(out, fin)
    got = lat.to_natural(out, F32, device="cpu").numpy()
    rd = lat.to_natural(fin, F32, device="cpu").numpy()
    expect, _ = optc.net_forward(U, Wr, rd)
    assert _rel(got, expect) < 1e-2
    site = np.linalg.norm((got - expect).reshape(-1, 12), axis=1) / np.linalg.norm(expect.reshape(-1, 12), axis=1)
    assert np.max(site) < 5e-2
    # switching back to the FP32 layers gives the 1e-5 result, and back again the same
    # tensor-core result (the weight images are rebuilt only when weights change)
    net.tensor_cores(False)
    out32 = lat.new_field(F32)
    net.apply(out32, fin)
    assert _rel(lat.to_natural(out32, F32, device="cpu").numpy(), expect) < 1e-5
    net.tensor_cores(True)
    out2 = lat.new_field(F32)
    net.apply(out2, fin)
    assert torch.equal(out2, out)


def test_tensor_core_weights_follow_training(dirac):
    """After training steps change the weights, the tensor-core layers use the new ones."""
    dims = (4, 4, 4, 8)
    lat, U = _lattice(dirac, dims)
    net = dirac.Ptc(lat, (1, 2, 1))
    net.tensor_cores(True)
    net.set_weights([w.numpy() for w in synth.ptc_weights((1, 2, 1), 3)])
    r = lat.to_device(synth.wilson_spinor(dims, 23).cuda(), F32)
    before = lat.new_field(F32)
    net.apply(before, r)
    vs = [lat.to_device(synth.wilson_spinor(dims, 30 + i).cuda(), F32) for i in range(4)]
    net.train(vs, steps=5, batch=2, lr=1e-2)
    after = lat.new_field(F32)
    net.apply(after, r)
    Wr = net.get_weights()
    rd = lat.to_natural(r, F32, device="cpu").numpy()
    expect, _ = optc.net_forward(U, Wr, rd)
    assert not torch.equal(before, after)
    assert _rel(lat.to_natural(after, F32, device="cpu").numpy(), expect) < 1e-2


def test_one_adam_step_matches_oracle(dirac):
    dims = (4, 4, 4, 4)
    lat, U = _lattice(dirac, dims)
    net = dirac.Ptc(lat, (1, 2, 1))
    net.set_weights(_weights((1, 2, 1), 13, 0.2))
    W0 = net.get_weights()
    r, v = synth.wilson_spinor(dims, 41), synth.wilson_spinor(dims, 42)
    fr, fv = lat.to_device(r.cuda(), F32), lat.to_device(v.cuda(), F32)
    lr = 1e-3
    losses = net.train([fv], rs=[fr], steps=1, batch=1, lr=lr)
    W1 = net.get_weights()
    rd = lat.to_natural(fr, F32, device="cpu").numpy()
    vd = lat.to_natural(fv, F32, device="cpu").numpy()
    L, og = optc.loss_and_grad(U, W0, rd, vd)
    assert abs(losses[0] - L) < 1e-5 * L
    for w0, w1, g in zip(W0, W1, og):
        z = np.zeros_like(w0)
        expect, _, _ = optc.adam_step(w0, g, z, z, 1, lr)
        # the first Adam step is lr * g / (|g| + eps) per real parameter: compare where
        # |g| is well above the FP32 gradient's rounding
        for part in (np.real, np.imag):
            gp = part(2 * g)
            big = np.abs(gp) > 1e-4 * np.max(np.abs(gp))
            assert np.max(np.abs(part(w1)[big] - part(expect)[big])) < 1e-6


def test_training_lowers_loss_and_reports_history(dirac):
    dims = (8, 8, 8, 8)
    lat, U = _lattice(dirac, dims, kappa=0.12)
    net = dirac.Ptc(lat, (1, 2, 1))
    vs = [lat.to_device(synth.wilson_spinor(dims, 600 + i).cuda(), F32) for i in range(8)]
    # default weights: K = 1, so the first loss is |M v - v|^2 / |v|^2
    l1 = net.train(vs[:1], steps=1, batch=1, lr=1e-12)[0]
    M = _oracle_M(U, 0.12)
    vd = lat.to_natural(vs[0], F32, device="cpu").numpy()
    assert l1 == pytest.approx(np.linalg.norm(M(vd) - vd) ** 2 / np.linalg.norm(vd) ** 2, rel=1e-4)
    net.set_weights([w.numpy() for w in synth.ptc_weights((1, 2, 1), 5)])
    loss = net.train(vs, steps=120, batch=4, lr=2e-2, seed=1)
    assert loss.shape == (120,)
    assert np.all(np.isfinite(loss))
    assert np.mean(loss[-10:]) < 0.2 * loss[0]


def _oracle_M(U, kappa):
    A = wilson.clover(U, 1.0)
    return lambda v: wilson.apply_M(U, A, kappa, v)


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_gcr_ptc_solve_reaches_1e10_and_beats_plain_gcr(dirac, tensor_cores):
    """8^4, kappa 0.124: a trained network inside flexible GCR (forced) converges to 1e-10
    (oracle true residual) in fewer iterations than GCR without a preconditioner, with
    the FP32 layers and with the tensor-core (BF16) layers."""
    dims = (8, 8, 8, 8)
    kappa = 0.124
    lat, U = _lattice(dirac, dims, kappa=kappa)
    net = dirac.Ptc(lat, (1, 2, 1))
    net.tensor_cores(tensor_cores)
    net.set_weights([w.numpy() for w in synth.ptc_weights((1, 2, 1), 6)])
    vs = [lat.to_device(synth.wilson_spinor(dims, 700 + i).cuda(), F32) for i in range(8)]
    net.train(vs, steps=200, batch=4, lr=2e-2, seed=2)
    b = synth.wilson_spinor(dims, 5002)
    fb = lat.to_device(b.cuda(), F64)
    M = _oracle_M(U, kappa)
    res = {}
    for name, alg, force in (("plain", dirac.GCR, None), ("ptc", dirac.GCR_PTC, True)):
        if force is not None:
            net.attach(force=force)
        fx = lat.new_field(F64)
        st = lat.solve(fx, fb, alg, tol=1e-10, max_iter=4000, k_max=16, delta=0.1,
                       prec_sloppy=F32, prec_precond=F32)
        x = lat.to_natural(fx, F64, device="cpu").numpy()
        rr = np.linalg.norm(b.numpy() - M(x)) / np.linalg.norm(b.numpy())
        assert rr <= 1e-10, (name, rr, st)
        res[name] = st
    assert res["ptc"]["precond"] == "ptc"
    assert res["plain"]["precond"] == "none"
    assert res["ptc"]["iters"] < res["plain"]["iters"]


def test_gcr_ptc_falls_back_to_schwarz(dirac):
    """An untrained network (K = 0: zero weights reduce nothing) loses the comparison: the
    solve uses the Schwarz preconditioner and reports both reductions."""
    dims = (8, 8, 8, 8)
    kappa = 0.124
    lat, U = _lattice(dirac, dims, kappa=kappa)
    net = dirac.Ptc(lat, (1, 2, 1))
    net.set_weights([np.zeros(s, dtype=complex) for s in net.shapes])
    net.attach(force=False)
    b = synth.wilson_spinor(dims, 5002)
    fb = lat.to_device(b.cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, dirac.GCR_PTC, tol=1e-10, max_iter=2000, delta=0.1,
                   prec_sloppy=F32, prec_precond=F32)
    assert st["precond"] == "schwarz"
    red_s, red_p = st["precond_reduction"]
    assert red_p == pytest.approx(1.0, abs=1e-6)
    assert red_s < 1.0
    x = lat.to_natural(fx, F64, device="cpu").numpy()
    M = _oracle_M(U, kappa)
    assert np.linalg.norm(b.numpy() - M(x)) / np.linalg.norm(b.numpy()) <= 1e-10


def test_gcr_ptc_without_network_and_bad_arguments(dirac):
    dims = (4, 4, 4, 4)
    lat, _ = _lattice(dirac, dims)
    fb = lat.to_device(synth.wilson_spinor(dims, 1).cuda(), F64)
    fx = lat.new_field(F64)
    st = lat.solve(fx, fb, dirac.GCR_PTC, raise_on_error=False)
    assert st["status"] == "ERR_STATE"
    with pytest.raises(dirac.DiracError):
        dirac.Ptc(lat, (1, 3, 1))
    with pytest.raises(dirac.DiracError):
        dirac.Ptc(lat, (2, 1))
    net = dirac.Ptc(lat, (1, 2, 1))
    with pytest.raises(ValueError):
        net.set_weights([np.zeros((9, 2, 1, 4, 4))])
    other, _ = _lattice(dirac, dims)
    assert dirac.dirac_ptc_attach(other.ctx, net.net, 0) == dirac.ERR_ARG
    # the context frees networks it still holds
    lat.close()
    net.close()


def test_tensor_core_wait_budget_reports_timeout(dirac):
    """Failure detection without a fault: with the MMA-issuing warp stopped (test stall),
    the producer warps' waits run out after their 50 ms budget, the kernel frees its tensor
    memory and returns, the next apply reports ERR_TIMEOUT, and after clearing, the same
    context and network give the normal result again."""
    import time
    dims = (8, 8, 8, 8)
    lat, U = _lattice(dirac, dims)
    net = dirac.Ptc(lat, (1, 2, 1))
    net.set_weights([w.numpy() for w in synth.ptc_weights((1, 2, 1), 8)])
    net.tensor_cores(True)
    fin = lat.to_device(synth.wilson_spinor(dims, 40).cuda(), F32)
    ref = lat.new_field(F32)
    net.apply(ref, fin)
    torch.cuda.synchronize()
    assert dirac.dirac_ptc_test_stall(net.net, 1, 0.05) == dirac.OK
    out = lat.new_field(F32)
    t0 = time.time()
    net.apply(out, fin)           # launches; the kernels give up and return
    torch.cuda.synchronize()
    assert time.time() - t0 < 10.0
    stream = torch.cuda.current_stream().cuda_stream
    assert dirac.dirac_ptc_apply(net.net, out.data_ptr(), fin.data_ptr(), stream) == dirac.ERR_TIMEOUT
    assert dirac.dirac_ptc_test_stall(net.net, 0, 2.0) == dirac.OK
    net.tensor_cores(True)        # clears the recorded error
    again = lat.new_field(F32)
    net.apply(again, fin)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
    assert dirac.dirac_ptc_test_stall(net.net, 1, 0.0) == dirac.ERR_ARG


def test_checkpoint_round_trip(dirac, tmp_path):
    """Weights saved as plain binary + JSON and loaded into a new network on another
    context give the same weights and the same application, bit for bit."""
    dims = (4, 4, 4, 8)
    lat, U = _lattice(dirac, dims)
    net = dirac.Ptc(lat, (1, 2, 2, 1))
    net.set_weights(_weights((1, 2, 2, 1), 31, 0.2))
    prefix = str(tmp_path / "ptc")
    net.save(prefix, meta={"kappa": 0.12, "dims": list(dims)})
    lat2, _ = _lattice(dirac, dims)
    net2 = dirac.Ptc(lat2, (1, 2, 2, 1))
    assert net2.load(prefix) == {"kappa": 0.12, "dims": list(dims)}
    for a, b in zip(net.get_weights(), net2.get_weights()):
        assert np.array_equal(a, b)
    r = synth.wilson_spinor(dims, 32)
    o1, o2 = lat.new_field(F32), lat2.new_field(F32)
    net.apply(o1, lat.to_device(r.cuda(), F32))
    net2.apply(o2, lat2.to_device(r.cuda(), F32))
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    with pytest.raises(ValueError):
        dirac.Ptc(lat2, (1, 2, 1)).load(prefix)
