"""Pins of the oracle's parallel-transport convolution network: gauge equivariance,
adjointness of the transports, and finite-difference checks of the analytic weight
gradients (FP64, 4^4). CPU only."""
import numpy as np
import torch

from oracle import ptc
from paper_1109_2935_gb300 import synth


def _fields(dims, seed=3):
    U = synth.wilson_gauge(dims, 0.5, 1, seed).numpy()
    r = synth.wilson_spinor(dims, seed + 1).numpy()
    v = synth.wilson_spinor(dims, seed + 2).numpy()
    return U, r, v


def _rand_w(rng, c_out, c_in, s=0.3):
    return s * (rng.normal(size=(ptc.NPATH, c_out, c_in, 4, 4))
                + 1j * rng.normal(size=(ptc.NPATH, c_out, c_in, 4, 4)))


def test_transport_adjoint_pairs():
    dims = (4, 4, 4, 6)
    U, r, v = _fields(dims)
    for p in range(ptc.NPATH):
        lhs = np.vdot(v, ptc.transport(U, r, p))
        rhs = np.vdot(ptc.transport_adjoint(U, v, p), r)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gauge_equivariance():
    dims = (4, 4, 4, 4)
    U, r, _ = _fields(dims)
    rng = np.random.default_rng(0)
    W1, W2 = _rand_w(rng, 2, 1), _rand_w(rng, 1, 2)
    LX, LY, LZ, LT = dims
    G = synth.haar_su3((LT, LZ, LY, LX), synth._gen(5, "cpu"), "cpu")
    Ut = synth.gauge_transform(torch.from_numpy(U), G).numpy()
    G = G.numpy()
    Gr = np.einsum("...ab,...sb->...sa", G, r)
    lhs, _ = ptc.net_forward(Ut, [W1, W2], Gr)
    rhs = np.einsum("...ab,...sb->...sa", G, ptc.net_forward(U, [W1, W2], r)[0])
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_identity_network():
    dims = (2, 2, 2, 4)
    U, r, _ = _fields(dims)
    k, _ = ptc.net_forward(U, [ptc.identity_weights(2, 1, 2.0), ptc.identity_weights(1, 2, 0.5)], r)
    assert np.max(np.abs(k - r)) < 1e-15


def test_weight_gradient_finite_differences():
    """dL/dconj(W): real part of a perturbation dW changes L by 2 Re <gW, dW>."""
    dims = (4, 4, 4, 4)
    U, r, v = _fields(dims, 11)
    rng = np.random.default_rng(1)
    W1, W2 = _rand_w(rng, 2, 1), _rand_w(rng, 1, 2)
    L, (g1, g2) = ptc.loss_and_grad(U, [W1, W2], r, v)
    eps = 1e-6
    for which, W, g in ((1, W1, g1), (2, W2, g2)):
        for trial in range(4):
            dW = _rand_w(rng, W.shape[1], W.shape[2], 1.0)
            Wp, Wm = W + eps * dW, W - eps * dW
            if which == 1:
                Lp = ptc.loss_and_grad(U, [Wp, W2], r, v)[0]
                Lm = ptc.loss_and_grad(U, [Wm, W2], r, v)[0]
            else:
                Lp = ptc.loss_and_grad(U, [W1, Wp], r, v)[0]
                Lm = ptc.loss_and_grad(U, [W1, Wm], r, v)[0]
            fd = (Lp - Lm) / (2 * eps)
            an = 2 * np.real(np.vdot(g, dW))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, fd, an)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2, so
    every step moves each real parameter by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    W = rng.normal(size=(3, 4)) + 1j * rng.normal(size=(3, 4))
    gW = rng.normal(size=(3, 4)) + 1j * rng.normal(size=(3, 4))
    m = np.zeros_like(W)
    v = np.zeros_like(W)
    lr, eps = 0.01, 1e-8
    cur = W.copy()
    for t in range(1, 6):
        cur, m, v = ptc.adam_step(cur, gW, m, v, t, lr, eps=eps)
        g = 2 * gW
        expect = W - t * lr * (g.real / (np.abs(g.real) + eps) + 1j * g.imag / (np.abs(g.imag) + eps))
        assert np.max(np.abs(cur - expect)) < 1e-12


def test_training_by_adam_reduces_loss():
    """A few Adam steps from random weights on one pair (r = M v) lower the loss."""
    from oracle import wilson
    dims = (4, 4, 4, 4)
    U, _, v = _fields(dims, 21)
    A = wilson.clover(U, 1.0)
    r = wilson.apply_M(U, A, 0.12, v)
    rng = np.random.default_rng(2)
    W1, W2 = _rand_w(rng, 2, 1, 0.05), _rand_w(rng, 1, 2, 0.05)
    m1, v1, m2, v2 = (np.zeros_like(W1), np.zeros_like(W1), np.zeros_like(W2), np.zeros_like(W2))
    L0 = None
    for t in range(1, 16):
        L, (g1, g2) = ptc.loss_and_grad(U, [W1, W2], r, v)
        L0 = L if L0 is None else L0
        W1, m1, v1 = ptc.adam_step(W1, g1, m1, v1, t, 0.02)
        W2, m2, v2 = ptc.adam_step(W2, g2, m2, v2, t, 0.02)
    assert ptc.loss_and_grad(U, [W1, W2], r, v)[0] < 0.7 * L0


def test_three_layer_gradient_finite_differences():
    """1 -> 2 -> 2 -> 1: the middle layer's gradient passes through two adjoint layers."""
    dims = (2, 2, 2, 4)
    U, r, v = _fields(dims, 13)
    rng = np.random.default_rng(6)
    Ws = [_rand_w(rng, 2, 1), _rand_w(rng, 2, 2), _rand_w(rng, 1, 2)]
    L, grads = ptc.loss_and_grad(U, Ws, r, v)
    eps = 1e-6
    for l in range(3):
        dW = _rand_w(rng, Ws[l].shape[1], Ws[l].shape[2], 1.0)
        Wp = [w.copy() for w in Ws]
        Wm = [w.copy() for w in Ws]
        Wp[l] = Wp[l] + eps * dW
        Wm[l] = Wm[l] - eps * dW
        fd = (ptc.loss_and_grad(U, Wp, r, v)[0] - ptc.loss_and_grad(U, Wm, r, v)[0]) / (2 * eps)
        an = 2 * np.real(np.vdot(grads[l], dW))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (l, fd, an)
