"""Gauge-equivariant parallel-transport convolution (PTC) network for the oracle
(test infrastructure). Not part of the paper: a learned preconditioner K_theta to
use in place of the Schwarz preconditioner inside flexible GCR (the flexible outer
solver of Sec. 3.2 accepts any, even nonlinear, K).

Layer (channels c_in -> c_out), for spinor fields psi_c(x) (4 spins x 3 colours):
    out_c(x) = sum_{c'} sum_{p in {0, +-x, +-y, +-z, +-t}} W[p, c, c'] [T_p psi_{c'}](x)
    T_0 psi(x)   = psi(x)
    T_+mu psi(x) = U_mu(x) psi(x + mu)            (parallel transport to x)
    T_-mu psi(x) = U_mu(x - mu)^dagger psi(x - mu)
with W[p, c, c'] a complex 4x4 matrix acting on spin only and the fermion boundary
sign on hops across an antiperiodic t boundary. Because W does not touch colour and
T_p transports colour, the layer commutes with gauge transformations. The network is
a chain of such layers from 1 channel back to 1 (e.g. 1 -> 2 -> 1), linear:
K(r) = L_n(... L_1(r)).

Path order: p = 0, then (+mu, -mu) for mu = x, y, z, t, i.e. index 1 + 2 mu + (0|1).
Loss for a pair (r, v): |K(r) - v|^2 / |v|^2. For a real loss of complex weights the
steepest-descent direction is the conjugate (Wirtinger) derivative dL/dconj(W).
"""
import numpy as np

from .lattice import all_coords, at, dims_of, fermion_sign, shift_coords

NPATH = 9


def transport(U, psi, p, antiperiodic_t=True):
    """[T_p psi](x) on the whole lattice; psi natural (T,Z,Y,X,4,3)."""
    if p == 0:
        return psi.copy()
    mu, back = (p - 1) // 2, (p - 1) % 2
    dims = dims_of(psi)
    xs = all_coords(dims)
    if not back:
        ys, w = shift_coords(xs, dims, mu, +1)
        sgn = fermion_sign(w, mu, antiperiodic_t)
        out = sgn[:, None, None] * np.einsum("nab,nsb->nsa", at(U, xs)[:, mu], at(psi, ys))
    else:
        ys, w = shift_coords(xs, dims, mu, -1)
        sgn = fermion_sign(w, mu, antiperiodic_t)
        out = sgn[:, None, None] * np.einsum("nba,nsb->nsa", at(U, ys)[:, mu].conj(), at(psi, ys))
    return out.reshape(psi.shape)


def transport_adjoint(U, phi, p, antiperiodic_t=True):
    """T_p^dagger: the adjoint of T_+mu is T_-mu and vice versa (T_0 is self-adjoint)."""
    if p == 0:
        return phi.copy()
    return transport(U, phi, p + 1 if (p - 1) % 2 == 0 else p - 1, antiperiodic_t)


def spin_apply(W, psi):
    """W (4x4) acting on the spin index of psi (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", W, psi)


def layer_forward(U, W, xs, antiperiodic_t=True):
    """W: (NPATH, c_out, c_in, 4, 4) complex; xs: list of c_in fields. Returns c_out fields."""
    c_out, c_in = W.shape[1], W.shape[2]
    ys = [np.zeros_like(xs[0]) for _ in range(c_out)]
    for p in range(NPATH):
        for ci in range(c_in):
            t = transport(U, xs[ci], p, antiperiodic_t)
            for co in range(c_out):
                ys[co] = ys[co] + spin_apply(W[p, co, ci], t)
    return ys


def layer_backward(U, W, xs, gys, antiperiodic_t=True):
    """Given dL/dconj(y_c) = gys[c], return (dL/dconj(x_c'), dL/dconj(W)).
    y = sum_p W_p T_p x is complex-linear, so dL/dconj(x) = sum_p T_p^dagger W_p^dagger gy
    and dL/dconj(W_p)[s, s'] = sum_{x, colour} gy[x, s, a] conj((T_p x)[x, s', a])."""
    c_out, c_in = W.shape[1], W.shape[2]
    gxs = [np.zeros_like(xs[0]) for _ in range(c_in)]
    gW = np.zeros_like(W)
    for p in range(NPATH):
        for ci in range(c_in):
            t = transport(U, xs[ci], p, antiperiodic_t)
            for co in range(c_out):
                gW[p, co, ci] = np.einsum("nsa,nta->st", gys[co].reshape(-1, 4, 3),
                                           t.conj().reshape(-1, 4, 3))
                gxs[ci] = gxs[ci] + transport_adjoint(
                    U, spin_apply(W[p, co, ci].conj().T, gys[co]), p, antiperiodic_t)
    return gxs, gW


def net_forward(U, Ws, r, antiperiodic_t=True):
    """K(r) for the layers Ws (first takes 1 channel, last gives 1); also returns every
    layer's output (activations[l] = output of layer l, activations[-1] = K(r))."""
    acts = []
    h = [r]
    for W in Ws:
        h = layer_forward(U, W, h, antiperiodic_t)
        acts.append(h)
    return h[0], acts


def loss_and_grad(U, Ws, r, v, antiperiodic_t=True):
    """L = |K(r) - v|^2 / |v|^2 and its conjugate derivatives w.r.t. every layer's W."""
    k, acts = net_forward(U, Ws, r, antiperiodic_t)
    vv = float(np.vdot(v, v).real)
    d = k - v
    L = float(np.vdot(d, d).real) / vv
    g = [d / vv]  # dL/dconj(K(r))
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        xin = [r] if l == 0 else acts[l - 1]
        g, grads[l] = layer_backward(U, Ws[l], xin, g, antiperiodic_t)
    return L, grads


def identity_weights(c_out, c_in, scale=1.0):
    """Weights that pass channel 0 through unchanged times `scale` (path 0 only)."""
    W = np.zeros((NPATH, c_out, c_in, 4, 4), dtype=np.complex128)
    W[0, 0, 0] = scale * np.eye(4)
    return W


def adam_step(W, gW, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015, Algorithm 1) on theta = (Re W, Im W), whose
    gradient is 2 dL/dconj(W) = 2 gW, taken separately on the real and imaginary parts.
    m, v: the moment estimates as complex arrays holding the real-part moments in .real
    and the imaginary-part moments in .imag; t: the step number after this one (>= 1).
    Returns the new (W, m, v)."""
    g = 2 * gW
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * (g.real ** 2 + 1j * g.imag ** 2)
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    step = mh.real / (np.sqrt(vh.real) + eps) + 1j * (mh.imag / (np.sqrt(vh.imag) + eps))
    return W - lr * step, m, v
