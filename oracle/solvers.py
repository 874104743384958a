"""Krylov solvers and the additive Schwarz preconditioner for the oracle
(test infrastructure; Sec. 3, Sec. 8.1, Algorithm 1). All arithmetic is float64 /
complex128 on natural-layout numpy arrays. Operators are passed as callables.

Inner product: (a, b) = sum conj(a_i) b_i (conjugate-linear in the first slot).
"""
import numpy as np

from . import wilson
from .lattice import all_coords


def dot(a, b):
    return np.vdot(a, b)


def norm2(a):
    return float(np.vdot(a, a).real)


# ---------------------------------------------------------------------------
# Additive Schwarz with minimal-residual block solves (Sec. 3.2, Sec. 8.1)
# ---------------------------------------------------------------------------

def schwarz_mr(U, A, kappa, b, block, n_steps, antiperiodic_t=True):
    """Non-overlapping additive Schwarz preconditioner K b (Sec. 3.2: equal to block
    Jacobi). On every block the Wilson-clover operator restricted to the block, with
    Dirichlet (zero) boundary conditions, is solved approximately by ``n_steps`` steps
    of minimal residual (Sec. 8.1) starting from x = 0:
        p = M_B r;  alpha = (p, r) / (p, p);  x += alpha r;  r -= alpha p.
    The inner products are taken over each block separately (block-local reductions,
    Sec. 8.1). A block whose (p, p) vanishes takes alpha = 0."""
    dims = wilson.dims_of(b)
    coords = all_coords(dims)
    bid = wilson.block_id(coords, block)
    _, inv = np.unique(bid, return_inverse=True)
    nb = inv.max() + 1
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(n_steps):
        p = wilson.apply_M(U, A, kappa, r, antiperiodic_t, block=block)
        pf, rf = p.reshape(len(coords), 12), r.reshape(len(coords), 12)
        pr = np.bincount(inv, weights=np.sum(pf.conj() * rf, axis=1).real, minlength=nb) \
            + 1j * np.bincount(inv, weights=np.sum(pf.conj() * rf, axis=1).imag, minlength=nb)
        pp = np.bincount(inv, weights=np.sum(np.abs(pf) ** 2, axis=1), minlength=nb)
        alpha = np.where(pp > 0, pr / np.where(pp > 0, pp, 1.0), 0.0)
        a = alpha[inv].reshape(r.shape[:4] + (1, 1))
        x = x + a * r
        r = r - a * p
    return x


# ---------------------------------------------------------------------------
# Conjugate gradients (Sec. 3.1, Hestenes-Stiefel) on a Hermitian positive operator
# ---------------------------------------------------------------------------

def cg(A, b, tol, max_iter, x0=None):
    """Textbook CG for A x = b with A Hermitian positive definite. Stops when
    ||b - A x|| <= tol ||b|| (iterated residual) or after max_iter iterations.
    Returns (x, info) with info["iters"] and the first iteration's scalars."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x)
    p = r.copy()
    rr = norm2(r)
    bb = norm2(b)
    info = {"iters": 0, "alpha0": None, "beta0": None}
    for k in range(max_iter):
        if rr <= tol * tol * bb:
            break
        Ap = A(p)
        alpha = rr / dot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = norm2(r)
        beta = rr_new / rr
        if k == 0:
            info["alpha0"], info["beta0"] = alpha, beta
        p = r + beta * p
        rr = rr_new
        info["iters"] = k + 1
    return x, info


# ---------------------------------------------------------------------------
# BiCGstab (Sec. 3.1, van der Vorst 1992)
# ---------------------------------------------------------------------------

def bicgstab(A, b, tol, max_iter, x0=None):
    """Textbook BiCGstab for a general non-Hermitian A; shadow residual = r_0.
    Stops when the iterated residual satisfies ||r|| <= tol ||b||."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x)
    rt = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    bb = norm2(b)
    info = {"iters": 0, "alpha0": None, "omega0": None}
    for k in range(max_iter):
        if norm2(r) <= tol * tol * bb:
            break
        rho_new = dot(rt, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho_new / dot(rt, v)
        s = r - alpha * v
        t = A(s)
        omega = dot(t, s) / dot(t, t).real
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        if k == 0:
            info["alpha0"], info["omega0"] = alpha, omega
        info["iters"] = k + 1
    return x, info


# ---------------------------------------------------------------------------
# GCR with a (possibly nonlinear) right preconditioner: Algorithm 1
# ---------------------------------------------------------------------------

def gcr(M, K, b, tol, max_iter, k_max, delta, x0=None):
    """Flexible GCR of Algorithm 1, all in float64.

    Reading of the printed algorithm: the orthogonalisation is modified Gram-Schmidt;
    "z_k = z_k / gamma_k" normalises the low-precision z_k; the restart residual is
    r_0 = b - M x (the system matrix); the tolerances are relative to ||b||; a
    cycle restarts when k = k_max, when ||r_k|| / ||r_0|| < delta (delta = 0 turns
    this test off) or when ||r_k|| < tol ||b||. The back-substitution solves
        gamma_l chi_l + sum_{i>l} beta_{l,i} chi_i = alpha_l   for l = k-1 ... 0."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.sqrt(norm2(b))
    r0 = b - M(x)
    rhat = r0.copy()
    r0norm = np.sqrt(norm2(r0))
    P, Z = [], []
    beta = np.zeros((k_max, k_max), dtype=np.complex128)
    gamma = np.zeros(k_max)
    alpha = np.zeros(k_max, dtype=np.complex128)
    info = {"iters": 0, "restarts": 0, "gamma0": None, "alpha0": None}
    it = 0
    k = 0
    while r0norm > tol * bnorm and it < max_iter:
        p = K(rhat)
        z = M(p)
        for i in range(k):
            beta[i, k] = dot(Z[i], z)
            z = z - beta[i, k] * Z[i]
        gamma[k] = np.sqrt(norm2(z))
        z = z / gamma[k]
        alpha[k] = dot(z, rhat)
        rhat = rhat - alpha[k] * z
        P.append(p)
        Z.append(z)
        if info["gamma0"] is None:
            info["gamma0"], info["alpha0"] = gamma[0], alpha[0]
        k += 1
        it += 1
        rnorm = np.sqrt(norm2(rhat))
        if k == k_max or rnorm / r0norm < delta or rnorm < tol * bnorm or it >= max_iter:
            chi = np.zeros(k, dtype=np.complex128)
            for l in range(k - 1, -1, -1):
                s = alpha[l] - sum(beta[l, i] * chi[i] for i in range(l + 1, k))
                chi[l] = s / gamma[l]
            for i in range(k):
                x = x + chi[i] * P[i]
            r0 = b - M(x)
            rhat = r0.copy()
            r0norm = np.sqrt(norm2(r0))
            P, Z = [], []
            k = 0
            info["restarts"] += 1
    info["iters"] = it
    return x, info


def true_residual(M, x, b):
    """||b - M x|| / ||b|| in float64."""
    return float(np.sqrt(norm2(b - M(x)) / norm2(b)))


# ---------------------------------------------------------------------------
# Multi-shift CG (Sec. 3.1, Eq. 4; Sec. 8.2)
# ---------------------------------------------------------------------------

def multishift_cg(A, b, shifts, tol, max_iter):
    """Solve (A + sigma_i) x_i = b for every shift with one Krylov space (Eq. 4), A
    Hermitian positive definite, all sigma_i >= 0.

    The base system is the smallest shift sigma_0 (the least well conditioned one),
    solved by plain CG with A' = A + sigma_0. Its residuals r_k and the residuals of a
    shifted system A' + s (s = sigma_i - sigma_0) are collinear, r^i_k = zeta_k r_k,
    because both lie in the same Krylov space and are orthogonal to it. Writing the
    CG three-term recurrence of both systems and equating coefficients gives
        zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1}
                     / (a_{k-1} zeta_{k-1} (1 + s a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k)),
        a^i_k = a_k zeta_{k+1} / zeta_k,     b^i_k = b_k (zeta_{k+1} / zeta_k)^2,
        x^i += a^i_k p^i_k,   p^i_{k+1} = zeta_{k+1} r_{k+1} + b^i_k p^i_k,
    with zeta_{-1} = zeta_0 = 1, a_{-1} = 1, b_{-1} = 0 and p^i_0 = b.
    A shifted system whose residual ||zeta^i r|| <= tol ||b|| is converged and is no
    longer updated (its zeta would underflow). Stops when the base system converges.
    Returns (list of x_i in the order of `shifts`, info)."""
    shifts = list(shifts)
    order = sorted(range(len(shifts)), key=lambda i: shifts[i])
    s0 = shifts[order[0]]
    n = len(shifts)
    x = [np.zeros_like(b) for _ in range(n)]
    p = [b.copy() for _ in range(n)]
    r = b.copy()
    rr = norm2(r)
    bb = norm2(b)
    zeta = np.ones(n)
    zeta_prev = np.ones(n)
    a_prev, b_prev = 1.0, 0.0
    info = {"iters": 0}
    active = [True] * n
    for k in range(max_iter):
        for i in range(n):
            if active[i] and zeta[i] ** 2 * rr <= tol * tol * bb:
                active[i] = False
        if not any(active):
            break
        i0 = order[0]
        Ap = A(p[i0]) + s0 * p[i0]
        a = rr / dot(p[i0], Ap).real
        r = r - a * Ap
        rr_new = norm2(r)
        bk = rr_new / rr
        for i in range(n):
            if not active[i]:
                continue
            s = shifts[i] - s0
            if i == i0:
                z_next = 1.0
            else:
                den = a_prev * zeta_prev[i] * (1.0 + s * a) + a * b_prev * (zeta_prev[i] - zeta[i])
                z_next = zeta[i] * zeta_prev[i] * a_prev / den
            ai = a * z_next / zeta[i]
            bi = bk * (z_next / zeta[i]) ** 2
            x[i] = x[i] + ai * p[i]
            p[i] = z_next * r + bi * p[i]
            zeta_prev[i], zeta[i] = zeta[i], z_next
        a_prev, b_prev = a, bk
        rr = rr_new
        info["iters"] = k + 1
    info["zeta"] = zeta.copy()
    return x, info
