"""Pins of the oracle's Schwarz preconditioner and Krylov solvers (Sec. 3, Sec. 8.1,
Algorithm 1) against dense linear algebra on tiny lattices. CPU only."""
import numpy as np
import pytest

from oracle import solvers, staggered, wilson
from oracle.lattice import all_coords
from paper_1109_2935_gb300 import synth


def _wilson_problem(dims, kappa=0.12, csw=1.0, seed=21):
    U = synth.wilson_gauge(dims, 0.5, 1, seed).numpy()
    A = wilson.clover(U, csw)
    M = lambda v: wilson.apply_M(U, A, kappa, v)
    b = synth.wilson_spinor(dims, seed + 1).numpy()
    return U, A, kappa, M, b


def _dense(M, shape):
    n = int(np.prod(shape))
    D = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        D[:, j] = M(e.reshape(shape)).ravel()
    return D


@pytest.fixture(scope="module")
def wilson24():
    dims = (2, 2, 2, 2)
    U, A, kappa, M, b = _wilson_problem(dims)
    D = _dense(M, b.shape)
    x = np.linalg.solve(D, b.ravel()).reshape(b.shape)
    return U, A, kappa, M, b, D, x


def test_bicgstab_matches_dense(wilson24):
    U, A, kappa, M, b, D, xd = wilson24
    x, info = solvers.bicgstab(M, b, 1e-12, 500)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert solvers.true_residual(M, x, b) < 1e-11


def test_cg_normal_matches_dense(wilson24):
    U, A, kappa, M, b, D, xd = wilson24
    Md = lambda v: wilson.apply_M(U, A, kappa, v, dagger=True)
    N = lambda v: Md(M(v))
    x, info = solvers.cg(N, b, 1e-12, 1000)
    xn = np.linalg.solve(D.conj().T @ D, b.ravel()).reshape(b.shape)
    assert np.linalg.norm(x - xn) / np.linalg.norm(xn) < 1e-10


def test_gcr_unpreconditioned_matches_dense(wilson24):
    U, A, kappa, M, b, D, xd = wilson24
    x, info = solvers.gcr(M, lambda r: r, b, 1e-12, 500, k_max=8, delta=0.0)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert info["restarts"] >= 1


def _dense_mr(D, b, n):
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(n):
        p = D @ r
        a = np.vdot(p, r) / np.vdot(p, p)
        x = x + a * r
        r = r - a * p
    return x


def test_schwarz_whole_lattice_block_is_plain_mr():
    dims = (4, 4, 2, 2)
    U, A, kappa, M, b = _wilson_problem(dims)
    D = _dense(M, b.shape)
    K = solvers.schwarz_mr(U, A, kappa, b, dims, 5)
    assert np.max(np.abs(K.ravel() - _dense_mr(D, b.ravel(), 5))) < 1e-12


def test_schwarz_block_is_dirichlet_principal_submatrix():
    """A source living on one block B gives K b supported on B, equal to MR on the
    principal submatrix M[B, B] of the full matrix (zero boundary conditions)."""
    dims = (4, 4, 4, 2)
    block = (2, 2, 2, 2)
    U, A, kappa, M, b = _wilson_problem(dims, kappa=0.124)
    D = _dense(M, b.shape)
    c = all_coords(dims)
    inB = (c[:, 0] >= 2) & (c[:, 1] < 2) & (c[:, 2] >= 2)
    mask = inB.reshape(dims[3], dims[2], dims[1], dims[0])
    bB = b * mask[..., None, None]
    K = solvers.schwarz_mr(U, A, kappa, bB, block, 4)
    assert np.max(np.abs(K[~mask])) == 0.0
    idx = np.repeat(np.where(inB)[0] * 12, 12) + np.tile(np.arange(12), inB.sum())
    sub = D[np.ix_(idx, idx)]
    xB = _dense_mr(sub, bB.reshape(-1)[idx], 4)
    assert np.max(np.abs(K.reshape(-1)[idx] - xB)) < 1e-12


def test_schwarz_single_site_blocks_use_clover_matrix():
    dims = (2, 2, 2, 4)
    U, A, kappa, M, b = _wilson_problem(dims)
    K = solvers.schwarz_mr(U, A, kappa, b, (1, 1, 1, 1), 3)
    Ahat = np.eye(12) + 2 * kappa * A.reshape(-1, 12, 12)
    bs = b.reshape(-1, 12)
    for s in range(bs.shape[0]):
        assert np.max(np.abs(K.reshape(-1, 12)[s] - _dense_mr(Ahat[s], bs[s], 3))) < 1e-13


def test_schwarz_is_block_additive_homogeneous_and_nonlinear():
    dims = (4, 4, 4, 4)
    block = (2, 2, 4, 2)
    U, A, kappa, M, b = _wilson_problem(dims)
    K = lambda v: solvers.schwarz_mr(U, A, kappa, v, block, 3)
    Kb = K(b)
    # block-Jacobi: K b = sum over blocks of K (b restricted to the block)
    bid = wilson.block_id(all_coords(dims), block).reshape(dims[::-1])
    acc = np.zeros_like(b)
    for v in np.unique(bid):
        acc += K(b * (bid == v)[..., None, None])
    assert np.max(np.abs(acc - Kb)) < 1e-13
    assert np.max(np.abs(K(2.0 * b) - 2.0 * Kb)) < 1e-13
    b2 = synth.wilson_spinor(dims, 99).numpy()
    assert np.max(np.abs(K(b + b2) - Kb - K(b2))) > 1e-3


def test_mr_step_minimises_residual():
    dims = (2, 2, 2, 2)
    U, A, kappa, M, b = _wilson_problem(dims)
    K1 = solvers.schwarz_mr(U, A, kappa, b, dims, 1)
    r1 = np.linalg.norm(b - M(K1))
    for eps in (1e-3, -1e-3, 1e-3j):
        r = np.linalg.norm(b - M(K1 * (1 + eps)))
        assert r > r1


def test_gcr_dd_matches_dense():
    dims = (4, 4, 2, 4)
    U, A, kappa, M, b = _wilson_problem(dims, kappa=0.125)
    D = _dense(M, b.shape)
    xd = np.linalg.solve(D, b.ravel()).reshape(b.shape)
    K = lambda r: solvers.schwarz_mr(U, A, kappa, r, (2, 2, 2, 2), 4)
    x, info = solvers.gcr(M, K, b, 1e-11, 300, k_max=6, delta=0.1)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
    assert solvers.true_residual(M, x, b) < 1e-11
    # preconditioning pays: fewer outer iterations than plain GCR
    _, info0 = solvers.gcr(M, lambda r: r, b, 1e-11, 300, k_max=6, delta=0.1)
    assert info["iters"] < info0["iters"]


def test_staggered_even_cg_matches_dense():
    dims = (4, 4, 4, 4)
    fat, lng = synth.asqtad_links(dims, 41, 42)
    fat, lng = fat.numpy(), lng.numpy()
    m = 0.05
    even = staggered.parity_mask(dims, 0)
    N = lambda v: staggered.apply_normal(fat, lng, m, v) * even[..., None]
    b = synth.staggered_spinor(dims, 43, parity=0).numpy()
    x, info = solvers.cg(N, b, 1e-12, 2000)
    Dn = _dense(N, b.shape)
    idx = np.repeat(np.where(even.ravel())[0] * 3, 3) + np.tile(np.arange(3), even.sum())
    xe = np.linalg.solve(Dn[np.ix_(idx, idx)], b.ravel()[idx])
    assert np.linalg.norm(x.ravel()[idx] - xe) / np.linalg.norm(xe) < 1e-10


def test_multishift_cg_matches_dense_for_every_shift():
    """Eq. 4: (M^dagger M + sigma_i) x_i = b, all shifts in one Krylov space, each
    solution equal to a dense solve, all done in the iterations of the smallest shift."""
    dims = (4, 4, 4, 4)
    fat, lng = synth.asqtad_links(dims, 51, 52)
    fat, lng = fat.numpy(), lng.numpy()
    m = 0.05
    even = staggered.parity_mask(dims, 0)
    N = lambda v: staggered.apply_normal(fat, lng, m, v) * even[..., None]
    b = synth.staggered_spinor(dims, 53, parity=0).numpy()
    shifts = [0.3, 0.0, 0.02, 1.5]
    xs, info = solvers.multishift_cg(N, b, shifts, 1e-12, 2000)
    Dn = _dense(N, b.shape)
    idx = np.repeat(np.where(even.ravel())[0] * 3, 3) + np.tile(np.arange(3), even.sum())
    Ae = Dn[np.ix_(idx, idx)]
    for sgm, x in zip(shifts, xs):
        xe = np.linalg.solve(Ae + sgm * np.eye(len(idx)), b.ravel()[idx])
        assert np.linalg.norm(x.ravel()[idx] - xe) / np.linalg.norm(xe) < 1e-10, sgm
    # the base (smallest-shift) system alone takes as many iterations
    _, info0 = solvers.cg(N, b, 1e-12, 2000)
    assert info["iters"] == info0["iters"]


def test_multishift_single_shift_is_plain_cg():
    dims = (2, 2, 2, 4)
    U = synth.wilson_gauge(dims, 0.5, 1, 61).numpy()
    A = wilson.clover(U, 1.0)
    Md = lambda v: wilson.apply_M(U, A, 0.12, v, dagger=True)
    N = lambda v: Md(wilson.apply_M(U, A, 0.12, v)) + 0.1 * v
    b = synth.wilson_spinor(dims, 62).numpy()
    (x,), _ = solvers.multishift_cg(lambda v: Md(wilson.apply_M(U, A, 0.12, v)), b, [0.1], 1e-12, 500)
    x0, _ = solvers.cg(N, b, 1e-12, 500)
    assert np.linalg.norm(x - x0) / np.linalg.norm(x0) < 1e-12
