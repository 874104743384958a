"""Batched solves (solve_batched): BiCGstab with reliable updates on many right-hand
sides of several lattices of different sizes, one iteration of all of them at a time
(batched operator, batched BLAS, replayed CUDA graph). Every right-hand side must reach
a true residual <= 1e-10 recomputed by the FP64 oracle (Eq. 2) from the returned x."""
import numpy as np
import pytest
import torch

from oracle import wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


def _problem(dirac, specs, recon=12):
    lats, xs, bs, nats = [], [], [], []
    for k, (dims, kappa, n) in enumerate(specs):
        U = synth.wilson_gauge(dims, 0.5, 0, 40 + k)
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, recon=(18, recon, recon))
        lat.load_gauge(U)
        fb = lat.field_bytes(dirac.F64)
        b = torch.zeros(n * fb, dtype=torch.uint8, device="cuda")
        src = []
        for r in range(n):
            psi = synth.wilson_spinor(dims, 500 + 17 * k + r)
            lat.import_spinor(b[r * fb:(r + 1) * fb], dirac.F64, -1, psi.cuda())
            src.append(psi.numpy())
        lats.append(lat)
        bs.append(b)
        xs.append(torch.zeros_like(b))
        nats.append((U.numpy(), kappa, src))
    return lats, xs, bs, nats


def _oracle_residuals(dirac, lats, xs, nats):
    out = []
    for lat, x, (Un, kappa, src) in zip(lats, xs, nats):
        A = wilson.clover(Un, 1.0)
        fb = lat.field_bytes(dirac.F64)
        for r, b in enumerate(src):
            xn = lat.to_natural(x[r * fb:(r + 1) * fb], dirac.F64, device="cpu").numpy()
            res = b - wilson.apply_M(Un, A, kappa, xn)
            out.append(np.linalg.norm(res) / np.linalg.norm(b))
    return out


@pytest.mark.parametrize("sloppy", [2, 1, 0])
def test_batched_bicgstab_reaches_1e10(dirac, sloppy):
    specs = [((4, 4, 4, 4), 0.130, 3), ((6, 6, 6, 10), 0.133, 5), ((8, 4, 4, 8), 0.136, 2)]
    lats, xs, bs, nats = _problem(dirac, specs)
    res = dirac.solve_many(lats, xs, bs, [s[2] for s in specs], tol=1e-10, max_iter=2000, delta=0.1,
                           prec_sloppy=sloppy)
    assert res["status"] == "OK"
    assert len(res["rhs"]) == 10
    for st in res["rhs"]:
        assert st["true_rel_resid"] <= 1e-10 and st["iters"] > 0
    for e in _oracle_residuals(dirac, lats, xs, nats):
        assert e <= 1e-10, e


def test_batched_matches_sequential_solves(dirac):
    """Each right-hand side's solution agrees with the single-system solve() to the
    accuracy both reach, and a zero source gives x = 0 without iterating."""
    specs = [((4, 4, 4, 6), 0.13, 3)]
    lats, xs, bs, nats = _problem(dirac, specs)
    lat = lats[0]
    fb = lat.field_bytes(dirac.F64)
    bs[0][fb:2 * fb].zero_()  # the second right-hand side is zero
    res = dirac.solve_many(lats, xs, bs, [3], tol=1e-11, prec_sloppy=dirac.F16)
    assert res["status"] == "OK"
    assert res["rhs"][1]["iters"] == 0 and torch.count_nonzero(xs[0][fb:2 * fb]) == 0
    for r in (0, 2):
        x1 = lat.new_field(dirac.F64)
        lat.solve(x1, bs[0][r * fb:(r + 1) * fb], dirac.BICGSTAB, tol=1e-11, delta=0.1, prec_sloppy=dirac.F16)
        a = lat.to_natural(x1, dirac.F64, device="cpu").numpy()
        b = lat.to_natural(xs[0][r * fb:(r + 1) * fb], dirac.F64, device="cpu").numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-8


def test_batched_initial_guess_and_errors(dirac):
    specs = [((4, 4, 4, 4), 0.13, 2), ((4, 4, 2, 4), 0.12, 1)]
    lats, xs, bs, nats = _problem(dirac, specs)
    res = dirac.solve_many(lats, xs, bs, [2, 1], tol=1e-10, prec_sloppy=dirac.F32)
    assert res["status"] == "OK"
    # restarting from the solution: converged before the first iteration
    res2 = dirac.solve_many(lats, xs, bs, [2, 1], tol=1e-10, prec_sloppy=dirac.F32, use_x0=True)
    assert res2["status"] == "OK" and all(st["iters"] == 0 for st in res2["rhs"])
    # a budget too small: NOT_CONVERGED, x holds the iterate
    for x in xs:
        x.zero_()
    res3 = dirac.solve_many(lats, xs, bs, [2, 1], tol=1e-14, max_iter=3, prec_sloppy=dirac.F32,
                            raise_on_error=False)
    assert res3["status"] == "ERR_NOT_CONVERGED"
    # a non-finite source is refused
    bs[0][:8] = 255
    res4 = dirac.solve_many(lats, xs, bs, [2, 1], raise_on_error=False)
    assert res4["status"] == "ERR_NONFINITE"


@pytest.mark.parametrize("sloppy", [2, 1])
def test_each_system_as_if_solved_alone(dirac, sloppy):
    """Batching does not change any system's iterates: every right-hand side, solved
    together with systems of other lattices that converge and update at other times,
    returns the bytes and the iteration and reliable-update counts of solve_batched on
    that right-hand side alone (per-system scalars, reductions, masks and reliable
    updates; the operator and BLAS per right-hand side do not depend on the others)."""
    specs = [((4, 4, 4, 6), 0.128, 2), ((6, 4, 4, 8), 0.135, 3)]
    lats, xs, bs, _ = _problem(dirac, specs)
    res = dirac.solve_many(lats, xs, bs, [s[2] for s in specs], tol=1e-10, max_iter=2000, delta=0.1,
                           prec_sloppy=sloppy)
    assert res["status"] == "OK"
    iters = [st["iters"] for st in res["rhs"]]
    assert len(set(iters)) > 1  # the systems really converge at different iterations
    k = 0
    for lat, x, b, (dims, kappa, n) in zip(lats, xs, bs, specs):
        fb = lat.field_bytes(dirac.F64)
        for r in range(n):
            x1 = torch.zeros(fb, dtype=torch.uint8, device="cuda")
            b1 = b[r * fb:(r + 1) * fb].clone()
            one = dirac.solve_many([lat], [x1], [b1], [1], tol=1e-10, max_iter=2000, delta=0.1,
                                   prec_sloppy=sloppy)
            assert one["status"] == "OK"
            assert one["rhs"][0]["iters"] == res["rhs"][k]["iters"], (k, one["rhs"][0], res["rhs"][k])
            assert one["rhs"][0]["reliable_updates"] == res["rhs"][k]["reliable_updates"]
            assert torch.equal(x1, x[r * fb:(r + 1) * fb]), k
            k += 1
