"""GPU parity of the additive Schwarz / block-MR preconditioner (Sec. 3.2, 8.1)
against the FP64 oracle through schwarz_precondition: several block shapes
(including a block spanning a whole extent, which keeps that extent's wrap), MR step
counts and storage precisions."""
import numpy as np
import pytest

from helpers import F16, F32, F64, check, dec_clover_hat, dec_links, dec_spinor
from oracle import solvers, wilson
from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,block,steps", [
    ((8, 8, 8, 8), (4, 4, 4, 4), 6),
    ((8, 4, 4, 8), (2, 2, 2, 2), 3),
    ((4, 4, 4, 4), (4, 4, 4, 4), 4),     # one block = the lattice: plain MR with wraps
    ((8, 4, 6, 4), (4, 2, 6, 2), 2),     # block spans the z extent
    ((4, 4, 4, 8), (1, 1, 1, 1), 3),     # single-site blocks: MR on the clover matrix
    ((8, 4, 4, 4), (4, 2, 2, 4), 3),     # block spans the antiperiodic t extent only
])
@pytest.mark.parametrize("prec,recon", [(F64, 18), (F64, 12), (F32, 12), (F32, 18), (F32, 8),
                                        (F16, 12), (F16, 18), (F16, 8)])
def test_schwarz_matches_oracle(dirac, dims, block, steps, prec, recon):
    kappa, csw = 0.124, 1.0
    U = synth.wilson_gauge(dims, 0.5, 2, 500 + sum(dims))
    b = synth.wilson_spinor(dims, 600 + sum(block))
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=csw, block=block,
                        mr_steps=steps, recon=(recon,) * 3)
    lat.load_gauge(U)
    x_in = lat.to_device(b.cuda(), prec)
    out = lat.new_field(prec)
    lat.schwarz(out, x_in, prec)
    got = lat.to_natural(out, prec, device="cpu").numpy()
    Un = U.numpy()
    Ahat = np.eye(12) + 2 * kappa * wilson.clover(Un, csw)
    Ad = (dec_clover_hat(Ahat, prec) - np.eye(12)) / (2 * kappa)
    ref = solvers.schwarz_mr(dec_links(Un, prec), Ad, kappa, dec_spinor(b.numpy(), prec), block, steps)
    check(got, ref, prec, 24, f"Schwarz dims={dims} block={block} prec={prec}")


def test_schwarz_zero_steps_and_zero_source(dirac):
    dims = (4, 4, 4, 4)
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=1.0, block=(2, 2, 2, 2),
                        mr_steps=0, recon=(18, 12, 12))
    lat.load_gauge(synth.wilson_gauge(dims, 0.5, 1, 3))
    x = lat.to_device(synth.wilson_spinor(dims, 4).cuda(), F32)
    out = lat.new_field(F32)
    out.fill_(7)
    lat.schwarz(out, x, F32)
    assert lat.norm2(out, F32) == 0.0          # zero MR steps: K = 0
    lat2 = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.12, csw=1.0, block=(2, 2, 2, 2),
                         mr_steps=3, recon=(18, 12, 12))
    lat2.load_gauge(synth.wilson_gauge(dims, 0.5, 1, 3))
    z = lat2.new_field(F16)
    out16 = lat2.new_field(F16)
    lat2.schwarz(out16, z, F16)                # zero source: alpha = 0 on every block
    assert lat2.norm2(out16, F16) == 0.0
