"""Shared helpers for the GPU parity tests: the oracle-side view of each storage
precision and the tolerance checks (FP64: global relative L2 <= 1e-12; FP32: global
relative L2 <= 1e-5; FP16 storage: per site ||gpu - oracle|| <= 1e-2 ||oracle||)."""
import numpy as np

from oracle import codecs

F64, F32, F16 = 0, 1, 2
TOL = {F64: 1e-12, F32: 1e-5}
FP16_SITE_TOL = 1e-2


def dec_spinor(psi, prec):
    if prec == F64:
        return psi
    if prec == F32:
        return codecs.spinor_single(psi)
    return codecs.spinor_half(psi)


def dec_links(U, prec):
    """Links as the kernel of that precision sees them. Reconstruction (12/8) is
    exact up to rounding in the kernel's own precision, so the oracle takes the
    stored precision's rounding of the full matrix."""
    if prec == F64:
        return U
    if prec == F32:
        return codecs.links_single(U)
    return codecs.links_half(U)


def dec_clover_hat(Ahat, prec):
    if prec == F64:
        return Ahat
    if prec == F32:
        return codecs.clover_single(Ahat)
    return codecs.clover_half(Ahat)


def site_norms(x, nr):
    return np.sqrt(np.sum(np.abs(x.reshape(-1, nr // 2)) ** 2, axis=1))


def check(gpu, ref, prec, nr, what=""):
    """Assert the precision's bound; returns the measured error figure."""
    gpu = np.asarray(gpu).reshape(-1, nr // 2)
    ref = np.asarray(ref).reshape(-1, nr // 2)
    if prec == F16:
        n = site_norms(ref, nr)
        e = site_norms(gpu - ref, nr)
        mask = n > 1e-12 * max(n.max(), 1e-300)
        err = float(np.max(e[mask] / n[mask])) if mask.any() else float(e.max())
        assert err <= FP16_SITE_TOL, f"{what}: FP16 per-site error {err:.3e}"
        return err
    err = float(np.linalg.norm(gpu - ref) / np.linalg.norm(ref))
    assert err <= TOL[prec], f"{what}: prec {prec} relative L2 error {err:.3e}"
    return err


def parity_mask(dims, parity):
    LX, LY, LZ, LT = dims
    t, z, y, x = np.meshgrid(np.arange(LT), np.arange(LZ), np.arange(LY), np.arange(LX),
                             indexing="ij")
    return (x + y + z + t) % 2 == parity
