"""dirac_cdot_noalloc, the allocation-free inner product for callers that cannot
allocate GPU memory (a host code whose own pool already owns the device memory, or a
stream-ordered section where cudaMalloc would synchronise the device). It must give
the same (x, y) and ||x||^2 as numpy on the exported fields and as the context-based
dirac_cdot / dirac_norm2, on two calls in a row (its fixed scratch array keeps the
previous call's contents), cover exactly the number of sites its scratch is sized
for, and reject larger fields and host pointers before queuing anything. Named so
that pytest collects it last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu

F64, F32, F16 = 0, 1, 2
MAX_SITES = 8_388_608  # 4096 blocks x 256 threads x 8 sites


def _call(dirac, x, y, prec, nr, vh, parity, res, stream=None):
    err = ctypes.create_string_buffer(256)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    rc = dirac.dirac_cdot_noalloc(x, y, prec, nr, vh, parity, res, stream, err, len(err))
    return rc, err.value


@pytest.mark.parametrize("kind,dims,prec,parity", [
    (0, (24, 24, 24, 32), F64, -1), (0, (24, 24, 24, 32), F32, -1), (0, (6, 6, 6, 10), F16, 0),
    (1, (8, 6, 4, 6), F32, 1), (1, (16, 16, 16, 32), F64, -1), (1, (16, 8, 8, 12), F16, -1),
    (1, (6, 6, 6, 10), F16, 1),
])
def test_cdot_noalloc_matches_numpy_and_cdot(dirac, kind, dims, prec, parity):
    lat = dirac.Lattice(dims, kind, kappa=0.1, mass=0.1)
    gen = synth.wilson_spinor if kind == 0 else synth.staggered_spinor
    fa = lat.to_device(gen(dims, 11).cuda(), prec, parity)
    fb = lat.to_device(gen(dims, 12).cuda(), prec, parity)
    # numpy on the decoded fields: what the kernel must reduce
    xa = lat.to_natural(fa, prec, parity, device="cpu").numpy().ravel()
    xb = lat.to_natural(fb, prec, parity, device="cpu").numpy().ravel()
    ref_np = complex(np.vdot(xa, xb))
    refn_np = float(np.vdot(xa, xa).real)
    ref = lat.cdot(fa, fb, prec, parity)
    refn = lat.norm2(fa, prec, parity)
    scale = np.sqrt(refn_np * float(np.vdot(xb, xb).real))
    tol = 1e-13 if prec == F64 else 1e-6
    nr = 24 if kind == 0 else 6
    Vh = lat.volume // 2
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    for call in range(2):
        res.fill_(float("nan"))
        rc, msg = _call(dirac, fa.data_ptr(), fb.data_ptr(), prec, nr, Vh, parity, res.data_ptr())
        assert rc == dirac.OK, msg
        torch.cuda.synchronize()
        got = res.cpu().tolist()
        assert abs(complex(got[0], got[1]) - ref_np) <= tol * scale, (call, got, ref_np)
        assert abs(got[2] - refn_np) <= tol * refn_np, (call, got, refn_np)
        assert abs(complex(got[0], got[1]) - ref) <= tol * scale, (call, got, ref)
        assert abs(got[2] - refn) <= tol * refn, (call, got, refn)


def _raw_staggered_half(vh, npar, seed):
    """A staggered FP16 field in the device layout, built directly: per parity 3 chunks
    of binary16 (re, im) pairs for Vh sites, then Vh FP32 norms. Returns the bytes on
    the GPU and the decoded complex values (binary16 x norm in FP32, as stored)."""
    g = torch.Generator().manual_seed(seed)
    halves = (torch.rand((npar, 3, vh, 2), generator=g) * 2 - 1).to(torch.float16)
    norms = (torch.rand((npar, vh), generator=g) * 1.5 + 0.5).to(torch.float32)
    parts = []
    for p in range(npar):
        parts.append(halves[p].contiguous().view(torch.uint8).reshape(-1))
        parts.append(norms[p].contiguous().view(torch.uint8).reshape(-1))
    buf = torch.cat(parts).cuda()
    dec = (halves.to(torch.float32) * norms[:, None, :, None]).to(torch.float64).numpy()
    return buf, dec[..., 0] + 1j * dec[..., 1]


def test_cdot_noalloc_at_the_size_limit(dirac):
    """Exactly the sites the scratch array covers (the grid uses every partial-sum slot
    and the ticket sits in the slot after them), FP16 staggered storage, two calls in a
    row; one site more is rejected on the host."""
    vh = MAX_SITES // 2
    x, xd = _raw_staggered_half(vh, 2, 5)
    y, yd = _raw_staggered_half(vh, 2, 6)
    ref = complex(np.vdot(xd.ravel(), yd.ravel()))
    refn = float(np.vdot(xd.ravel(), xd.ravel()).real)
    scale = np.sqrt(refn * float(np.vdot(yd.ravel(), yd.ravel()).real))
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    for call in range(2):
        res.fill_(float("nan"))
        rc, msg = _call(dirac, x.data_ptr(), y.data_ptr(), F16, 6, vh, -1, res.data_ptr())
        assert rc == dirac.OK, msg
        torch.cuda.synchronize()
        got = res.cpu().tolist()
        assert abs(complex(got[0], got[1]) - ref) <= 1e-6 * scale, (call, got, ref)
        assert abs(got[2] - refn) <= 1e-6 * refn, (call, got, refn)
    # one half-field of MAX_SITES + 1 sites: rejected before any launch
    res.fill_(7.0)
    rc, msg = _call(dirac, x.data_ptr(), y.data_ptr(), F16, 6, MAX_SITES + 1, 0, res.data_ptr())
    assert rc == dirac.ERR_ARG and b"exceed the maximum" in msg
    torch.cuda.synchronize()
    assert res.cpu().tolist() == [7.0, 7.0, 7.0]


def test_cdot_noalloc_rejects_oversize(dirac):
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    # 2 * 4,194,305 sites > 8,388,608: rejected on the host before any launch
    rc, msg = _call(dirac, x.data_ptr(), x.data_ptr(), F32, 24, 4194305, -1, res.data_ptr(), stream=0)
    assert rc == dirac.ERR_ARG
    assert b"exceed the maximum" in msg


def test_cdot_noalloc_rejects_host_pointers(dirac):
    """A host result (page-locked or pageable) or host field is refused with ERR_ARG:
    the kernel would otherwise dereference it on the GPU."""
    dims = (4, 4, 4, 4)
    lat = dirac.Lattice(dims, 0, kappa=0.1)
    f = lat.to_device(synth.wilson_spinor(dims, 3).cuda(), F32, -1)
    Vh = lat.volume // 2
    pinned = torch.full((3,), 5.0, dtype=torch.float64).pin_memory()
    pageable = (ctypes.c_double * 3)(5.0, 5.0, 5.0)
    dev_res = torch.zeros(3, dtype=torch.float64, device="cuda")
    host_field = torch.zeros(f.numel(), dtype=torch.uint8).pin_memory()
    for res_ptr in (pinned.data_ptr(), ctypes.addressof(pageable)):
        rc, msg = _call(dirac, f.data_ptr(), f.data_ptr(), F32, 24, Vh, -1, res_ptr)
        assert rc == dirac.ERR_ARG and b"result must be device memory" in msg
    rc, msg = _call(dirac, host_field.data_ptr(), f.data_ptr(), F32, 24, Vh, -1, dev_res.data_ptr())
    assert rc == dirac.ERR_ARG and b"x and y must be device memory" in msg
    torch.cuda.synchronize()
    assert pinned.tolist() == [5.0, 5.0, 5.0] and list(pageable) == [5.0, 5.0, 5.0]
    # the entry point still works afterwards
    rc, msg = _call(dirac, f.data_ptr(), f.data_ptr(), F32, 24, Vh, -1, dev_res.data_ptr())
    assert rc == dirac.OK, msg
    torch.cuda.synchronize()
    assert abs(dev_res[2].item() - lat.norm2(f, F32)) <= 1e-6 * lat.norm2(f, F32)
