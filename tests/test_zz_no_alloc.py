"""dirac_cdot_noalloc, the allocation-free inner product for callers that cannot
allocate GPU memory (a host code whose own pool already owns the device memory, or a
stream-ordered section where cudaMalloc would synchronise the device). It must give
the same (x, y) and ||x||^2 as the context-based dirac_cdot / dirac_norm2, on two
calls in a row (its fixed scratch array keeps the previous call's contents), and
reject fields larger than its scratch covers. Named so that pytest collects it last."""
import ctypes

import pytest
import torch

from paper_1109_2935_gb300 import synth

pytestmark = pytest.mark.gpu

F64, F32, F16 = 0, 1, 2


@pytest.mark.parametrize("kind,dims,prec,parity", [
    (0, (24, 24, 24, 32), F64, -1), (0, (24, 24, 24, 32), F32, -1), (0, (6, 6, 6, 10), F16, 0),
    (1, (8, 6, 4, 6), F32, 1), (1, (16, 16, 16, 32), F64, -1),
])
def test_cdot_noalloc_matches_cdot(dirac, kind, dims, prec, parity):
    lat = dirac.Lattice(dims, kind, kappa=0.1, mass=0.1)
    gen = synth.wilson_spinor if kind == 0 else synth.staggered_spinor
    fa = lat.to_device(gen(dims, 11).cuda(), prec, parity)
    fb = lat.to_device(gen(dims, 12).cuda(), prec, parity)
    ref = lat.cdot(fa, fb, prec, parity)
    refn = lat.norm2(fa, prec, parity)
    tol = 1e-13 if prec == F64 else 1e-6
    nr = 24 if kind == 0 else 6
    Vh = lat.volume // 2
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        res.fill_(float("nan"))
        rc = dirac.dirac_cdot_noalloc(fa.data_ptr(), fb.data_ptr(), prec, nr, Vh, parity,
                                      res.data_ptr(), stream, err, len(err))
        assert rc == dirac.OK, err.value
        torch.cuda.synchronize()
        got = res.cpu().tolist()
        assert abs(complex(got[0], got[1]) - ref) <= tol * abs(refn), (call, got, ref)
        assert abs(got[2] - refn) <= tol * refn, (call, got, refn)


def test_cdot_noalloc_rejects_oversize(dirac):
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    # 2 * 4,194,305 sites > 8,388,608: rejected on the host before any launch
    rc = dirac.dirac_cdot_noalloc(x.data_ptr(), x.data_ptr(), F32, 24, 4194305, -1,
                                  res.data_ptr(), None, err, len(err))
    assert rc == dirac.ERR_ARG
    assert b"exceed the maximum" in err.value
