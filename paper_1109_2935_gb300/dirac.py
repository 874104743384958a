"""Thin ctypes binding of libdirac (C ABI in include/dirac.h).

The functions here carry the C names and only marshal arguments: every operator,
preconditioner, BLAS and solver step runs in the CUDA library. There is no Python or
CPU fallback: importing this module fails loudly when ``libdirac.so`` has not been
built (``python -m paper_1109_2935_gb300.build``).

Spinor arguments are device pointers (ints, e.g. ``tensor.data_ptr()``) in the
library's device layout; ``Lattice`` below wraps a context and accepts torch tensors.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdirac.so")

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_UNSUPPORTED = -1, -2, -3, -4
ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = -5, -6, -7, -8, -9
ERR_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_UNSUPPORTED",
             -5: "ERR_NOT_CONVERGED", -6: "ERR_BREAKDOWN", -7: "ERR_NONFINITE",
             -8: "ERR_TIMEOUT", -9: "ERR_STATE"}

WILSON_CLOVER, ASQTAD = 0, 1
F64, F32, F16 = 0, 1, 2
PARITY_FULL, PARITY_EVEN, PARITY_ODD = -1, 0, 1
CG_NORMAL, CG_EVEN_NORMAL, BICGSTAB, GCR_DD, GCR, BICGSTAB_EO, GCR_EO, GCR_PTC = 0, 1, 2, 3, 4, 5, 6, 7
PRECOND_NAMES = {0: "none", 1: "schwarz", 2: "ptc"}


class DiracParams(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("t_antiperiodic", ctypes.c_int),
                ("kind", ctypes.c_int), ("kappa", ctypes.c_double), ("csw", ctypes.c_double),
                ("mass", ctypes.c_double), ("block", ctypes.c_int * 4), ("mr_steps", ctypes.c_int),
                ("recon", ctypes.c_int * 3), ("prec_mask", ctypes.c_uint)]


class SolverParams(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("k_max", ctypes.c_int), ("delta", ctypes.c_double), ("use_x0", ctypes.c_int),
                ("prec_sloppy", ctypes.c_int), ("prec_precond", ctypes.c_int)]


class SolverStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("dslash_calls", ctypes.c_int),
                ("precond_calls", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("flops", ctypes.c_double),
                ("precond_kind", ctypes.c_int), ("precond_reduction", ctypes.c_double * 2),
                ("precond_rate", ctypes.c_double * 2), ("precond_switches", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["precond_reduction"] = list(self.precond_reduction)
        d["precond_rate"] = list(self.precond_rate)
        d["precond"] = PRECOND_NAMES.get(self.precond_kind, self.precond_kind)
        return d


class PtcParams(ctypes.Structure):
    _fields_ = [("layers", ctypes.c_int), ("channels", ctypes.c_int * 5)]


class PtcTrainParams(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdirac.so is not built ({LIB_PATH}); run "
                      "`python -m paper_1109_2935_gb300.build`")
lib = ctypes.CDLL(LIB_PATH)

_vp, _ci, _cd, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_pd = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "dirac_create": (_ci, [ctypes.POINTER(DiracParams), ctypes.POINTER(_vp)]),
    "dirac_destroy": (_ci, [_vp]),
    "dirac_last_error": (ctypes.c_char_p, [_vp]),
    "dirac_field_bytes": (_sz, [_vp, _ci, _ci]),
    "dirac_load_gauge": (_ci, [_vp, _vp, _ci, _ci, _vp]),
    "dirac_import_spinor": (_ci, [_vp, _vp, _ci, _ci, _vp, _ci, _vp]),
    "dirac_export_spinor": (_ci, [_vp, _vp, _ci, _vp, _ci, _ci, _vp]),
    "dirac_apply": (_ci, [_vp, _vp, _vp, _ci, _ci, _vp]),
    "dirac_apply_dagger": (_ci, [_vp, _vp, _vp, _ci, _ci, _vp]),
    "dirac_apply_normal": (_ci, [_vp, _vp, _vp, _ci, _ci, _vp]),
    "dirac_apply_ds": (_ci, [_vp, _vp, _vp, _ci, _vp]),
    "dirac_set_ds_residual": (_ci, [_vp, _ci]),
    "schwarz_precondition": (_ci, [_vp, _vp, _vp, _ci, _vp]),
    "dirac_apply_eo": (_ci, [_vp, _vp, _vp, _ci, _ci, _vp]),
    "dirac_apply_multi": (_ci, [_vp, _vp, _vp, _ci, _ci, _vp]),
    "dirac_batch_create": (_ci, [ctypes.POINTER(_vp), _ci, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                 ctypes.POINTER(_ci), _ci, _vp, ctypes.POINTER(_vp)]),
    "dirac_batch_apply": (_ci, [_vp, _vp]),
    "dirac_batch_capture": (_ci, [_vp, _ci, _vp]),
    "dirac_batch_info": (_ci, [_vp, ctypes.POINTER(_ci), ctypes.POINTER(_ci), ctypes.POINTER(_ci),
                               ctypes.POINTER(ctypes.c_double)]),
    "dirac_batch_destroy": (_ci, [_vp]),
    "dirac_batch_set_tensor_cores": (_ci, [_vp, _ci]),
    "dirac_batch_kernel_info": (_ci, [_vp, ctypes.POINTER(_ci), _pd, _pd]),
    "dirac_norm2": (_ci, [_vp, _vp, _ci, _ci, _pd, _vp]),
    "dirac_cdot": (_ci, [_vp, _vp, _vp, _ci, _ci, _pd, _vp]),
    "dirac_caxpy_norm": (_ci, [_vp, _cd, _cd, _vp, _vp, _ci, _ci, _pd, _vp]),
    "dirac_convert": (_ci, [_vp, _vp, _ci, _vp, _ci, _ci, _vp]),
    "solve": (_ci, [_vp, _vp, _vp, ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), _vp]),
    "dirac_cdot_noalloc": (_ci, [_vp, _vp, _ci, _ci, ctypes.c_longlong, _ci, _vp, _vp,
                                 ctypes.c_char_p, _sz]),
    "solve_batched": (_ci, [ctypes.POINTER(_vp), _ci, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                            ctypes.POINTER(_ci), ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), _vp]),
    "solve_multishift": (_ci, [_vp, ctypes.POINTER(_vp), _vp, ctypes.POINTER(ctypes.c_double), _ci,
                               ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats), _vp]),
    "dirac_ptc_create": (_ci, [_vp, ctypes.POINTER(PtcParams), ctypes.POINTER(_vp)]),
    "dirac_ptc_num_weights": (ctypes.c_longlong, [_vp]),
    "dirac_ptc_set_weights": (_ci, [_vp, _pd, ctypes.c_longlong]),
    "dirac_ptc_get_weights": (_ci, [_vp, _pd, ctypes.c_longlong]),
    "dirac_ptc_apply": (_ci, [_vp, _vp, _vp, _vp]),
    "dirac_ptc_gradient": (_ci, [_vp, _vp, _vp, _pd, _pd, _vp]),
    "dirac_ptc_train": (_ci, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ci,
                              ctypes.POINTER(PtcTrainParams), _pd, _vp]),
    "dirac_ptc_attach": (_ci, [_vp, _vp, _ci]),
    "dirac_ptc_set_tensor_cores": (_ci, [_vp, _ci]),
    "dirac_ptc_test_stall": (_ci, [_vp, _ci, _cd]),
    "dirac_ptc_destroy": (_ci, [_vp]),
    "dirac_dd_create": (_ci, [_vp, _ci, _ci, ctypes.POINTER(_vp)]),
    "dirac_dd_create_grid": (_ci, [_vp, ctypes.POINTER(_ci), _ci, ctypes.POINTER(_vp)]),
    "dirac_dd_scatter": (_ci, [_vp, _vp, _vp]),
    "dirac_dd_apply": (_ci, [_vp, _ci, _vp]),
    "dirac_dd_gather": (_ci, [_vp, _vp, _vp]),
    "dirac_dd_info": (_ci, [_vp, ctypes.POINTER(_ci), ctypes.POINTER(ctypes.c_longlong)]),
    "dirac_dd_destroy": (_ci, [_vp]),
}
EXPORTED = tuple(_SIGS)
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype, _f.argtypes = _res, _args
    globals()[_name] = _f


class DiracError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Lattice:
    """A libdirac context plus torch-tensor marshalling. Owns nothing but the context."""

    def __init__(self, dims, kind=WILSON_CLOVER, kappa=0.12, csw=0.0, mass=0.0,
                 t_antiperiodic=True, block=None, mr_steps=6, recon=(18, 12, 12),
                 prec_mask=7):
        if block is None:  # largest of 4, 2, 1 dividing each extent
            block = tuple(next(b for b in (4, 2, 1) if d % b == 0) for d in dims)
        p = DiracParams()
        p.dims[:] = list(dims)
        p.t_antiperiodic = int(t_antiperiodic)
        p.kind = kind
        p.kappa, p.csw, p.mass = kappa, csw, mass
        p.block[:] = list(block)
        p.mr_steps = mr_steps
        p.recon[:] = list(recon)
        p.prec_mask = prec_mask
        self.params = p
        self.dims = tuple(dims)
        self.kind = kind
        self.nr = 24 if kind == WILSON_CLOVER else 6
        h = _vp()
        rc = dirac_create(ctypes.byref(p), ctypes.byref(h))
        if rc != OK:
            raise DiracError(rc, "dirac_create rejected the parameters")
        self.ctx = h

    def close(self):
        if self.ctx:
            dirac_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc, what):
        if rc != OK:
            raise DiracError(rc, f"{what}: {dirac_last_error(self.ctx).decode()}")
        return rc

    @property
    def volume(self):
        v = 1
        for d in self.dims:
            v *= d
        return v

    def field_bytes(self, prec, parity=PARITY_FULL):
        return dirac_field_bytes(self.ctx, prec, parity)

    def new_field(self, prec, parity=PARITY_FULL, device="cuda"):
        import torch
        return torch.zeros(self.field_bytes(prec, parity), dtype=torch.uint8, device=device)

    def load_gauge(self, links, which=0, stream=None):
        """links: complex128 [t,z,y,x,mu,3,3] tensor (CPU or CUDA), natural layout."""
        import torch
        t = torch.view_as_real(links.contiguous()) if links.is_complex() else links.contiguous()
        on_dev = int(t.is_cuda)
        self.check(dirac_load_gauge(self.ctx, t.data_ptr(), which, on_dev, _stream(stream)),
                   "dirac_load_gauge")
        if not on_dev:
            torch.cuda.synchronize()

    def import_spinor(self, dst, prec, parity, natural, stream=None):
        import torch
        t = torch.view_as_real(natural.contiguous()) if natural.is_complex() else natural.contiguous()
        self.check(dirac_import_spinor(self.ctx, dst.data_ptr(), prec, parity, t.data_ptr(),
                                       int(t.is_cuda), _stream(stream)), "dirac_import_spinor")
        return dst

    def export_spinor(self, src, prec, parity, natural, stream=None):
        """natural: complex128 tensor to fill (CPU or CUDA)."""
        import torch
        t = torch.view_as_real(natural)
        self.check(dirac_export_spinor(self.ctx, t.data_ptr(), int(t.is_cuda), src.data_ptr(),
                                       prec, parity, _stream(stream)), "dirac_export_spinor")
        return natural

    def natural_shape(self):
        LX, LY, LZ, LT = self.dims
        return (LT, LZ, LY, LX, 4, 3) if self.nr == 24 else (LT, LZ, LY, LX, 3)

    def to_device(self, natural, prec, parity=PARITY_FULL):
        f = self.new_field(prec, parity)
        return self.import_spinor(f, prec, parity, natural)

    def to_natural(self, field, prec, parity=PARITY_FULL, device="cuda"):
        import torch
        out = torch.zeros(self.natural_shape(), dtype=torch.complex128, device=device)
        self.export_spinor(field, prec, parity, out)
        if device != "cuda":
            torch.cuda.synchronize()
        return out

    def apply(self, out, inp, parity=PARITY_FULL, prec=F64, stream=None):
        return self.check(dirac_apply(self.ctx, out.data_ptr(), inp.data_ptr(), parity, prec,
                                      _stream(stream)), "dirac_apply")

    def apply_dagger(self, out, inp, parity=PARITY_FULL, prec=F64, stream=None):
        return self.check(dirac_apply_dagger(self.ctx, out.data_ptr(), inp.data_ptr(), parity,
                                             prec, _stream(stream)), "dirac_apply_dagger")

    def apply_ds(self, out, inp, dagger=False, stream=None):
        """M (or M^dagger) on FP64 full fields in double-single arithmetic."""
        return self.check(dirac_apply_ds(self.ctx, out.data_ptr(), inp.data_ptr(), int(dagger), _stream(stream)),
                          "dirac_apply_ds")

    def set_ds_residual(self, on):
        return self.check(dirac_set_ds_residual(self.ctx, int(on)), "dirac_set_ds_residual")

    def apply_normal(self, out, inp, parity=PARITY_FULL, prec=F64, stream=None):
        return self.check(dirac_apply_normal(self.ctx, out.data_ptr(), inp.data_ptr(), parity,
                                             prec, _stream(stream)), "dirac_apply_normal")

    def apply_eo(self, out, inp, prec=F64, dagger=False, stream=None):
        return self.check(dirac_apply_eo(self.ctx, out.data_ptr(), inp.data_ptr(), prec, int(dagger),
                                         _stream(stream)), "dirac_apply_eo")

    def apply_multi(self, out, inp, nrhs, prec=F16, stream=None):
        """out_r = M in_r for nrhs consecutive full fields in `inp` / `out`."""
        return self.check(dirac_apply_multi(self.ctx, out.data_ptr(), inp.data_ptr(), nrhs, prec,
                                            _stream(stream)), "dirac_apply_multi")

    def schwarz(self, out, inp, prec=F16, stream=None):
        return self.check(schwarz_precondition(self.ctx, out.data_ptr(), inp.data_ptr(), prec,
                                               _stream(stream)), "schwarz_precondition")

    def norm2(self, x, prec, parity=PARITY_FULL, stream=None):
        r = ctypes.c_double()
        self.check(dirac_norm2(self.ctx, x.data_ptr(), prec, parity, ctypes.byref(r),
                               _stream(stream)), "dirac_norm2")
        return r.value

    def cdot(self, x, y, prec, parity=PARITY_FULL, stream=None):
        r = (ctypes.c_double * 2)()
        self.check(dirac_cdot(self.ctx, x.data_ptr(), y.data_ptr(), prec, parity, r,
                              _stream(stream)), "dirac_cdot")
        return complex(r[0], r[1])

    def caxpy_norm(self, a, x, y, prec, parity=PARITY_FULL, stream=None):
        r = ctypes.c_double()
        a = complex(a)
        self.check(dirac_caxpy_norm(self.ctx, a.real, a.imag, x.data_ptr(), y.data_ptr(), prec,
                                    parity, ctypes.byref(r), _stream(stream)), "dirac_caxpy_norm")
        return r.value

    def convert(self, dst, dprec, src, sprec, parity=PARITY_FULL, stream=None):
        return self.check(dirac_convert(self.ctx, dst.data_ptr(), dprec, src.data_ptr(), sprec,
                                        parity, _stream(stream)), "dirac_convert")

    def solve(self, x, b, alg, tol=1e-10, max_iter=10000, k_max=16, delta=0.0, use_x0=False,
              prec_sloppy=F64, prec_precond=F64, stream=None, raise_on_error=True):
        sp = SolverParams(alg, tol, max_iter, k_max, delta, int(use_x0), prec_sloppy, prec_precond)
        st = SolverStats()
        rc = solve(self.ctx, x.data_ptr(), b.data_ptr(), ctypes.byref(sp), ctypes.byref(st),
                   _stream(stream))
        if raise_on_error and rc != OK:
            raise DiracError(rc, f"solve: {dirac_last_error(self.ctx).decode()} "
                                 f"(stats {st.as_dict()})")
        d = st.as_dict()
        d["status"] = ERR_NAMES.get(rc, rc)
        return d

    def solve_multishift(self, xs, b, shifts, alg, tol=1e-10, max_iter=10000, delta=0.1,
                         prec_sloppy=F32, stream=None, raise_on_error=True):
        """Eq. 4: (M^dagger M + sigma_j) x_j = b for every shift (Sec. 8.2 strategy).
        Returns the stats of the multi-shift stage and of each refinement."""
        n = len(shifts)
        sp = SolverParams(alg, tol, max_iter, 16, delta, 1, prec_sloppy, prec_sloppy)
        st = (SolverStats * (n + 1))()
        ptrs = (_vp * n)(*[x.data_ptr() for x in xs])
        sh = (ctypes.c_double * n)(*shifts)
        rc = solve_multishift(self.ctx, ptrs, b.data_ptr(), sh, n, ctypes.byref(sp), st,
                              _stream(stream))
        if raise_on_error and rc != OK:
            raise DiracError(rc, f"solve_multishift: {dirac_last_error(self.ctx).decode()}")
        return {"status": ERR_NAMES.get(rc, rc), "multishift": st[0].as_dict(),
                "refine": [st[1 + j].as_dict() for j in range(n)]}


def solve_many(lattices, xs, bs, nrhs, tol=1e-10, max_iter=10000, delta=0.1, prec_sloppy=F16,
               use_x0=False, stream=None, raise_on_error=True):
    """solve_batched: BiCGstab with reliable updates on nrhs[l] consecutive FP64 full fields
    of xs[l] / bs[l] for every lattice, all right-hand sides iterated together. Returns the
    status and one statistics dict per right-hand side (lattice-major)."""
    n = len(lattices)
    ctxs = (_vp * n)(*[l.ctx.value if hasattr(l.ctx, "value") else l.ctx for l in lattices])
    xp = (_vp * n)(*[t.data_ptr() for t in xs])
    bp = (_vp * n)(*[t.data_ptr() for t in bs])
    r = (_ci * n)(*nrhs)
    sp = SolverParams(BICGSTAB, tol, max_iter, 16, delta, int(use_x0), prec_sloppy, prec_sloppy)
    st = (SolverStats * sum(nrhs))()
    rc = solve_batched(ctxs, n, xp, bp, r, ctypes.byref(sp), st, _stream(stream))
    if raise_on_error and rc != OK:
        raise DiracError(rc, f"solve_batched: {dirac_last_error(lattices[0].ctx).decode()}")
    return {"status": ERR_NAMES.get(rc, rc), "rhs": [st[j].as_dict() for j in range(sum(nrhs))]}


class Batch:
    """A batched-operator plan over several lattices (dirac_batch_*): M of each lattice
    applied to its consecutive right-hand sides in one persistent launch."""

    def __init__(self, lattices, outs, ins, nrhs, prec=F16, stream=None):
        n = len(lattices)
        self.keep = (lattices, outs, ins)
        ctxs = (_vp * n)(*[l.ctx.value if hasattr(l.ctx, "value") else l.ctx for l in lattices])
        o = (_vp * n)(*[t.data_ptr() for t in outs])
        i = (_vp * n)(*[t.data_ptr() for t in ins])
        r = (_ci * n)(*nrhs)
        h = _vp()
        rc = dirac_batch_create(ctxs, n, o, i, r, prec, _stream(stream), ctypes.byref(h))
        if rc != OK:
            raise DiracError(rc, "dirac_batch_create failed")
        self.plan = h

    def info(self):
        rg, per, grid, ms = _ci(), _ci(), _ci(), ctypes.c_double()
        dirac_batch_info(self.plan, ctypes.byref(rg), ctypes.byref(per), ctypes.byref(grid), ctypes.byref(ms))
        return {"rhs_per_cta": rg.value, "ctas_per_sm": per.value, "grid": grid.value,
                "tuned_ms": ms.value}

    def set_tensor_cores(self, on):
        """Select the tensor-core kernel (FP16 storage) or the CUDA-core kernel."""
        rc = dirac_batch_set_tensor_cores(self.plan, int(on))
        if rc != OK:
            raise DiracError(rc, "dirac_batch_set_tensor_cores failed")

    def kernel_info(self):
        on, cc, tc = _ci(), ctypes.c_double(), ctypes.c_double()
        dirac_batch_kernel_info(self.plan, ctypes.byref(on), ctypes.byref(cc), ctypes.byref(tc))
        return {"tensor_cores": bool(on.value), "cuda_core_ms": cc.value, "tensor_core_ms": tc.value}

    def apply(self, stream=None):
        rc = dirac_batch_apply(self.plan, _stream(stream))
        if rc != OK:
            raise DiracError(rc, "dirac_batch_apply failed")

    def capture(self, napply, stream=None):
        rc = dirac_batch_capture(self.plan, napply, _stream(stream))
        if rc != OK:
            raise DiracError(rc, "dirac_batch_capture failed")

    def close(self):
        if self.plan:
            dirac_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ptc:
    """A gauge-equivariant parallel-transport convolution network on a Wilson-clover
    lattice (dirac_ptc_*): K = L_n ... L_1 with channels (1, c_1, ..., 1). Weights are
    exchanged as a list of complex arrays shaped (9, c_out, c_in, 4, 4) per layer;
    fields are FP32 full fields in the library layout (``Lattice.to_device(.., F32)``)."""

    def __init__(self, lattice, channels=(1, 2, 1)):
        self.lat = lattice
        self.channels = tuple(channels)
        p = PtcParams()
        p.layers = len(channels) - 1
        p.channels[:len(channels)] = list(channels)
        h = _vp()
        lattice.check(dirac_ptc_create(lattice.ctx, ctypes.byref(p), ctypes.byref(h)), "dirac_ptc_create")
        self.net = h
        self.shapes = [(9, channels[l + 1], channels[l], 4, 4) for l in range(len(channels) - 1)]
        self.n = dirac_ptc_num_weights(self.net)

    def set_weights(self, ws):
        import numpy as np
        flat = np.concatenate([np.asarray(w, dtype=np.complex128).reshape(-1) for w in ws])
        if flat.size != self.n:
            raise ValueError(f"expected {self.n} complex weights, got {flat.size}")
        buf = np.ascontiguousarray(flat).view(np.float64)
        self.lat.check(dirac_ptc_set_weights(self.net, buf.ctypes.data_as(_pd), self.n),
                       "dirac_ptc_set_weights")

    def _split(self, flat):
        out, off = [], 0
        for s in self.shapes:
            k = s[0] * s[1] * s[2] * s[3] * s[4]
            out.append(flat[off:off + k].reshape(s))
            off += k
        return out

    def get_weights(self):
        import numpy as np
        buf = np.zeros(2 * self.n)
        self.lat.check(dirac_ptc_get_weights(self.net, buf.ctypes.data_as(_pd), self.n),
                       "dirac_ptc_get_weights")
        return self._split(buf.view(np.complex128))

    def apply(self, out, inp, stream=None):
        return self.lat.check(dirac_ptc_apply(self.net, out.data_ptr(), inp.data_ptr(), _stream(stream)),
                              "dirac_ptc_apply")

    def gradient(self, r, v, stream=None):
        """(loss, [dL/dconj(W_l)]) of one pair, L = |K r - v|^2 / |v|^2."""
        import numpy as np
        loss = ctypes.c_double()
        buf = np.zeros(2 * self.n)
        self.lat.check(dirac_ptc_gradient(self.net, r.data_ptr(), v.data_ptr(), ctypes.byref(loss),
                                          buf.ctypes.data_as(_pd), _stream(stream)), "dirac_ptc_gradient")
        return loss.value, self._split(buf.view(np.complex128))

    def train(self, vs, rs=None, steps=100, batch=4, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
              seed=0, stream=None):
        """Adam on the pairs (r_i, v_i) (r_i = M v_i computed by the library when rs is
        None). Returns the batch loss before each step."""
        import numpy as np
        n = len(vs)
        vp = (_vp * n)(*[v.data_ptr() for v in vs])
        rp = (_vp * n)(*[r.data_ptr() for r in rs]) if rs is not None else None
        P = PtcTrainParams(steps, batch, lr, beta1, beta2, eps, seed)
        loss = np.zeros(max(steps, 1))
        self.lat.check(dirac_ptc_train(self.net, rp, vp, n, ctypes.byref(P), loss.ctypes.data_as(_pd),
                                       _stream(stream)), "dirac_ptc_train")
        return loss[:steps]

    def tensor_cores(self, on=True):
        """Inference on the tensor cores (BF16, FP32 accumulate) or the FP32 layers."""
        return self.lat.check(dirac_ptc_set_tensor_cores(self.net, int(on)), "dirac_ptc_set_tensor_cores")

    def attach(self, force=False):
        return self.lat.check(dirac_ptc_attach(self.lat.ctx, self.net, int(force)), "dirac_ptc_attach")

    def detach(self):
        return self.lat.check(dirac_ptc_attach(self.lat.ctx, None, 0), "dirac_ptc_attach")

    def save(self, prefix, meta=None):
        """Checkpoint: the weights as raw little-endian FP64 (re, im) pairs in layer order
        ([p][c_out][c_in][s][t], the C ABI order) to prefix.bin, and prefix.json with the
        channel list, the weight count and `meta` (e.g. kappa, lattice, training run)."""
        import json
        import numpy as np
        flat = np.concatenate([w.reshape(-1) for w in self.get_weights()]).astype("<c16")
        flat.view("<f8").tofile(prefix + ".bin")
        with open(prefix + ".json", "w") as f:
            json.dump({"format": "ptc-weights-v1", "channels": list(self.channels), "complex_weights": int(self.n),
                       "dtype": "float64 little-endian (re, im) pairs", "meta": meta or {}}, f, indent=1)

    def load(self, prefix):
        """Restore weights saved by save(); the channel lists must match."""
        import json
        import numpy as np
        with open(prefix + ".json") as f:
            info = json.load(f)
        if tuple(info["channels"]) != self.channels or info["complex_weights"] != self.n:
            raise ValueError(f"checkpoint is for channels {info['channels']}, this network has {self.channels}")
        flat = np.fromfile(prefix + ".bin", dtype="<f8").view(np.complex128)
        if flat.size != self.n:
            raise ValueError("checkpoint size does not match its description")
        self.set_weights(self._split(flat))
        return info.get("meta", {})

    def close(self):
        if self.net and self.lat.ctx:
            dirac_ptc_destroy(self.net)
        self.net = None


class DomainDecomposition:
    """dirac_dd_*: the Wilson-clover operator over virtual ranks with ghost zones and face
    exchange, on one GPU. `ranks` is a number of t-slabs or a grid (gx, gy, gz, gt) of
    ranks per dimension."""

    def __init__(self, lattice, ranks, prec):
        self.lat = lattice
        h = _vp()
        if isinstance(ranks, (tuple, list)):
            grid = (_ci * 4)(*[int(v) for v in ranks])
            lattice.check(dirac_dd_create_grid(lattice.ctx, grid, prec, ctypes.byref(h)), "dirac_dd_create_grid")
        else:
            lattice.check(dirac_dd_create(lattice.ctx, int(ranks), prec, ctypes.byref(h)), "dirac_dd_create")
        self.dd = h

    def info(self):
        dims = (_ci * 4)()
        fb = ctypes.c_longlong()
        dirac_dd_info(self.dd, dims, ctypes.byref(fb))
        return {"local_dims": tuple(dims), "face_bytes": fb.value}

    def scatter(self, field, stream=None):
        return self.lat.check(dirac_dd_scatter(self.dd, field.data_ptr(), _stream(stream)), "dirac_dd_scatter")

    def apply(self, dagger=False, stream=None):
        return self.lat.check(dirac_dd_apply(self.dd, int(dagger), _stream(stream)), "dirac_dd_apply")

    def gather(self, field, stream=None):
        return self.lat.check(dirac_dd_gather(self.dd, field.data_ptr(), _stream(stream)), "dirac_dd_gather")

    def close(self):
        if self.dd:
            dirac_dd_destroy(self.dd)
            self.dd = None
