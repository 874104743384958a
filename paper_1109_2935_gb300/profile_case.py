"""Run one operator of the library on a seeded synthetic lattice, a few times, for a
profiler to capture (``ncu -k <kernel> ...``) and for a quick CUDA-event timing.

    python -m paper_1109_2935_gb300.profile_case batch --dims 24 24 24 64 --nrhs 12 --kernel tc
    python -m paper_1109_2935_gb300.profile_case batch --dims 24 24 24 64 --nrhs 12 --kernel cc
    python -m paper_1109_2935_gb300.profile_case ptc --dims 16 16 16 16 --channels 1 2 2 1
    python -m paper_1109_2935_gb300.profile_case wilson --dims 24 24 24 64 --prec f16
    python -m paper_1109_2935_gb300.profile_case schwarz --dims 24 24 24 128 --prec f16

Each case does `--warmup` untimed applications and `--steps` timed ones and prints one
JSON line (milliseconds per application and algorithmic GB/s of the operator). Every
step runs in the library's kernels; nothing here computes the operator.

Cases:
  batch   the multi-right-hand-side Wilson-clover operator (Eq. 2) on one lattice with
          FP16 storage: `cc` the CUDA-core batched kernel, `tc` the tensor-core kernel;
          algorithmic bytes per site: nrhs x (in + out) = nrhs x 104, plus the links
          (4 x 24 B) and clover (148 B) once.
  ptc     one application of a learned preconditioner network of the given channels
          (FP32 fields; `--tensor-cores 0` for the FP32 layers).
  wilson  the full operator M on one right-hand side in the given storage precision
          (algorithmic bytes per site: FP64-18 1536, FP32-12 672, FP16-12 344).
  schwarz the Schwarz preconditioner K (4^4 blocks, 6 minimal-residual steps) in the given
          storage precision; flops per site: 6 x (1872 for M_B + 192 for the MR update and
          the three block reductions).
"""
import argparse
import json

SITE_BYTES = {"f64": 1536, "f32": 672, "f16": 344}
# 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 80.5


def _event_ms(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _lattice(dirac, synth, dims, prec_mask, kappa=0.133, recon=12):
    U = synth.wilson_gauge(dims, 0.5, 3, 4003, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=1.0, recon=(18, recon, recon),
                        prec_mask=prec_mask)
    lat.load_gauge(U)
    return lat


def case_batch(args, dirac, synth):
    import torch
    dims, nrhs = tuple(args.dims), args.nrhs
    lat = _lattice(dirac, synth, dims, (1 << dirac.F64) | (1 << dirac.F16))
    fb = lat.field_bytes(dirac.F16)
    x = torch.empty(nrhs * fb, dtype=torch.uint8, device="cuda")
    for r in range(nrhs):
        lat.import_spinor(x[r * fb:(r + 1) * fb], dirac.F16, -1, synth.wilson_spinor(dims, 4004 + r, device="cuda"))
    y = torch.empty_like(x)
    b = dirac.Batch([lat], [y], [x], [nrhs], dirac.F16)
    kinfo = b.kernel_info()
    if args.kernel == "tc" and kinfo["tensor_core_ms"] < 0:
        raise SystemExit("the tensor-core kernel is not available for this lattice")
    b.set_tensor_cores(args.kernel == "tc")
    ms = _event_ms(b.apply, args.steps, args.warmup)
    alg = lat.volume * (nrhs * 104 + 4 * 24 + 148)
    b.close()
    lat.close()
    return {"case": "batch", "kernel": args.kernel, "dims": dims, "nrhs": nrhs, "ms": round(ms, 4),
            "alg_bytes": alg, "alg_GBps": round(alg / ms / 1e6, 1)}


def case_ptc(args, dirac, synth):
    dims, ch = tuple(args.dims), tuple(args.channels)
    lat = _lattice(dirac, synth, dims, (1 << dirac.F64) | (1 << dirac.F32), kappa=0.1355)
    net = dirac.Ptc(lat, ch)
    net.set_weights([w.numpy() for w in synth.ptc_weights(ch, 5003)])
    net.tensor_cores(bool(args.tensor_cores))
    x = lat.to_device(synth.wilson_spinor(dims, 5002, device="cuda"), dirac.F32)
    y = lat.new_field(dirac.F32)
    ms = _event_ms(lambda: net.apply(y, x), args.steps, args.warmup)
    lat.close()
    return {"case": "ptc", "channels": ch, "tensor_cores": bool(args.tensor_cores), "dims": dims,
            "ms": round(ms, 4)}


def case_wilson(args, dirac, synth):
    dims = tuple(args.dims)
    pid = {"f64": dirac.F64, "f32": dirac.F32, "f16": dirac.F16}[args.prec]
    lat = _lattice(dirac, synth, dims, (1 << dirac.F64) | (1 << pid), kappa=0.135,
                   recon=18 if args.prec == "f64" else 12)
    x = lat.to_device(synth.wilson_spinor(dims, 4004, device="cuda"), pid)
    y = lat.new_field(pid)
    ms = _event_ms(lambda: lat.apply(y, x, dirac.PARITY_FULL, pid), args.steps, args.warmup)
    alg = lat.volume * SITE_BYTES[args.prec]
    lat.close()
    return {"case": "wilson", "prec": args.prec, "dims": dims, "ms": round(ms, 4),
            "alg_GBps": round(alg / ms / 1e6, 1)}


def case_schwarz(args, dirac, synth):
    dims = tuple(args.dims)
    pid = {"f64": dirac.F64, "f32": dirac.F32, "f16": dirac.F16}[args.prec]
    U = synth.wilson_gauge(dims, 0.5, 3, 4003, device="cuda")
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=0.124, csw=1.0, block=(4, 4, 4, 4), mr_steps=6,
                        recon=(18, 12, 12), prec_mask=(1 << dirac.F64) | (1 << pid))
    lat.load_gauge(U)
    x = lat.to_device(synth.wilson_spinor(dims, 4004, device="cuda"), pid)
    y = lat.new_field(pid)
    ms = _event_ms(lambda: lat.schwarz(y, x, pid), args.steps, args.warmup)
    flops = lat.volume * 6 * (1872 + 192)
    lat.close()
    return {"case": "schwarz", "prec": args.prec, "dims": dims, "ms": round(ms, 4),
            "tflops": round(flops / ms / 1e9, 2), "frac_of_fp32_peak": round(flops / ms / 1e9 / FP32_PEAK_TFLOPS, 4)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("case", choices=["batch", "ptc", "wilson", "schwarz"])
    ap.add_argument("--dims", type=int, nargs=4, default=[24, 24, 24, 64])
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--kernel", choices=["cc", "tc"], default="tc")
    ap.add_argument("--channels", type=int, nargs="+", default=[1, 2, 2, 1])
    ap.add_argument("--tensor-cores", type=int, default=1)
    ap.add_argument("--prec", choices=["f64", "f32", "f16"], default="f16")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    args = ap.parse_args(argv)
    from paper_1109_2935_gb300 import dirac, synth
    fn = {"batch": case_batch, "ptc": case_ptc, "wilson": case_wilson, "schwarz": case_schwarz}[args.case]
    print(json.dumps(fn(args, dirac, synth)))


if __name__ == "__main__":
    main()
