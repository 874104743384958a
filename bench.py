"""Benchmark: Wilson-clover dslash HBM GB/s (fraction of the HBM roofline) and solve
seconds to a true residual of 1e-10, mixed precision vs plain FP64.

Workload: the 24^3x128 Wilson-clover lattice (c_sw = 1.0, kappa = 0.1350, random SU(3)
links exp(i sigma H) with sigma = 0.5 followed by 3 APE-like smoothing steps, clover
from the plaquette leaves; Schwarz blocks 4^4 with 6 MR steps). Synthetic, seeded
inputs stand in for the paper's production configurations.

A timed step is one application of the full clover operator M = Ahat - kappa D in the
headline storage precision (FP32 storage, 12-real links). `value` is algorithmic
bytes per application x applications / time. After the timed region the other
precisions are timed the same way and the solves are run (not part of `value`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs the same workload on its own GPU (independent
replicas, weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (24, 24, 24, 128)
KAPPA, CSW, SIGMA, SMEAR = 0.1350, 1.0, 0.5, 3
KAPPA_SOLVE = 0.124          # below the critical kappa of this smoothed field
SEED_GAUGE, SEED_SRC = 2001, 2002
BLOCK, MR_STEPS = (4, 4, 4, 4), 6

# algorithmic bytes per lattice site of one full clover-operator application:
# 4 links (forward; the backward ones belong to neighbours) + spinor in + spinor out + clover
SITE_BYTES = {
    "f64": 4 * 18 * 8 + 24 * 8 + 24 * 8 + 72 * 8,        # 1536 (18-real links)
    "f32": 4 * 12 * 4 + 24 * 4 + 24 * 4 + 72 * 4,        # 672  (12-real links)
    "f16": 4 * 12 * 2 + (48 + 4) * 2 + 72 * 2 + 4,       # 344  (12-real links, norms)
}
SITE_FLOPS = 1872
PREC_ID = {"f64": 0, "f32": 1, "f16": 2}
HEADLINE = "f32"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR (default: the system's temporary directory)
        import tempfile
        out_dir = os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------- CPU oracle
def cpu_info():
    """Host cores this process may use and the CPU model name (best effort)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return cores, model or platform.processor() or platform.machine()


_ORACLE_FIELDS = {}


def _oracle_worker_init(paths):
    """Spawned oracle worker: map the gauge field, source and clover (written once by the
    parent) read-only; no copy per worker."""
    import numpy as np
    for k, path in paths.items():
        _ORACLE_FIELDS[k] = np.load(path, mmap_mode="r")


def _oracle_worker_apply(sites):
    """The oracle's M at a chunk of sites (what one worker does in one step)."""
    from oracle import wilson
    f = _ORACLE_FIELDS
    return wilson.apply_M(f["U"], f["A"], KAPPA, f["psi"], True, sites=sites)


class OracleSample:
    """The FP64 numpy oracle applying M at a fixed random sample of sites of the
    24^3x128 workload, the oracle as it stands: on one core, and on all host cores by a
    spawned process pool that splits the sample into chunks (each worker calls the same
    oracle function on its chunk). Field generation, the clover at the sampled sites and
    the pool start are set-up, outside the timed applications."""

    def __init__(self, n_sites, fields=None):
        import numpy as np
        import torch
        from oracle import wilson
        from oracle.lattice import all_coords
        from paper_1109_2935_gb300 import synth
        if fields is None:
            dev = "cuda" if torch.cuda.is_available() else "cpu"
            U = synth.wilson_gauge(DIMS, SIGMA, SMEAR, SEED_GAUGE, device=dev)
            psi = synth.wilson_spinor(DIMS, SEED_SRC, device=dev)
        else:
            U, psi = fields
        self.U = U.cpu().numpy()
        self.psi = psi.cpu().numpy()
        coords = all_coords(DIMS)
        rng = np.random.default_rng(5)
        self.sites = coords[rng.choice(len(coords), n_sites, replace=False)]
        self.A = np.zeros((DIMS[3], DIMS[2], DIMS[1], DIMS[0], 12, 12), dtype=np.complex128)
        s = self.sites
        self.A[s[:, 3], s[:, 2], s[:, 1], s[:, 0]] = wilson.clover(self.U, CSW, sites=s)
        self.n = n_sites
        self.pool = None
        self.tmp = None
        self.cores, self.cpu_model = cpu_info()

    def step(self):
        """One application on one core; returns its seconds."""
        from oracle import wilson
        t0 = time.perf_counter()
        self.out = wilson.apply_M(self.U, self.A, KAPPA, self.psi, True, sites=self.sites)
        return time.perf_counter() - t0

    def start_pool(self):
        """Write the fields once (the clover as a sparse file: only sampled sites are
        stored) and start one spawned worker per core."""
        import multiprocessing as mp
        import tempfile
        import numpy as np
        base = "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else None
        self.tmp = tempfile.mkdtemp(prefix="oracle_", dir=base)
        paths = {k: os.path.join(self.tmp, k + ".npy") for k in ("U", "psi", "A")}
        np.save(paths["U"], self.U)
        np.save(paths["psi"], self.psi)
        A = np.lib.format.open_memmap(paths["A"], mode="w+", dtype=np.complex128, shape=self.A.shape)
        s = self.sites
        A[s[:, 3], s[:, 2], s[:, 1], s[:, 0]] = self.A[s[:, 3], s[:, 2], s[:, 1], s[:, 0]]
        A.flush()
        del A
        self.chunks = np.array_split(self.sites, 4 * self.cores)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                 initargs=(paths,))

    def step_all_cores(self):
        """One application with every core working on its chunks; returns its seconds."""
        import numpy as np
        t0 = time.perf_counter()
        parts = self.pool.map(_oracle_worker_apply, self.chunks, chunksize=1)
        dt = time.perf_counter() - t0
        self.out_all = np.concatenate(parts)
        return dt

    def close(self):
        import shutil
        if self.pool is not None:
            self.pool.terminate()
            self.pool.join()
            self.pool = None
        if self.tmp:
            shutil.rmtree(self.tmp, ignore_errors=True)
            self.tmp = None


ORACLE_SITES = 65536


def oracle_baseline(orc, steps_one=3, steps_all=5):
    """Time the oracle on one core and on all cores (same sample); the two results must
    agree bit for bit (the same arithmetic per site)."""
    import numpy as np
    orc.step()
    t1 = [orc.step() for _ in range(steps_one)]
    orc.start_pool()
    try:
        orc.step_all_cores()
        ta = [orc.step_all_cores() for _ in range(steps_all)]
        same = bool(np.array_equal(orc.out_all, orc.out.reshape(orc.out_all.shape)))
    finally:
        orc.close()
    one = SITE_BYTES["f64"] * orc.n * len(t1) / sum(t1) / 1e9
    allc = SITE_BYTES["f64"] * orc.n * len(ta) / sum(ta) / 1e9
    sample = (f"FP64 numpy oracle, M at {orc.n} fixed random sites of 24^3x128 per step; all cores: "
              f"{orc.cores} spawned processes on chunks of the sample, {len(ta)} steps ({sum(ta):.2f} s); "
              f"one core: {len(t1)} steps ({sum(t1):.2f} s); FP64 1536 B/site count")
    return {"value": round(allc, 4), "unit": "GB/s", "cores": orc.cores, "kind": "oracle",
            "sample": sample, "cpu_model": orc.cpu_model,
            "one_core": {"value": round(one, 4), "unit": "GB/s", "cores": 1},
            "all_cores_speedup": round(allc / one, 2), "all_cores_equal_one_core": same}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle as the reference arm (rank 0 only), on all of
    the host's cores."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    orc = OracleSample(ORACLE_SITES)
    orc.start_pool()
    try:
        for _ in range(args.warmup):
            orc.step_all_cores()
        times = [orc.step_all_cores() for _ in range(args.steps)]
    finally:
        orc.close()
    tot = sum(times)
    n_sites = orc.n
    value = SITE_BYTES["f64"] * n_sites * len(times) / tot / 1e9
    sample = (f"M at {n_sites} fixed random sites of 24^3x128 per step, FP64 numpy oracle, "
              f"{orc.cores} spawned processes")
    line = {
        "impl": "reference",
        "metric": "Wilson-clover dslash HBM GB/s (algorithmic bytes, % of HBM roofline); "
                  "solve s to true resid 1e-10 vs plain FP64",
        "value": value, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "wilson-clover 24x24x24x128 csw=1.0 kappa=0.135 sigma=0.5 smear=3",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": orc.cores, "kind": "oracle",
                         "sample": sample, "cpu_model": orc.cpu_model},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true", help="skip the solve section")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e timing")
    ap.add_argument("--no-asqtad", action="store_true", help="skip the asqtad rows")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched multi-RHS row")
    ap.add_argument("--no-ptc", action="store_true", help="skip the learned-preconditioner row")
    ap.add_argument("--no-wilson-solve", action="store_true", help="skip the 24^3x128 solves")
    ap.add_argument("--asqtad-dims", type=int, nargs=4, default=[48, 48, 48, 144],
                    help="asqtad lattice (48^3x144 unless profiling a smaller case)")
    ap.add_argument("--dims", type=int, nargs=4, default=list(DIMS),
                    help="lattice extents (profiling cases use a smaller lattice)")
    ap.add_argument("--precs", default="f64,f32,f16", help="precisions to keep and time")
    ap.add_argument("--solve-profile", choices=["gcr_dd", "bicgstab", "bicgstab_eo"],
                    help="run only this mixed solve (FP16 Krylov space and preconditioner) at kappa 0.124 on "
                         "--dims, for a launch list; prints its statistics as one JSON line")
    ap.add_argument("--solve-iters", type=int, default=48, help="iteration budget of --solve-profile")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1109_2935_gb300 import dirac, synth

    if args.solve_profile:
        return solve_profile(args, dirac, synth, dev)
    dims = tuple(args.dims)
    precs = [p for p in args.precs.split(",") if p in PREC_ID]
    if HEADLINE not in precs:
        precs.append(HEADLINE)
    U = synth.wilson_gauge(dims, SIGMA, SMEAR, SEED_GAUGE, device=dev)
    src = synth.wilson_spinor(dims, SEED_SRC, device=dev)
    mask = sum(1 << PREC_ID[p] for p in precs) | 1  # FP64 kept for the solves
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=KAPPA, csw=CSW, block=BLOCK,
                        mr_steps=MR_STEPS, recon=(18, 12, 12), prec_mask=mask)
    lat.load_gauge(U)
    V = lat.volume
    stream = torch.cuda.current_stream(dev)
    fields = {}
    for name in precs:
        pid = PREC_ID[name]
        x = lat.to_device(src, pid)
        y = lat.new_field(pid)
        fields[name] = (x, y)
    torch.cuda.synchronize()

    def time_apply(name, steps, warmup):
        x, y = fields[name]
        pid = PREC_ID[name]
        for _ in range(warmup):
            lat.apply(y, x, dirac.PARITY_FULL, pid, stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev[0].record(stream)
        for i in range(steps):
            lat.apply(y, x, dirac.PARITY_FULL, pid, stream)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - t0
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        return sum(per), per, wall

    peak, peak_kind = _peaks()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    total_ms, per, wall = time_apply(HEADLINE, args.steps, args.warmup)
    clk = clocks.stop()
    total_ms_max = max_over_ranks(world, total_ms, dev)
    bytes_per_launch = SITE_BYTES[HEADLINE] * V
    value = sum_over_ranks(world, bytes_per_launch * args.steps, dev) / (total_ms_max / 1e3) / 1e9
    avg_launch_ms = total_ms / args.steps
    achieved = bytes_per_launch / (avg_launch_ms / 1e3) / 1e9

    # other precisions, same protocol (not part of `value`)
    per_prec = {}
    for name in precs:
        n = max(50, args.steps // 5) if name != "f64" else max(20, args.steps // 20)
        tms, p, _ = time_apply(name, n, 5)
        ms = tms / n
        gbs = SITE_BYTES[name] * V / (ms / 1e3) / 1e9
        per_prec[name] = {"ms": round(ms, 5), "alg_GBps": round(gbs, 1),
                          "frac_of_hbm": round(gbs / peak, 4),
                          "gflops": round(SITE_FLOPS * V / (ms / 1e3) / 1e9, 1)}

    # the other rows of the path on the same lattice: parity dslash, Schwarz K, BLAS
    rows = measure_wilson_rows(lat, dirac, fields, precs, stream, peak)

    # e2e: through the C ABI with host (pinned) natural-layout buffers
    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(lat, dirac, src, fields, stream, args, world, dev, bytes_per_launch)

    # solves (second half of the metric), timed separately
    solves = None
    if not args.no_solve and not args.no_wilson_solve and dims == DIMS:
        solves = run_solves(dirac, synth, U, src, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and dims == DIMS:
        orc = OracleSample(ORACLE_SITES, (U, src))
        cpu = oracle_baseline(orc)
        # M of every precision against the oracle at the same sites (one more launch each):
        # the headline kernel is checked in the run that reports it, and each mixed-
        # precision operator's error against FP64 is reported
        import numpy as np
        s_ = orc.sites
        ref = orc.out.reshape(len(s_), -1)
        bounds = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-2}
        errs = {}
        for name in precs:
            xh, yh = fields[name]
            lat.apply(yh, xh, -1, PREC_ID[name], stream)
            got = lat.to_natural(yh, PREC_ID[name], device="cpu").numpy()
            got = got[s_[:, 3], s_[:, 2], s_[:, 1], s_[:, 0]].reshape(len(s_), -1)
            site = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            errs[name] = {"max_site_rel_err": float(f"{site.max():.3e}"),
                          "rel_l2_err": float(f"{np.linalg.norm(got - ref) / np.linalg.norm(ref):.3e}"),
                          "bound": bounds[name]}
        cpu["error_vs_oracle"] = {"sites": orc.n, "per_precision": errs}
        e = errs[HEADLINE]["max_site_rel_err"]
        cpu["parity_headline"] = {"sites": orc.n, "max_site_rel_err": e, "bound": bounds[HEADLINE],
                                  "ok": bool(e <= bounds[HEADLINE])}
    workload = "wilson-clover %dx%dx%dx%d csw=1.0 kappa=0.135 sigma=0.5 smear=3" % dims
    del fields
    lat.close()
    torch.cuda.empty_cache()
    if not args.no_batch:
        rows["batched_multi_rhs"] = measure_batch(dirac, synth, dev, stream, peak)
        if not args.no_solve:
            rows["batched_solves"] = measure_batched_solves(dirac, synth, dev)
            rows["batched_solves_small_lattices"] = measure_batched_solves(dirac, synth, dev, BATCH_SMALL,
                                                                           BATCH_SMALL_RHS)
    if not args.no_ptc and not args.no_solve:
        rows["ptc_preconditioner"] = measure_ptc(dirac, synth, dev, stream)
    if not args.no_asqtad:
        ad = tuple(args.asqtad_dims)
        rows["asqtad_%dx%dx%dx%d" % ad] = measure_asqtad(dirac, synth, dev, stream, peak,
                                                         not args.no_solve, ad)
    return finish(args, world, rank, dev, value, total_ms_max, achieved, peak, peak_kind,
                  bytes_per_launch, per_prec, clk, e2e, cpu, solves, wall, workload, V, rows)


# FP32 peak for ALU-bound kernels: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# parity dslash, algorithmic bytes per OUTPUT site: 8 links + spinor in + spinor out
HOP_BYTES = {"f64": 8 * 18 * 8 + 2 * 24 * 8, "f32": 8 * 12 * 4 + 2 * 24 * 4,
             "f16": 8 * 12 * 2 + 2 * 52}
# asqtad parity dslash per OUTPUT site: 8 fat (18 reals) + 8 long (18 / 12 / 12) + in + out
STAG_BYTES = {"f64": 8 * 18 * 8 + 8 * 18 * 8 + 2 * 6 * 8, "f32": 8 * 18 * 4 + 8 * 12 * 4 + 2 * 6 * 4,
              "f16": 8 * 18 * 2 + 8 * 12 * 2 + 2 * 16}


def _event_time(fn, n, stream, warm=3):
    import torch
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def measure_wilson_rows(lat, dirac, fields, precs, stream, peak):
    import time as _t
    import torch
    V, Vh = lat.volume, lat.volume // 2
    out = {"dslash_parity": {}, "schwarz": {}, "blas_caxpy_norm": {}}
    for name in precs:
        pid = PREC_ID[name]
        x, y = fields[name]
        hb = lat.field_bytes(pid, 0)
        n = 20 if name == "f64" else 100
        ms = _event_time(lambda: lat.apply(y[:hb], x[hb:], 0, pid, stream), n, stream)
        gbs = HOP_BYTES[name] * Vh / (ms / 1e3) / 1e9
        out["dslash_parity"][name] = {"ms": round(ms, 5), "alg_GBps": round(gbs, 1),
                                      "frac_of_hbm": round(gbs / peak, 4)}
        n = 3 if name == "f64" else 20
        ms = _event_time(lambda: lat.schwarz(y, x, pid, stream), n, stream, warm=1)
        flops = MR_STEPS * (SITE_FLOPS + 192) * V
        tf = flops / (ms / 1e3) / 1e12
        out["schwarz"][name] = {"ms": round(ms, 4), "tflops": round(tf, 2),
                                "frac_of_fp32_peak": round(tf / FP32_PEAK_TFLOPS, 4),
                                "bound": "alu", "flops_per_site": MR_STEPS * (SITE_FLOPS + 192)}
        # BLAS: y += a x with ||y||^2 through the C ABI (includes its stream sync)
        reps = 20
        t0 = _t.perf_counter()
        for _ in range(reps):
            lat.caxpy_norm(1e-3, x, y, pid, stream=stream)
        ms = (_t.perf_counter() - t0) / reps * 1e3
        fb = lat.field_bytes(pid)
        out["blas_caxpy_norm"][name] = {"ms_per_call_incl_sync": round(ms, 4),
                                        "GBps_incl_sync": round(3 * fb / (ms / 1e3) / 1e9, 1)}
    out["schwarz"]["fp32_peak_tflops"] = round(FP32_PEAK_TFLOPS, 1)
    # domain decomposition along t emulated on this GPU (virtual ranks, ghost zones,
    # face exchange by device copies): one application of M, and its bit-exactness
    out["domain_decomposition"] = {}
    for name in precs:
        if name == "f64":
            continue
        pid = PREC_ID[name]
        x, y = fields[name]
        lat.apply(y, x, -1, pid, stream)
        # t-slabs, and grids that cut every dimension (Sec. 6.1-6.3)
        for P in (2, 4, 8, (2, 2, 2, 2), (2, 2, 2, 4)):
            grid = P if isinstance(P, tuple) else (1, 1, 1, P)
            if any(d % (2 * g) for d, g in zip(lat.dims, grid)):
                continue
            dd = dirac.DomainDecomposition(lat, P, pid)
            dd.scatter(x, stream=stream)
            ms = _event_time(lambda: dd.apply(stream=stream), 20, stream)
            g = torch.zeros_like(y)
            dd.gather(g, stream=stream)
            torch.cuda.synchronize()
            gbs = SITE_BYTES[name] * V / (ms / 1e3) / 1e9
            key = f"ranks_{P}" if not isinstance(P, tuple) else "grid_" + "x".join(map(str, P))
            out["domain_decomposition"].setdefault(name, {})[key] = {
                "ms": round(ms, 4), "alg_GBps": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
                "face_bytes": dd.info()["face_bytes"],
                # FP16: the two kernels round the decode product differently (one FP16 ulp)
                "bitwise_equal_single_domain": bool(torch.equal(g, y)) if name != "f16" else None}
            dd.close()
    return out


# links exp(i sigma H) with sigma = 0.5 and no smoothing: the smoothed field of the
# 24^3x128 workload is past its critical point at these kappa (no solver converges there),
# this rougher field is not
BATCH_SMEAR = 0
BATCH_LATTICES = (((16, 16, 16, 32), 0.130, 4001), ((24, 24, 24, 64), 0.133, 4003),
                  ((32, 32, 32, 64), 0.136, 4005))
BATCH_RHS = 12
# bytes per site of one batched application: per right-hand side spinor in + out
# (FP16 52 + 52, FP32 96 + 96), once per site 4 links + the clover (FP16 96 + 148,
# FP32 192 + 288)


def measure_batch(dirac, synth, dev, stream, peak):
    """12 right-hand sides on each of 16^3x32, 24^3x64, 32^3x64 (FP16 storage as
    configured, and FP32): single-RHS launches vs one multi-RHS launch per lattice vs
    one persistent launch over all lattices (autotuned) vs its CUDA-graph replay."""
    return {name: measure_batch_prec(dirac, synth, dev, stream, peak, pid)
            for name, pid in (("f16", dirac.F16), ("f32", dirac.F32))}


def measure_batch_prec(dirac, synth, dev, stream, peak, prec):
    import torch
    pname = "f16" if prec == dirac.F16 else "f32"
    shared = 96 + 148 if prec == dirac.F16 else 192 + 288
    per_rhs = 104 if prec == dirac.F16 else 192
    lats, ins, outs = [], [], []
    for dims, kappa, seed in BATCH_LATTICES:
        U = synth.wilson_gauge(dims, 0.5, BATCH_SMEAR, seed, device=dev)
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=CSW, recon=(18, 12, 12),
                            prec_mask=(1 << dirac.F64) | (1 << prec))
        lat.load_gauge(U)
        fb = lat.field_bytes(prec)
        x = torch.empty(BATCH_RHS * fb, dtype=torch.uint8, device=dev)
        for r in range(BATCH_RHS):
            lat.import_spinor(x[r * fb:(r + 1) * fb], prec, -1,
                              synth.wilson_spinor(dims, seed + 1 + r, device=dev))
        lats.append(lat)
        ins.append(x)
        outs.append(torch.empty_like(x))
    torch.cuda.synchronize()
    sites = sum(l.volume for l in lats)
    alg_bytes = sum(l.volume * (BATCH_RHS * per_rhs + shared) for l in lats)
    single_bytes = sites * BATCH_RHS * SITE_BYTES[pname]

    def single():
        for lat, x, y in zip(lats, ins, outs):
            fb = lat.field_bytes(prec)
            for r in range(BATCH_RHS):
                lat.apply(y[r * fb:(r + 1) * fb], x[r * fb:(r + 1) * fb], dirac.PARITY_FULL, prec, stream)

    def multi():
        for lat, x, y in zip(lats, ins, outs):
            lat.apply_multi(y, x, BATCH_RHS, prec, stream)

    res = {"lattices": [list(d) for d, _, _ in BATCH_LATTICES], "rhs_per_lattice": BATCH_RHS,
           "sites": sites, "alg_bytes_per_application": alg_bytes}
    for name, fn, n in (("single_rhs_launches", single, 10), ("multi_rhs_per_lattice", multi, 20)):
        ms = _event_time(fn, n, stream)
        res[name] = {"ms": round(ms, 4), "site_rhs_per_s": round(sites * BATCH_RHS / (ms / 1e3) / 1e9, 3),
                     "alg_GBps": round(alg_bytes / (ms / 1e3) / 1e9, 1)}
    b = dirac.Batch(lats, outs, ins, [BATCH_RHS] * len(lats), prec, stream)
    ms = _event_time(b.apply, 20, stream)
    res["persistent_batched"] = {"ms": round(ms, 4), **b.info(),
                                 "site_rhs_per_s": round(sites * BATCH_RHS / (ms / 1e3) / 1e9, 3),
                                 "alg_GBps": round(alg_bytes / (ms / 1e3) / 1e9, 1),
                                 "frac_of_hbm": round(alg_bytes / (ms / 1e3) / 1e9 / peak, 4),
                                 "single_rhs_equiv_GBps": round(single_bytes / (ms / 1e3) / 1e9, 1)}
    # both kernels of the plan, each timed on its own: the CUDA-core kernel (one warp per
    # right-hand side) and, with FP16 storage, the tensor-core kernel
    kinfo = b.kernel_info()
    res["persistent_batched"]["tensor_cores"] = kinfo["tensor_cores"]
    kern = {}
    for kname, on in (("cuda_cores", False), ("tensor_cores", True)):
        if on and kinfo["tensor_core_ms"] < 0:
            continue
        b.set_tensor_cores(on)
        kms = _event_time(b.apply, 20, stream)
        kern[kname] = {"ms": round(kms, 4), "alg_GBps": round(alg_bytes / (kms / 1e3) / 1e9, 1),
                       "frac_of_hbm": round(alg_bytes / (kms / 1e3) / 1e9 / peak, 4),
                       "site_rhs_per_s": round(sites * BATCH_RHS / (kms / 1e3) / 1e9, 3)}
    b.set_tensor_cores(kinfo["tensor_cores"])
    res["kernels"] = kern
    napply = 10
    b.capture(napply, stream)
    ms = _event_time(b.apply, 5, stream) / napply
    res["graph_replay"] = {"napply": napply, "ms_per_application": round(ms, 4),
                           "alg_GBps": round(alg_bytes / (ms / 1e3) / 1e9, 1)}
    res["speedup_vs_single_rhs"] = round(res["single_rhs_launches"]["ms"] / res["persistent_batched"]["ms"], 3)
    b.close()
    for lat in lats:
        lat.close()
    return res


# many small lattices (launch-latency territory for one-at-a-time solves)
BATCH_SMALL = (((8, 8, 8, 8), 0.130, 6001), ((8, 8, 8, 12), 0.131, 6003), ((12, 12, 12, 12), 0.132, 6005),
               ((8, 8, 16, 16), 0.133, 6007), ((12, 12, 12, 16), 0.134, 6009), ((16, 16, 16, 16), 0.135, 6011),
               ((8, 8, 8, 16), 0.136, 6013), ((12, 12, 16, 16), 0.130, 6015))
BATCH_SMALL_RHS = 8


def measure_batched_solves(dirac, synth, dev, lattices=None, nrhs_each=None):
    """The batched workload's 36 systems (12 right-hand sides on each lattice) solved to a
    true residual of 1e-10: all together by solve_batched (mixed FP16/FP64 BiCGstab, one
    iteration of every system at a time on the batched operator) vs the same mixed solver
    one system at a time vs plain FP64 BiCGstab one system at a time."""
    import torch
    BATCH_LAT = BATCH_LATTICES if lattices is None else lattices
    BATCH_RHS_N = BATCH_RHS if nrhs_each is None else nrhs_each
    lats, xs, bs = [], [], []
    for dims, kappa, seed in BATCH_LAT:
        U = synth.wilson_gauge(dims, 0.5, BATCH_SMEAR, seed, device=dev)
        lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=kappa, csw=CSW, recon=(18, 12, 12),
                            prec_mask=(1 << dirac.F64) | (1 << dirac.F16))
        lat.load_gauge(U)
        fb = lat.field_bytes(dirac.F64)
        b = torch.empty(BATCH_RHS_N * fb, dtype=torch.uint8, device=dev)
        for r in range(BATCH_RHS_N):
            lat.import_spinor(b[r * fb:(r + 1) * fb], dirac.F64, -1,
                              synth.wilson_spinor(dims, seed + 100 + r, device=dev))
        lats.append(lat)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    torch.cuda.synchronize()
    nrhs = [BATCH_RHS_N] * len(lats)
    out = {"systems": sum(nrhs), "lattices": [list(d) for d, _, _ in BATCH_LAT], "rhs_per_lattice": BATCH_RHS_N,
           "tol": 1e-10, "gauge": "sigma 0.5, no smoothing"}
    t0 = time.perf_counter()
    r = dirac.solve_many(lats, xs, bs, nrhs, tol=1e-10, max_iter=4000, delta=0.1, prec_sloppy=dirac.F16,
                         raise_on_error=False)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    its = [st["iters"] for st in r["rhs"]]
    out["batched_mixed_f16"] = {"status": r["status"], "seconds": round(t_b, 3), "iters_max": max(its),
                                "iters_mean": round(sum(its) / len(its), 1),
                                "worst_true_rel_resid": float("%.3g" % max(st["true_rel_resid"] for st in r["rhs"]))}
    for tag, sp, delta in (("sequential_mixed_f16", dirac.F16, 0.1), ("sequential_plain_f64", dirac.F64, 0.0)):
        tot, itot, worst, status = 0.0, 0, 0.0, "OK"
        for lat, b in zip(lats, bs):
            fb = lat.field_bytes(dirac.F64)
            x = lat.new_field(dirac.F64)
            for k in range(BATCH_RHS_N):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                st = lat.solve(x, b[k * fb:(k + 1) * fb], dirac.BICGSTAB, tol=1e-10, max_iter=4000, delta=delta,
                               prec_sloppy=sp, raise_on_error=False)
                torch.cuda.synchronize()
                tot += time.perf_counter() - t1
                itot += st["iters"]
                worst = max(worst, st["true_rel_resid"])
                if st["status"] != "OK":
                    status = st["status"]
        out[tag] = {"status": status, "seconds": round(tot, 3), "iters_total": itot,
                    "worst_true_rel_resid": float("%.3g" % worst)}
    b_s = out["batched_mixed_f16"]["seconds"]
    out["speedup_vs_sequential_mixed"] = round(out["sequential_mixed_f16"]["seconds"] / b_s, 3)
    out["speedup_vs_plain_f64"] = round(out["sequential_plain_f64"]["seconds"] / b_s, 3)
    for lat in lats:
        lat.close()
    return out


MS_SHIFTS = (0.0, 0.0005, 0.005, 0.05)


def multishift_bench(lat, dirac, b, torch):
    """Eq. 4 with 4 shifts, Sec. 8.2 strategy (FP32 multi-shift CG, then mixed FP64/FP32
    refinement of each solution) vs one mixed FP64/FP32 CG per shift from zero."""
    xs = [lat.new_field(dirac.F64, 0) for _ in MS_SHIFTS]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = lat.solve_multishift(xs, b, list(MS_SHIFTS), dirac.CG_EVEN_NORMAL, tol=1e-10,
                              max_iter=6000, delta=0.1, prec_sloppy=dirac.F32, raise_on_error=False)
    torch.cuda.synchronize()
    t_ms = time.perf_counter() - t0
    out = {"shifts": list(MS_SHIFTS), "status": st["status"], "seconds": round(t_ms, 3),
           "multishift_iters": st["multishift"]["iters"],
           "multishift_seconds": round(st["multishift"]["seconds"], 3),
           "refine_iters": [r["iters"] for r in st["refine"]],
           "true_rel_resid": [float(f"{r['true_rel_resid']:.3g}") for r in st["refine"]]}
    seq_t, seq_it = 0.0, []
    for sgm, x in zip(MS_SHIFTS, xs):
        x.zero_()
        # a single-shift call is one mixed FP64/FP32 CG on (M^dagger M + sigma) from zero
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = lat.solve_multishift([x], b, [sgm], dirac.CG_EVEN_NORMAL, tol=1e-10, max_iter=6000,
                                 delta=0.1, prec_sloppy=dirac.F32, raise_on_error=False)
        torch.cuda.synchronize()
        seq_t += time.perf_counter() - t1
        seq_it.append(r["multishift"]["iters"] + r["refine"][0]["iters"])
    out["sequential_mixed_seconds"] = round(seq_t, 3)
    out["sequential_mixed_iters"] = seq_it
    out["speedup_vs_sequential_mixed"] = round(seq_t / t_ms, 3) if t_ms > 0 else None
    return out


def measure_asqtad(dirac, synth, dev, stream, peak, do_solve, dims):
    """Asqtad parity dslash and even-site normal operator (48^3x144, m = 0.01), and
    CG on (M^dagger M)_ee, mixed FP64/FP32 vs plain FP64. (An FP16 Krylov space
    stagnates near 3e-4 on this operator, so it is not part of the comparison.)"""
    import torch
    fat, lng = synth.asqtad_links(dims, 3001, 3002, device=dev)
    src = synth.staggered_spinor(dims, 3003, device=dev, parity=0)
    lat = dirac.Lattice(dims, dirac.ASQTAD, mass=0.01, recon=(18, 12, 12))
    lat.load_gauge(fat, 1)
    lat.load_gauge(lng, 2)
    del fat, lng
    torch.cuda.empty_cache()
    Vh = lat.volume // 2
    res = {"dslash_parity": {}, "normal_even": {}}
    for name, pid in PREC_ID.items():
        xin = lat.to_device(src, pid, 0)
        yout = lat.new_field(pid, 1)
        n = 10 if name == "f64" else 50
        ms = _event_time(lambda: lat.apply(yout, xin, 1, pid, stream), n, stream)
        gbs = STAG_BYTES[name] * Vh / (ms / 1e3) / 1e9
        res["dslash_parity"][name] = {"ms": round(ms, 4), "alg_GBps": round(gbs, 1),
                                      "frac_of_hbm": round(gbs / peak, 4),
                                      "gflops": round(1146 * Vh / (ms / 1e3) / 1e9, 1)}
        ye = lat.new_field(pid, 0)
        ms = _event_time(lambda: lat.apply_normal(ye, xin, 0, pid, stream), n // 2, stream)
        res["normal_even"][name] = {"ms": round(ms, 4),
                                    "alg_GBps": round(2 * STAG_BYTES[name] * Vh / (ms / 1e3) / 1e9, 1)}
        del xin, yout, ye
    if do_solve:
        b = lat.to_device(src, dirac.F64, 0)
        x = lat.new_field(dirac.F64, 0)
        sol = {}
        for tag, sp, delta in (("cg_mixed_f32", dirac.F32, 0.1), ("cg_f64", dirac.F64, 0.0)):
            torch.cuda.synchronize()
            st = lat.solve(x, b, dirac.CG_EVEN_NORMAL, tol=1e-10, max_iter=4000, delta=delta,
                           prec_sloppy=sp, raise_on_error=False)
            sol[tag] = {k: (float(f"{v:.4g}") if isinstance(v, float) else v) for k, v in st.items()}
        for tag in ("cg_mixed_f32",):
            if sol[tag]["status"] == "OK" and sol["cg_f64"]["status"] == "OK":
                sol[tag + "_speedup_vs_f64"] = round(sol["cg_f64"]["seconds"] / sol[tag]["seconds"], 3)
        res["solve_cg_even_m0.01"] = sol
        res["solve_multishift_m0.01"] = multishift_bench(lat, dirac, b, torch)
    lat.close()
    return res


def time_e2e(lat, dirac, src, fields, stream, args, world, dev, bytes_per_launch):
    import torch
    V = lat.volume
    nat_in = torch.view_as_real(src.cpu()).contiguous().pin_memory()
    nat_out = torch.empty_like(nat_in).pin_memory()
    x, y = fields[HEADLINE]
    pid = PREC_ID[HEADLINE]
    sptr = stream.cuda_stream
    e2e_steps = max(5, min(20, args.steps // 50))

    def e2e_step():
        dirac.dirac_import_spinor(lat.ctx, x.data_ptr(), pid, -1, nat_in.data_ptr(), 0, sptr)
        dirac.dirac_apply(lat.ctx, y.data_ptr(), x.data_ptr(), -1, pid, sptr)
        dirac.dirac_export_spinor(lat.ctx, nat_out.data_ptr(), 0, y.data_ptr(), pid, -1, sptr)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0, dev)
    e2e_value = sum_over_ranks(world, bytes_per_launch * e2e_steps, dev) / e2e_s / 1e9
    nat_bytes = V * 24 * 8
    return {"value": round(e2e_value, 3), "unit": "GB/s", "h2d_bytes_per_step": nat_bytes,
            "d2h_bytes_per_step": nat_bytes, "steps": e2e_steps}


def finish(args, world, rank, dev, value, total_ms_max, achieved, peak, peak_kind,
           bytes_per_launch, per_prec, clk, e2e, cpu, solves, wall, workload, V, rows):
    if rank == 0:
        line = {
            "metric": "Wilson-clover dslash HBM GB/s (algorithmic bytes, % of HBM roofline); "
                      "solve s to true resid 1e-10 vs plain FP64",
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms_max / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload,
                       "op": "full clover M, FP32 storage, 12-real links",
                       "global_batch": world, "parallelism": f"replicas{world}",
                       "l2": "inputs (1.19 GB per application) larger than L2, no flush"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_kind": peak_kind, "traffic": None,
                         "kernel": "wilson_kernel<P32,12,full>",
                         "bytes_per_launch": bytes_per_launch},
            "per_precision": per_prec,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "solve": solves,
            "rows": rows,
            "wall_s_timed": round(wall, 4),
        }
        traffic = _traffic_from_profile(tuple(args.dims))
        if traffic:
            line["roofline"]["traffic"] = traffic
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _traffic_from_profile(dims):
    """DRAM bytes per launch of the headline kernel from the committed ncu summary, or
    None when the summary does not cover this lattice or the kernel sources changed
    since the counters were taken (the summary records a hash of them)."""
    import hashlib
    import re
    src = os.path.join(ROOT, "paper_1109_2935_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("field.cuh", "wilson.cuh"):
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    try:
        with open(os.path.join(ROOT, "profiles", "wilson_clover_M_f32_24x24x24x64.md")) as f:
            text = f.read()
    except OSError:
        return None
    m = re.search(r"csrc/wilson.cuh\): ([0-9a-f]{16})", text)
    t = re.search(r"dram_bytes_per_launch_%dx%dx%dx%d: (\d+)" % dims, text)
    if not m or not t or m.group(1) != h.hexdigest()[:16]:
        return None
    return int(t.group(1))


PTC_DIMS, PTC_KAPPA, PTC_CHANNELS = (16, 16, 16, 16), 0.1355, (1, 2, 2, 1)
PTC_STEPS, PTC_BATCH, PTC_LR = 400, 4, 1e-2


def train_ptc(dirac, synth, dev, kappa):
    """A PTC network trained on the 16^4 field (sigma 0.5, 3 smoothing steps, gauge seed
    5001, source 5002) at `kappa`: pairs v = x* - x_k from GCR-DD iterates x_k of the
    source (x* its 1e-10 solution) plus 8 Gaussian v, r = M v, Adam. Returns the lattice,
    the network and a report."""
    import torch
    U = synth.wilson_gauge(PTC_DIMS, SIGMA, SMEAR, 5001, device=dev)
    lat = dirac.Lattice(PTC_DIMS, dirac.WILSON_CLOVER, kappa=kappa, csw=CSW, block=BLOCK,
                        mr_steps=MR_STEPS, recon=(18, 12, 12))
    lat.load_gauge(U)
    F64, F32, F16 = dirac.F64, dirac.F32, dirac.F16
    b = lat.to_device(synth.wilson_spinor(PTC_DIMS, 5002).to(dev), F64)
    xs = lat.new_field(F64)
    t0 = time.time()
    lat.solve(xs, b, dirac.GCR_DD, tol=1e-10, max_iter=4000, k_max=16, delta=0.1,
              prec_sloppy=F32, prec_precond=F16, raise_on_error=False)
    vs = []
    for k in (2, 4, 8, 16, 32, 64, 128, 256):
        xk = lat.new_field(F64)
        lat.solve(xk, b, dirac.GCR_DD, tol=1e-10, max_iter=k, k_max=16, delta=0.1,
                  prec_sloppy=F32, prec_precond=F16, raise_on_error=False)
        lat.caxpy_norm(-1.0, xs, xk, F64)          # xk <- x_k - x*, the sign is irrelevant
        v = lat.new_field(F32)
        lat.convert(v, F32, xk, F64)
        vs.append(v)
    n_solver = len(vs)
    for i in range(8):
        vs.append(lat.to_device(synth.wilson_spinor(PTC_DIMS, 5100 + i).to(dev), F32))
    make_s = time.time() - t0
    net = dirac.Ptc(lat, PTC_CHANNELS)
    net.set_weights([w.numpy() for w in synth.ptc_weights(PTC_CHANNELS, 5003)])
    torch.cuda.synchronize()
    t0 = time.time()
    loss = net.train(vs, steps=PTC_STEPS, batch=PTC_BATCH, lr=PTC_LR, seed=1)
    torch.cuda.synchronize()
    ttrain = time.time() - t0
    rep = {"lattice": "16x16x16x16", "kappa": kappa, "channels": list(PTC_CHANNELS),
           "pairs": {"solver_iterates": n_solver, "gaussian": len(vs) - n_solver, "make_s": round(make_s, 3)},
           "steps": PTC_STEPS, "batch": PTC_BATCH, "lr": PTC_LR, "seconds": round(ttrain, 4),
           "ms_per_step": round(1e3 * ttrain / PTC_STEPS, 4),
           "loss_first": round(float(loss[0]), 5), "loss_last10": round(float(loss[-10:].mean()), 5)}
    return lat, net, vs, b, rep


def ptc_apply_rates(lat, net, fin, stream, dims):
    """One application of the network: tensor-core (BF16 operands, FP32 accumulation)
    and FP32 CUDA-core layers, nominal flops per site of the layer arithmetic."""
    ch = PTC_CHANNELS
    flops = sum(8 * min(ch[l], ch[l + 1]) * 264 + 9 * ch[l] * ch[l + 1] * 384 for l in range(len(ch) - 1))
    V = dims[0] * dims[1] * dims[2] * dims[3]
    fout = fin.clone()
    out = {"flop_per_site": flops}
    for name, on in (("tensor_cores", True), ("fp32", False)):
        net.tensor_cores(on)
        ms = _event_time(lambda: net.apply(fout, fin, stream=stream), 50, stream)
        tf = flops * V / (ms * 1e-3) / 1e12
        out[name] = {"ms": round(ms, 4), "TFLOPs_nominal": round(tf, 2)}
    out["fp32"]["frac_of_fp32_peak"] = round(out["fp32"]["TFLOPs_nominal"] / FP32_PEAK_TFLOPS, 3)
    out["speedup_tensor_cores"] = round(out["fp32"]["ms"] / out["tensor_cores"]["ms"], 3)
    # the solves that follow use the faster path on this lattice
    fast = out["tensor_cores"]["ms"] < out["fp32"]["ms"]
    net.tensor_cores(fast)
    out["solver_uses"] = "tensor_cores" if fast else "fp32"
    return out


def _solve_row(lat, x, b, alg, sp, pp, budget):
    st = lat.solve(x, b, alg, tol=1e-10, max_iter=budget, k_max=16, delta=0.1, prec_sloppy=sp,
                   prec_precond=pp, raise_on_error=False)
    return {k: (float(f"{v:.4g}") if isinstance(v, float) else v) for k, v in st.items()
            if k in ("status", "iters", "restarts", "reliable_updates", "true_rel_resid", "seconds",
                     "precond", "precond_reduction", "precond_rate", "precond_switches", "precond_calls",
                     "dslash_calls")}


def measure_ptc(dirac, synth, dev, stream):
    """Learned PTC preconditioner on 16^4, kappa 0.1355, c_sw 1.0: training, the
    network's application rate, and GCR with K = network / Schwarz / none against plain
    FP64 GCR and FP64 GCR-DD, all to 1e-10."""
    import torch
    lat, net, vs, b, rep = train_ptc(dirac, synth, dev, PTC_KAPPA)
    F64, F32, F16 = dirac.F64, dirac.F32, dirac.F16
    out = {"workload": "16x16x16x16 csw=1.0 kappa=0.1355 sigma=0.5 smear=3", "train": rep}
    out["apply"] = ptc_apply_rates(lat, net, vs[-1], stream, PTC_DIMS)
    res = {}
    runs = [("gcr_f64", dirac.GCR, F64, F64, None), ("gcr_dd_f64", dirac.GCR_DD, F64, F64, None),
            ("gcr_mixed", dirac.GCR, F32, F32, None), ("gcr_dd_mixed", dirac.GCR_DD, F32, F16, None),
            ("gcr_ptc_mixed", dirac.GCR_PTC, F32, F32, True),
            ("gcr_ptc_select_mixed", dirac.GCR_PTC, F32, F16, False)]
    for name, alg, sp, pp, force in runs:
        if force is not None:
            net.attach(force=force)
        torch.cuda.synchronize()
        res[name] = _solve_row(lat, lat.new_field(F64), b, alg, sp, pp, 4000)
    for name in ("gcr_mixed", "gcr_dd_mixed", "gcr_ptc_mixed", "gcr_ptc_select_mixed"):
        r = res[name]
        for ref in ("gcr_f64", "gcr_dd_f64"):
            if r["status"] == "OK" and res[ref]["status"] == "OK":
                r[f"speedup_vs_{ref}"] = round(res[ref]["seconds"] / r["seconds"], 3)
        if r["status"] == "OK" and res["gcr_dd_mixed"]["status"] == "OK":
            r["iters_vs_gcr_dd_mixed"] = round(r["iters"] / res["gcr_dd_mixed"]["iters"], 3)
            r["speedup_vs_gcr_dd_mixed"] = round(res["gcr_dd_mixed"]["seconds"] / r["seconds"], 3)
    out["solves"] = res
    net.close()
    lat.close()
    return out


def solve_profile(args, dirac, synth, dev):
    """One mixed solve of the bench workload with a bounded iteration budget, so that a
    launch list covers whole solver steps (restarts and reliable updates included)."""
    import torch
    dims = tuple(args.dims)
    alg = {"gcr_dd": dirac.GCR_DD, "bicgstab": dirac.BICGSTAB, "bicgstab_eo": dirac.BICGSTAB_EO}[args.solve_profile]
    lat = dirac.Lattice(dims, dirac.WILSON_CLOVER, kappa=KAPPA_SOLVE, csw=CSW, block=BLOCK,
                        mr_steps=MR_STEPS, recon=(18, 12, 12))
    lat.load_gauge(synth.wilson_gauge(dims, SIGMA, SMEAR, SEED_GAUGE, device=dev))
    b = lat.to_device(synth.wilson_spinor(dims, SEED_SRC, device=dev), dirac.F64)
    x = lat.new_field(dirac.F64)
    torch.cuda.synchronize()
    st = lat.solve(x, b, alg, tol=1e-10, max_iter=args.solve_iters, k_max=16, delta=0.1,
                   prec_sloppy=dirac.F16, prec_precond=dirac.F16, raise_on_error=False)
    torch.cuda.synchronize()
    print(json.dumps({"solve_profile": args.solve_profile, "dims": list(dims), "kappa": KAPPA_SOLVE,
                      "stats": {k: (float(f"{v:.4g}") if isinstance(v, float) else v) for k, v in st.items()}}))
    lat.close()
    return 0


def run_solves(dirac, synth, U, src, dev):
    """Mixed-precision vs plain-FP64 solves on the same 24^3x128 field."""
    import torch
    out = {}
    for kappa, tag, budget, gcr_budget in ((KAPPA_SOLVE, "kappa_0.124", 4000, 1000),
                                           (KAPPA, "kappa_0.135", 600, 2000)):
        lat = dirac.Lattice(DIMS, dirac.WILSON_CLOVER, kappa=kappa, csw=CSW, block=BLOCK,
                            mr_steps=MR_STEPS, recon=(18, 12, 12))
        lat.load_gauge(U)
        b = lat.to_device(src, dirac.F64)
        x = lat.new_field(dirac.F64)
        res = {}
        runs = [("gcr_f64", dirac.GCR, dirac.F64, dirac.F64, 0.0),
                ("gcr_dd_mixed", dirac.GCR_DD, dirac.F16, dirac.F16, 0.1),
                ("gcr_dd_f64", dirac.GCR_DD, dirac.F64, dirac.F64, 0.0),
                ("bicgstab_mixed", dirac.BICGSTAB, dirac.F16, dirac.F16, 0.1),
                ("bicgstab_f64", dirac.BICGSTAB, dirac.F64, dirac.F64, 0.0),
                ("bicgstab_eo_mixed", dirac.BICGSTAB_EO, dirac.F16, dirac.F16, 0.1),
                ("bicgstab_eo_f64", dirac.BICGSTAB_EO, dirac.F64, dirac.F64, 0.0)]
        for name, alg, sp, pp, delta in runs:
            if kappa == KAPPA and name.endswith("f64"):
                continue
            torch.cuda.synchronize()
            st = lat.solve(x, b, alg, tol=1e-10, max_iter=budget if alg not in (dirac.GCR_DD, dirac.GCR) else gcr_budget,
                           k_max=16, delta=delta, prec_sloppy=sp, prec_precond=pp, raise_on_error=False)
            res[name] = {k: (float(f"{v:.4g}") if isinstance(v, float) else v) for k, v in st.items()}
        # learned preconditioner: weights trained on the 16^4 field at the same kappa
        plat, pnet, _, _, rep = train_ptc(dirac, synth, dev, kappa)
        w = pnet.get_weights()
        plat.close()
        net = dirac.Ptc(lat, PTC_CHANNELS)
        net.set_weights(w)
        res["ptc_apply"] = ptc_apply_rates(lat, net, lat.to_device(src, dirac.F32), torch.cuda.current_stream(),
                                           DIMS)
        # forced network (FP32 Krylov space, as the network's layers); adaptive choice between
        # the network and the FP16 Schwarz preconditioner with the FP16 Krylov space of GCR-DD
        for name, force, sp, pp in (("gcr_ptc_mixed", True, dirac.F32, dirac.F32),
                                    ("gcr_ptc_select_mixed", False, dirac.F16, dirac.F16)):
            net.attach(force=force)
            torch.cuda.synchronize()
            res[name] = _solve_row(lat, x, b, dirac.GCR_PTC, sp, pp, gcr_budget)
            res[name]["trained_on"] = rep
        for alg in ("gcr_dd", "bicgstab", "bicgstab_eo", "gcr_ptc", "gcr_ptc_select"):
            a, b_ = res.get(f"{alg}_mixed"), res.get(f"{alg}_f64") or res.get("gcr_dd_f64")
            if a and b_ and a["status"] == "OK" and b_["status"] == "OK":
                res[f"{alg}_speedup_vs_f64"] = round(b_["seconds"] / a["seconds"], 3)
            g = res.get("gcr_f64")
            if a and g and a["status"] == "OK" and g["status"] == "OK":
                res[f"{alg}_speedup_vs_plain_gcr_f64"] = round(g["seconds"] / a["seconds"], 3)
        out[tag] = res
        lat.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
