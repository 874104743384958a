/*
 * dirac.h -- C ABI of libdirac, a single-GPU (sm_103a) implementation of the solver
 * hot path of "Scaling Lattice QCD beyond 100 GPUs" (Babich et al., SC11):
 * the Wilson-clover and improved-staggered (asqtad) Dirac operators, the
 * non-overlapping additive Schwarz preconditioner, and the Krylov solvers around
 * them (CG, BiCGstab, mixed-precision GCR-DD of Algorithm 1).
 *
 * Problem statement (Sec. 2.1, Eq. 1): solve M x = b for a large sparse M.
 *
 * General rules
 *  - Every function returns an int status: DIRAC_OK (0) or a negative DIRAC_ERR_*.
 *    No function aborts, exits or throws across this boundary. After an error,
 *    dirac_last_error(ctx) holds a one-line description.
 *  - All GPU work is enqueued on the stream argument (a cudaStream_t passed as
 *    void*; NULL means the legacy default stream). Functions that return host
 *    values (reductions, solve) synchronise that stream before returning.
 *  - Spinor arguments are CALLER-OWNED DEVICE POINTERS in the library's device
 *    layout (below); sizes come from dirac_field_bytes(). Input and output of one
 *    call must not alias. Gauge and clover fields are copied into library-owned
 *    device storage by dirac_load_gauge and live until dirac_destroy.
 *  - One context is used by one host thread at a time.
 *
 * Natural (host-application) layout, FP64, x fastest and t slowest (Sec. 6.2):
 *    links   [t][z][y][x][mu][3][3][re,im]     mu = 0,1,2,3 = x,y,z,t
 *    Wilson spinor    [t][z][y][x][spin 4][colour 3][re,im]
 *    staggered spinor [t][z][y][x][colour 3][re,im]
 *
 * Device layout of a spinor field (Sec. 5: fields reordered for coalescing;
 * Sec. 6.1 / Fig. 2: Vh = V/2 sites per parity):
 *    a parity half-field holds the Vh sites of one parity in checkerboard order
 *    cb = lex/2 (lex = ((t*LZ + z)*LY + y)*LX + x, parity = (x+y+z+t) mod 2);
 *    it is an array of 16-byte (F64 Wilson/staggered, F32 Wilson, F16 Wilson),
 *    8-byte (F32 staggered) or 4-byte (F16 staggered) chunks, chunk-major:
 *    chunk k of site cb sits at  base + (k*Vh + cb) * chunk_bytes,
 *    and the reals of a site are ordered (spin, colour, re/im). F16 fields hold
 *    binary16 values of v/n followed by Vh FP32 per-site norms n = max|v|.
 *    A full field is the even half-field followed by the odd half-field.
 */
#ifndef DIRAC_H
#define DIRAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dirac_ctx dirac_ctx;

enum {
  DIRAC_OK = 0,
  DIRAC_ERR_ARG = -1,           /* invalid argument (sizes, enums, null pointers) */
  DIRAC_ERR_CUDA = -2,          /* a CUDA call failed; the message names it */
  DIRAC_ERR_OOM = -3,           /* device allocation failed */
  DIRAC_ERR_UNSUPPORTED = -4,   /* operation not defined for this operator/precision */
  DIRAC_ERR_NOT_CONVERGED = -5, /* max_iter reached; x holds the last iterate */
  DIRAC_ERR_BREAKDOWN = -6,     /* a Krylov denominator vanished */
  DIRAC_ERR_NONFINITE = -7,     /* NaN/Inf in a residual norm */
  DIRAC_ERR_TIMEOUT = -8,       /* reserved: a bounded device wait ran out */
  DIRAC_ERR_STATE = -9          /* e.g. apply before the gauge field was loaded */
};

typedef enum { DIRAC_WILSON_CLOVER = 0, DIRAC_ASQTAD = 1 } dirac_kind;
typedef enum { DIRAC_PREC_F64 = 0, DIRAC_PREC_F32 = 1, DIRAC_PREC_F16 = 2 } dirac_prec;
/* Gauge compression, Sec. 5 strategy (a): reals stored per SU(3) link. */
typedef enum { DIRAC_RECON_18 = 18, DIRAC_RECON_12 = 12, DIRAC_RECON_8 = 8 } dirac_recon;
/* Output parity: FULL = whole lattice, EVEN/ODD = one checkerboard. */
typedef enum { DIRAC_PARITY_FULL = -1, DIRAC_PARITY_EVEN = 0, DIRAC_PARITY_ODD = 1 } dirac_parity;

typedef struct {
  int dims[4];          /* LX, LY, LZ, LT: each even, >= 2 */
  int t_antiperiodic;   /* 1: fermion hops across the t boundary get a factor -1 */
  dirac_kind kind;
  double kappa;         /* Wilson-clover hopping parameter, kappa = 1/(2(4+m)) (Eq. 2) */
  double csw;           /* clover coefficient; 0 = plain Wilson */
  double mass;          /* asqtad mass m (Eq. 3) */
  int block[4];         /* Schwarz block extents; each divides dims; block volume <= 256 */
  int mr_steps;         /* minimal-residual steps per block solve (Sec. 8.1) */
  int recon[3];         /* dirac_recon per precision F64/F32/F16 for the Wilson links and
                           the asqtad long links (fat links are always 18: not unitary) */
  unsigned prec_mask;   /* bit p set: keep the operator in precision p (0 = all three) */
} dirac_params;

/* Create a context for one lattice. Allocates the library-owned gauge/clover storage
 * lazily at dirac_load_gauge. Returns DIRAC_ERR_ARG for odd or non-positive dims,
 * blocks that do not tile the lattice, or unknown enums. */
int dirac_create(const dirac_params* params, dirac_ctx** out);
int dirac_destroy(dirac_ctx* ctx);
const char* dirac_last_error(const dirac_ctx* ctx);

/* Bytes of one spinor field in the device layout for precision/parity. */
size_t dirac_field_bytes(const dirac_ctx* ctx, dirac_prec prec, dirac_parity parity);

/* Load a gauge field given in the natural FP64 layout (host or device memory,
 * on_device = 0/1) and convert it on the GPU into every precision of prec_mask with
 * that precision's compression. which = 0: Wilson links U (also builds the clover
 * term A of Eq. 2 from the plaquette leaves, and stores 1 + 2 kappa A); 1: asqtad fat
 * links; 2: asqtad long links (Eq. 3). The caller keeps ownership of `links`. */
int dirac_load_gauge(dirac_ctx* ctx, const double* links, int which, int on_device, void* stream);

/* Convert a spinor between the natural FP64 layout (host or device) and the device
 * layout of precision `prec`. For a parity half-field only the sites of that parity
 * are read (import) or written (export); the natural array always spans the lattice.
 * With FP64 or FP32 storage, a host array in page-locked memory (or any host memory
 * where the GPU uses the host's page tables) is accessed in place by the conversion
 * kernel; other host memory, and FP16 storage, go through a device staging copy. Calls with a host array return after it has been
 * read / written. */
int dirac_import_spinor(dirac_ctx* ctx, void* dst, dirac_prec prec, dirac_parity parity,
                        const double* src_natural, int src_on_device, void* stream);
int dirac_export_spinor(dirac_ctx* ctx, double* dst_natural, int dst_on_device,
                        const void* src, dirac_prec prec, dirac_parity parity, void* stream);

/* out = M in (Eq. 2 in kappa form M = 1 + 2 kappa A - kappa D; Eq. 3 M = m - D/2) on
 * full fields when parity == FULL. With parity EVEN/ODD: out_p = D_{p,1-p} in_{1-p},
 * the hopping block of D alone (half-fields in and out). `in` and `out` are device
 * fields of precision `prec`; the operator runs in that precision. */
int dirac_apply(dirac_ctx* ctx, void* out, const void* in, dirac_parity parity, dirac_prec prec,
                void* stream);
/* Same with the adjoint: Wilson gamma5 M gamma5 (projectors swapped), asqtad m + D/2
 * (parity form: D^dagger = -D). */
int dirac_apply_dagger(dirac_ctx* ctx, void* out, const void* in, dirac_parity parity,
                       dirac_prec prec, void* stream);
/* The Wilson-clover M (dagger = 1: M^dagger) on FP64 full fields, evaluated in
 * double-single arithmetic (pairs of binary32 values, about 48 significant bits; the
 * sum and product steps are exact error-free transformations): agrees with the FP64
 * dirac_apply to ~1e-14 relative and runs on the FP32 pipes. When switched on, solve()
 * uses it for the FP64 true residuals of its restarts and reliable updates (Sec. 8.2 keeps
 * only those, the solution and the global sums above the sloppy precision); a residual it
 * finds below the tolerance, and the final residual of every solve, are recomputed with
 * the FP64 operator. DIRAC_ERR_UNSUPPORTED unless Wilson-clover with 18-real FP64 links.
 * dirac_set_ds_residual(ctx, 1) makes solve() and solve_batched() use it for those
 * residuals; the default (0) is the FP64 operator throughout, which measured faster. */
int dirac_apply_ds(dirac_ctx* ctx, void* out, const void* in, int dagger, void* stream);
int dirac_set_ds_residual(dirac_ctx* ctx, int on);

/* Normal operator M^dagger M. FULL: whole lattice (both kinds). EVEN/ODD: asqtad
 * only, (M^dagger M)_pp = m^2 - 1/4 D_{p,1-p} D_{1-p,p} on a half-field (Sec. 3.1:
 * the staggered normal matrix decouples the parities). */
int dirac_apply_normal(dirac_ctx* ctx, void* out, const void* in, dirac_parity parity,
                       dirac_prec prec, void* stream);

/* Even-odd (Schur complement) form of the Wilson-clover operator (Sec. 3.1: even-odd
 * preconditioning, solving the Schur complement system): on EVEN half-fields
 *     out = Ahat_ee in - kappa^2 D_eo Ahat_oo^-1 D_oe in      (dagger = 1: the adjoint)
 * with Ahat^-1 built alongside Ahat by dirac_load_gauge. Wilson-clover only. */
int dirac_apply_eo(dirac_ctx* ctx, void* out, const void* in, dirac_prec prec, int dagger, void* stream);

/* Batched Wilson-clover operator (many right-hand sides, several lattices per launch).
 * The paper applies M to one right-hand side at a time; batching reuses each site's
 * links and clover across the right-hand sides of a tile (read from DRAM once).
 *
 * dirac_apply_multi: out_r = M in_r for r < nrhs on one lattice; in and out each hold
 * nrhs consecutive full fields (dirac_field_bytes(ctx, prec, FULL) apart), no overlap.
 *
 * dirac_batch_create: a plan applying M of ctxs[l] to nrhs[l] consecutive full fields
 * in[l] -> out[l] for l < nlat (1..16 lattices of any sizes; one precision, the same
 * link compression) in ONE persistent launch. Creating the plan autotunes the tile
 * shape (right-hand sides per CTA x resident CTAs per SM) by timing each candidate on
 * `stream` (it writes `out`), then synchronises. dirac_batch_capture records napply
 * launches in a CUDA graph; afterwards dirac_batch_apply replays the graph (napply
 * applications) instead of one direct launch. The plan keeps the pointers it was given. */
typedef struct dirac_batch dirac_batch;
int dirac_apply_multi(dirac_ctx* ctx, void* out, const void* in, int nrhs, dirac_prec prec, void* stream);
int dirac_batch_create(dirac_ctx* const* ctxs, int nlat, void* const* out, const void* const* in,
                       const int* nrhs, dirac_prec prec, void* stream, dirac_batch** plan);
int dirac_batch_apply(dirac_batch* plan, void* stream);
int dirac_batch_capture(dirac_batch* plan, int napply, void* stream);
int dirac_batch_info(const dirac_batch* plan, int* rhs_per_cta, int* ctas_per_sm, int* grid,
                     double* tuned_ms);
int dirac_batch_destroy(dirac_batch* plan);
/* Tensor-core form of the batched operator, for FP16 storage with 12- or 18-real links
 * (not in the paper: a multi-right-hand-side extension). Per site the link-times-
 * spinor products of all right-hand sides of a tile are one dense contraction (Eq. 2:
 * rows = right-hand sides, K = 8 spin-projected hops x 3 colours, columns = colour) run
 * with FP16 operands and FP32 accumulation on the tensor cores, the clover blocks as a
 * fourth k-tile; results agree with dirac_apply in FP16 within the FP16 per-site bound,
 * not bit for bit. dirac_batch_create times it beside the CUDA-core kernel and keeps the
 * faster one. dirac_batch_set_tensor_cores selects it (1) or the CUDA-core kernel (0);
 * DIRAC_ERR_UNSUPPORTED when the plan has no tensor-core form; a captured graph is
 * dropped (capture again). dirac_batch_kernel_info reports the kernel in use and the
 * creation timings in ms (-1: not timed). */
int dirac_batch_set_tensor_cores(dirac_batch* plan, int on);
int dirac_batch_kernel_info(const dirac_batch* plan, int* tensor_cores, double* cuda_core_ms,
                            double* tensor_core_ms);

/* out = K in: the non-overlapping additive Schwarz preconditioner of Sec. 3.2 / 8.1
 * for the Wilson-clover operator. On every block (params.block) the operator with
 * Dirichlet (zero) block boundaries is solved by params.mr_steps minimal-residual
 * steps from x = 0, with block-local inner products. Full fields of precision
 * `prec`. DIRAC_ERR_UNSUPPORTED for asqtad. */
int schwarz_precondition(dirac_ctx* ctx, void* out, const void* in, dirac_prec prec, void* stream);

/* BLAS-1 on device fields (Sec. 6.1: contiguous fields make BLAS and reductions
 * straightforward). All accumulate in FP64; results are returned to host memory
 * after a stream synchronisation. dot = sum conj(x_i) y_i. */
int dirac_norm2(dirac_ctx* ctx, const void* x, dirac_prec prec, dirac_parity parity,
                double* result, void* stream);
int dirac_cdot(dirac_ctx* ctx, const void* x, const void* y, dirac_prec prec,
               dirac_parity parity, double result[2], void* stream);
/* y += a x, then result = ||y||^2 (a complex: a_re + i a_im). */
int dirac_caxpy_norm(dirac_ctx* ctx, double a_re, double a_im, const void* x, void* y,
                     dirac_prec prec, dirac_parity parity, double* result, void* stream);
/* dst (precision dprec) = src (precision sprec), element-wise with re-encoding. */
int dirac_convert(dirac_ctx* ctx, void* dst, dirac_prec dprec, const void* src, dirac_prec sprec,
                  dirac_parity parity, void* stream);

/* Allocation-free inner product, for callers that must not allocate GPU memory.
 * (The paper has no counterpart; this is a library-usage addition.)
 * Who needs it: a host application that has already handed all of the GPU's memory
 * to its own pool allocator, or that calls in from a stream-ordered section where a
 * cudaMalloc would implicitly synchronise the device and stall its other streams,
 * cannot create a dirac_ctx (dirac_create allocates its reduction scratch). This
 * entry point needs no context and allocates nothing: it computes
 *     result[0] + i result[1] = (x, y) = sum conj(x_i) y_i,   result[2] = ||x||^2
 * for two spinor fields in the device layout (reals_per_site 24 Wilson or 6
 * staggered; sites_per_parity = Vh; parity FULL for a full field), accumulating in
 * FP64 like dirac_cdot, and writes the three doubles to the caller's DEVICE pointer
 * `result` without synchronising the stream.
 * Scratch: a fixed 98,312-byte device array inside the library (every GPU that loads
 * the library holds it until the process exits). One call covers at most 8,388,608
 * sites (npar * sites_per_parity); larger fields are rejected with DIRAC_ERR_ARG and
 * a message in `err` (err may be NULL; err_len bytes including the terminator).
 * x, y and result must be device (or managed) memory; a host pointer is rejected with
 * DIRAC_ERR_ARG before anything is queued. An error already pending from earlier
 * asynchronous work is reported (DIRAC_ERR_CUDA, left pending) and nothing is queued.
 * Every call shares the array: calls that overlap on the GPU (other streams or other
 * host threads) race and give wrong results; serialise them. The first call on each
 * device looks up the array's device address (once per device and CUDA context, with
 * that device current; again after a device reset); make that first call before any
 * stream capture. */
int dirac_cdot_noalloc(const void* x, const void* y, dirac_prec prec, int reals_per_site,
                       long long sites_per_parity, dirac_parity parity, double* result,
                       void* stream, char* err, size_t err_len);

typedef enum {
  DIRAC_SOLVER_CG_NORMAL = 0,      /* CG on M^dagger M x = b, full lattice (Sec. 3.1) */
  DIRAC_SOLVER_CG_EVEN_NORMAL = 1, /* CG on (M^dagger M)_ee x_e = b_e, asqtad (Sec. 3.1) */
  DIRAC_SOLVER_BICGSTAB = 2,       /* BiCGstab on M x = b, Wilson-clover (Sec. 3.1) */
  DIRAC_SOLVER_GCR_DD = 3,         /* GCR with the Schwarz preconditioner (Algorithm 1) */
  DIRAC_SOLVER_GCR = 4,            /* GCR of Algorithm 1 with K = 1 */
  DIRAC_SOLVER_BICGSTAB_EO = 5,    /* BiCGstab on the even-odd Schur system (Sec. 3.1), then
                                      x_o = Ahat_oo^-1 (b_o + kappa D_oe x_e); x, b full fields */
  DIRAC_SOLVER_GCR_EO = 6,         /* unpreconditioned GCR on the even-odd Schur system */
  DIRAC_SOLVER_GCR_PTC = 7         /* GCR of Algorithm 1 with K = the attached PTC network, or
                                      the Schwarz preconditioner when that reduces the
                                      initial residual more (dirac_ptc_attach) */
} dirac_solver;

typedef struct {
  dirac_solver alg;
  double tol;           /* target ||b - A x|| / ||b|| of the solved system, in FP64 */
  int max_iter;         /* Krylov iterations (GCR: preconditioned directions) */
  int k_max;            /* GCR Krylov subspace size (Algorithm 1) */
  double delta;         /* GCR: restart when ||r_k||/||r_0|| < delta (0 = off);
                           CG/BiCGstab: reliable update when ||r|| < delta * max ||r||
                           since the last update (0 = pure, no updates) */
  int use_x0;           /* 1: x holds the initial guess on entry */
  dirac_prec prec_sloppy;  /* precision of the Krylov vectors and the inner operator */
  dirac_prec prec_precond; /* precision of the Schwarz preconditioner (GCR_DD) */
} dirac_solver_params;

typedef struct {
  int iters, restarts, reliable_updates, dslash_calls, precond_calls;
  double true_rel_resid;   /* final ||b - A x|| / ||b|| recomputed in FP64 */
  double seconds;          /* wall time of the solve including the final sync */
  double flops;            /* operator + preconditioner + BLAS flops from per-site counts */
  int precond_kind;        /* preconditioner of the last cycle: 0 none, 1 Schwarz, 2 PTC */
  double precond_reduction[2]; /* GCR_PTC: ||r0 - M K r0|| / ||r0|| of K = Schwarz, PTC (the
                                  test that picks the first cycle's preconditioner) */
  double precond_rate[2];  /* GCR_PTC: last measured residual reduction per second
                              (ln ||r|| per second) of K = Schwarz, PTC; -1 if never run */
  int precond_switches;    /* GCR_PTC: changes of preconditioner at restarts */
} dirac_solver_stats;

/* Solve A x = b in FP64 (A = M, M^dagger M or (M^dagger M)_ee per alg). x and b are
 * caller-owned FP64 device fields (full fields, or EVEN half-fields for
 * CG_EVEN_NORMAL). Returns DIRAC_OK when the FP64 true residual meets tol,
 * DIRAC_ERR_NOT_CONVERGED when max_iter ran out (x = last iterate, stats filled). */
int solve(dirac_ctx* ctx, void* x, const void* b, const dirac_solver_params* params,
          dirac_solver_stats* stats, void* stream);

/* Batched solves (not in the paper: the multi-right-hand-side extension of solve):
 * M_l x_{l,r} = b_{l,r} for r < nrhs[l] on nlat (1..16) Wilson-clover lattices of any
 * sizes, at most 256 right-hand sides in all. x[l] and b[l] hold nrhs[l] consecutive
 * FP64 full fields (caller-owned device memory; x is read as the initial guess iff
 * params->use_x0). Every right-hand side runs its own BiCGstab (params->alg must be
 * DIRAC_SOLVER_BICGSTAB) with reliable updates every params->delta in
 * params->prec_sloppy, to params->tol; one iteration of all of them is one batched
 * operator application per BiCGstab operator step (the CUDA-core batched kernel),
 * single BLAS launches over all right-hand sides and a replayed CUDA graph. A reliable
 * update recomputes the FP64 residual of the right-hand sides that ask for one only; a
 * converged right-hand side is skipped by every later launch and stops changing while the
 * others continue; each right-hand side's result (bytes, iterations, reliable updates) is
 * that of solving it alone. stats: one entry per
 * right-hand side (lattice-major): its iterations, reliable updates and final FP64 true
 * residual; seconds is the wall time of the whole call. Returns DIRAC_ERR_NOT_CONVERGED
 * (or BREAKDOWN / NONFINITE) if some right-hand side did not reach tol; the others keep
 * their solutions. Synchronises stream. */
int solve_batched(dirac_ctx* const* ctxs, int nlat, void* const* x, const void* const* b, const int* nrhs,
                  const dirac_solver_params* params, dirac_solver_stats* stats, void* stream);

/* Multi-shift solve of Eq. 4, (M^dagger M + sigma_j) x_j = b for j < nshift (1..16,
 * sigma_j >= 0), the strategy of Sec. 8.2: a multi-shift CG in params->prec_sloppy
 * builds one Krylov space for every shift (down to a relative residual of 1e-6 in
 * FP32, 1e-3 in FP16), then each x_j is refined by mixed-precision CG on its own
 * system, warm-started, with reliable updates every params->delta, to params->tol.
 * params->alg: DIRAC_SOLVER_CG_EVEN_NORMAL (asqtad, even half-fields) or
 * DIRAC_SOLVER_CG_NORMAL (full fields). x: nshift distinct FP64 device fields
 * (outputs); b: FP64 device field. stats (may be NULL): nshift + 1 entries, [0] the
 * multi-shift stage, [1 + j] the refinement of shift j (true_rel_resid of shift j).
 * Returns DIRAC_ERR_NOT_CONVERGED if some refinement ran out of iterations. */
int solve_multishift(dirac_ctx* ctx, void* const* x, const void* b, const double* shifts, int nshift,
                     const dirac_solver_params* params, dirac_solver_stats* stats, void* stream);

/* ------------------------------------------------------------------ learned preconditioner
 * A gauge-equivariant parallel-transport convolution (PTC) network K, a learned
 * preconditioner for the flexible GCR of Algorithm 1 (whose outer iteration accepts any
 * preconditioner, Sec. 3.2). The paper has no such network: this is an extension. Layer
 * l maps channels_in = channels[l-1] spinor fields to channels[l] fields:
 *   out_c(x) = sum_c' sum_p W_l[p][c][c'] (T_p in_c')(x),  p = 0, +x, -x, +y, ..., -t
 *   T_0 = 1, (T_+mu f)(x) = U_mu(x) f(x+mu), (T_-mu f)(x) = U_mu(x-mu)^dagger f(x-mu)
 * with W a complex 4x4 spin matrix (colour untouched, so K commutes with gauge
 * transformations), the fermion boundary sign on hops across an antiperiodic t edge,
 * and no nonlinearity (K is linear). Weights are FP32 complex, stored per layer as
 * [p (9)][c_out][c_in][s (4)][s' (4)], (re, im) interleaved; on the host they are
 * passed as FP64 (re, im) pairs in the same order, layers consecutive.
 * Fields are FP32 full fields in the device layout of the context (dirac_field_bytes
 * with DIRAC_PREC_F32, parity FULL); the context must keep FP32 (prec_mask bit 1) and
 * be a Wilson-clover context with its gauge field loaded. */
typedef struct dirac_ptc dirac_ptc;
typedef struct {
  int layers;          /* 1..4 */
  int channels[5];     /* channels[0] = channels[layers] = 1; the others 1, 2 or 4 */
} dirac_ptc_params;

typedef struct {
  int steps;           /* Adam steps */
  int batch;           /* pairs per step, 1..16 */
  double lr, beta1, beta2, eps;  /* Adam (Kingma and Ba): step lr, moment decays, eps */
  unsigned seed;       /* order in which pairs are visited (epochs reshuffled) */
} dirac_ptc_train_params;

/* Create a network on ctx whose layers pass channel 0 through on the local path (K = 1;
 * hidden channels zero: a caller that trains sets perturbed initial weights first, or
 * the zero channels stay zero). The context owns it: dirac_destroy destroys networks
 * still alive. Returns DIRAC_ERR_ARG for bad channel lists,
 * DIRAC_ERR_UNSUPPORTED for an asqtad context or one without FP32. */
int dirac_ptc_create(dirac_ctx* ctx, const dirac_ptc_params* params, dirac_ptc** net);
/* Number of complex weights (sum over layers of 9 * 16 * c_out * c_in). */
long long dirac_ptc_num_weights(const dirac_ptc* net);
/* Copy n (= dirac_ptc_num_weights) complex weights from / to host memory, FP64 pairs. */
int dirac_ptc_set_weights(dirac_ptc* net, const double* w, long long n);
int dirac_ptc_get_weights(const dirac_ptc* net, double* w, long long n);
/* out = K in (FP32 full fields, distinct; asynchronous on stream; FP32 layers unless
 * tensor cores are switched on by dirac_ptc_set_tensor_cores). */
int dirac_ptc_apply(dirac_ptc* net, void* out, const void* in, void* stream);
/* Loss L = ||K r - v||^2 / ||v||^2 of one pair and its derivative with respect to the
 * conjugate weights, dL/dconj(W), into grad (host, FP64 pairs, num_weights entries);
 * loss and grad may be NULL. Synchronises stream. */
int dirac_ptc_gradient(dirac_ptc* net, const void* r, const void* v, double* loss, double* grad,
                       void* stream);
/* Train on pairs (r_i, v_i), i < npairs: Adam on the mean over a batch of
 * ||K r_i - v_i||^2 / ||v_i||^2. r may be NULL: then r_i = M v_i is computed (FP32)
 * by the library. r[i], v[i]: FP32 full fields owned by the caller, unchanged.
 * loss (host, may be NULL): params->steps entries, the batch loss before each step.
 * Synchronises stream. */
int dirac_ptc_train(dirac_ptc* net, const void* const* r, const void* const* v, int npairs,
                    const dirac_ptc_train_params* params, double* loss, void* stream);
/* on = 1: dirac_ptc_apply and the GCR_PTC solver run every layer on the tensor cores
 * (tcgen05, BF16 operands, FP32 accumulation: relative error ~1e-3, which the flexible
 * outer GCR absorbs); on = 0 (default): the FP32 CUDA-core layers used for training. A
 * tensor-core wait that gives up makes the next apply return DIRAC_ERR_TIMEOUT. */
int dirac_ptc_set_tensor_cores(dirac_ptc* net, int on);
/* Failure detection tests only (no counterpart in the paper). Every wait of the
 * tensor-core pipeline has a time budget, wait_seconds (default 2 s); with stall = 1 the
 * warp that issues the tensor-core instructions stops after loading the weights, as if
 * it had died, so the other warps' waits run out: the kernel records the error, frees its
 * tensor memory and returns, and the next dirac_ptc_apply returns DIRAC_ERR_TIMEOUT
 * (dirac_ptc_set_tensor_cores clears the error). stall = 0 restores normal operation. */
int dirac_ptc_test_stall(dirac_ptc* net, int stall, double wait_seconds);
/* Make net the preconditioner of DIRAC_SOLVER_GCR_PTC on ctx (NULL detaches). With
 * force = 0, every such solve starts with whichever of the network and the Schwarz
 * preconditioner gives the smaller ||r0 - M K r0||, runs the other one for one restart
 * cycle, and from then on each cycle uses the preconditioner with the higher measured
 * residual reduction per second of its last cycle (Schwarz is the fallback); force = 1
 * always uses the network. stats report the one-step reductions, the measured rates, the
 * switches and the preconditioner of the last cycle. */
int dirac_ptc_attach(dirac_ctx* ctx, dirac_ptc* net, int force);
/* Free the network (detaching it first). NULL is a no-op. */
int dirac_ptc_destroy(dirac_ptc* net);

/* ------------------------------------------------------------------ domain decomposition
 * The paper's multi-GPU scheme (Sec. 6: partitioning in up to four dimensions, spin-
 * projected face exchange, interior computation overlapping the communication) for the
 * Wilson-clover operator, emulated on one GPU: the lattice is cut by a grid of
 * grid[0] x grid[1] x grid[2] x grid[3] virtual ranks (every L_mu / grid_mu an even
 * integer >= 2; at most 256 ranks), each with its own local links, clover and spinors, a
 * stream, send buffers and, for every cut dimension, two ghost zones of one slice.
 * dirac_dd_apply packs each rank's boundary slices spin-projected (12 reals per face site:
 * FP64 in FP64, else FP32), copies them into the neighbours' ghost zones (device-to-device
 * copies ordered by events), and runs the interior (overlapping the exchange) and the
 * boundary sites as separate kernels. Backward-hop links of the faces are exchanged once,
 * by the create call. The result equals dirac_apply(FULL) of the whole lattice bit for bit
 * in FP64 and FP32 (FP16: to one binary16 unit per site after re-encoding). Fields: `in` /
 * `out` of scatter / gather are full fields of ctx in precision `prec`. All calls are
 * asynchronous on stream except create / destroy (which synchronise the device).
 * Errors: DIRAC_ERR_ARG for a grid that does not divide the lattice as required,
 * DIRAC_ERR_OOM when rank storage cannot be allocated. */
typedef struct dirac_dd dirac_dd;
/* grid: ranks per dimension (x, y, z, t); 1 leaves a dimension whole */
int dirac_dd_create_grid(dirac_ctx* ctx, const int* grid, dirac_prec prec, dirac_dd** dd);
/* nranks ranks along t: the grid (1, 1, 1, nranks) */
int dirac_dd_create(dirac_ctx* ctx, int nranks, dirac_prec prec, dirac_dd** dd);
/* global field -> every rank's local input */
int dirac_dd_scatter(dirac_dd* dd, const void* in, void* stream);
/* out_r = M in_r (dagger = 1: M^dagger) on every rank */
int dirac_dd_apply(dirac_dd* dd, int dagger, void* stream);
/* every rank's local output -> global field */
int dirac_dd_gather(dirac_dd* dd, void* out, void* stream);
/* local dims of a rank; bytes of the spinor faces one rank receives per application */
int dirac_dd_info(const dirac_dd* dd, int* local_dims, long long* face_bytes);
int dirac_dd_destroy(dirac_dd* dd);

#ifdef __cplusplus
}
#endif
#endif /* DIRAC_H */
