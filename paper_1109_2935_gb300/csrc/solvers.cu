// Krylov solvers behind solve(): CG on the normal equations, BiCGstab (Sec. 3.1) and
// the mixed-precision flexible GCR of Algorithm 1 with the Schwarz preconditioner
// (Sec. 8.1). The outer iterate x, the source b and the restart / reliable-update
// residual live in FP64; the Krylov vectors and the inner operator use the sloppy
// precision; the preconditioner runs in its own precision.
//
// Scalars stay on the GPU: reductions write device slots, one-thread kernels do the
// scalar algebra (and guard every division), BLAS kernels read their coefficients
// from the slots. The host reads each iteration's residual norm from mapped memory
// one iteration behind (the next iteration is already queued), so the GPU never
// waits for the host inside an iteration. Decisions taken one iteration late (a
// reliable update, a GCR restart, stopping) are harmless: one more Krylov step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace dirac {

using cplx = std::complex<double>;

// NVTX range for a solver phase (host timeline of profilers; no cost without one)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

namespace {

constexpr int KMAX = 20;
// device scalar slots (doubles); every slot is 4 wide
enum : int {
  S_RHO = 0, S_RHOOLD = 4, S_ALPHA = 8, S_OMEGA = 12, S_SIGMA = 16, S_TS = 20, S_RN = 24,
  S_BETA = 28, S_NBW = 32, S_NALPHA = 36, S_NOMEGA = 40, S_PAP = 44, S_RR = 48, S_ONE = 52,
  S_FLAG = 56, S_TMP = 60, S_ZZ = 64, S_INVG = 68, S_B0 = 72, S_RH = 76,
  S_GB = 128,                       // beta_{i,k}: slot (i * KMAX + k), value at +1, +2
  S_GG = S_GB + 4 * KMAX * KMAX,    // gamma_k
  S_GA = S_GG + 4 * KMAX,           // alpha_k (re, im)
  S_GC = S_GA + 4 * KMAX,           // chi_k (re, im)
  KSH = 16,                         // multi-shift: at most 16 shifts
  S_MSC = S_GC + 4 * KMAX,          // per shift: a_j, zeta_{k+1,j}, b_j, active_j
  S_MSZ = S_MSC + 4 * KSH,          // zeta_{k,j}
  S_MSZP = S_MSZ + KSH,             // zeta_{k-1,j}
  S_MSCV = S_MSZP + KSH,            // converged_j
  S_MSSH = S_MSCV + KSH,            // sigma_j
  S_MSAB = S_MSSH + KSH,            // a_{k-1}, b_{k-1} of the base system
  S_END = S_MSAB + 4
};
enum : int { FLAG_OK = 0, FLAG_BREAKDOWN = 1, FLAG_NONFINITE = 2 };

__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }
__device__ __forceinline__ void flag(double* S, int f) { if (S[S_FLAG] == FLAG_OK) S[S_FLAG] = f; }
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& qr, double& qi) {
  double d = br * br + bi * bi;
  qr = (ar * br + ai * bi) / d;
  qi = (ai * br - ar * bi) / d;
}

// --------------------------------------------------------------- scalar kernels
__global__ void k_init(double* S) {
  for (int i = 0; i < S_END; ++i) S[i] = 0;
  S[S_ONE] = 1;
  S[S_RHOOLD] = 1; S[S_ALPHA] = 1; S[S_OMEGA] = 1;
}
__global__ void k_set(double* S, int slot, double v0, double v1) { S[slot] = v0; S[slot + 1] = v1; }
__global__ void k_mirror(const double* S, int slot, double* mirror, int which, int it) {
  mirror[4 * which + 0] = S[slot];
  mirror[4 * which + 1] = S[S_FLAG];
  mirror[4 * which + 2] = it;
}

// BiCGstab: beta = (rho/rho_old)(alpha/omega); coefficient -beta*omega
__global__ void k_bicg1(double* S) {
  double q1r, q1i, q2r, q2i;
  if (S[S_RHOOLD] == 0 && S[S_RHOOLD + 1] == 0) { flag(S, FLAG_BREAKDOWN); }
  if (S[S_OMEGA] == 0 && S[S_OMEGA + 1] == 0) { flag(S, FLAG_BREAKDOWN); }
  if (S[S_FLAG] != FLAG_OK) {
    S[S_BETA] = S[S_BETA + 1] = S[S_NBW] = S[S_NBW + 1] = 0;
    return;
  }
  cdiv(S[S_RHO], S[S_RHO + 1], S[S_RHOOLD], S[S_RHOOLD + 1], q1r, q1i);
  cdiv(S[S_ALPHA], S[S_ALPHA + 1], S[S_OMEGA], S[S_OMEGA + 1], q2r, q2i);
  double br = q1r * q2r - q1i * q2i, bi = q1r * q2i + q1i * q2r;
  S[S_BETA] = br; S[S_BETA + 1] = bi;
  double wr = S[S_OMEGA], wi = S[S_OMEGA + 1];
  S[S_NBW] = -(br * wr - bi * wi); S[S_NBW + 1] = -(br * wi + bi * wr);
}
// alpha = rho / (r0, v)
__global__ void k_bicg2(double* S) {
  double sr = S[S_SIGMA], si = S[S_SIGMA + 1];
  if (bad(sr) || bad(si)) flag(S, FLAG_NONFINITE);
  else if (sr == 0 && si == 0) flag(S, FLAG_BREAKDOWN);
  double ar = 0, ai = 0;
  if (S[S_FLAG] == FLAG_OK) cdiv(S[S_RHO], S[S_RHO + 1], sr, si, ar, ai);
  S[S_ALPHA] = ar; S[S_ALPHA + 1] = ai;
  S[S_NALPHA] = -ar; S[S_NALPHA + 1] = -ai;
}
// omega = (t, s) / (t, t)
__global__ void k_bicg3(double* S) {
  double tt = S[S_TS + 2];
  if (bad(tt) || bad(S[S_TS]) || bad(S[S_TS + 1])) flag(S, FLAG_NONFINITE);
  else if (tt == 0) flag(S, FLAG_BREAKDOWN);
  double wr = 0, wi = 0;
  if (S[S_FLAG] == FLAG_OK) { wr = S[S_TS] / tt; wi = S[S_TS + 1] / tt; }
  S[S_OMEGA] = S[S_FLAG] == FLAG_OK ? wr : 1; S[S_OMEGA + 1] = S[S_FLAG] == FLAG_OK ? wi : 0;
  S[S_NOMEGA] = -wr; S[S_NOMEGA + 1] = -wi;
}
// rho_old = rho; rho = (r0, r)
__global__ void k_bicg4(double* S, double* mirror, int which, int it) {
  S[S_RHOOLD] = S[S_RHO]; S[S_RHOOLD + 1] = S[S_RHO + 1];
  S[S_RHO] = S[S_RN + 1]; S[S_RHO + 1] = S[S_RN + 2];
  if (bad(S[S_RN])) flag(S, FLAG_NONFINITE);
  mirror[4 * which + 0] = S[S_RN];
  mirror[4 * which + 1] = S[S_FLAG];
  mirror[4 * which + 2] = it;
}
// after a reliable update: rho = (r0, r) from a cdot into S_TMP
__global__ void k_bicg_rho(double* S) { S[S_RHO] = S[S_TMP]; S[S_RHO + 1] = S[S_TMP + 1]; }

// CG: alpha = rr / (p, Ap)
__global__ void k_cg1(double* S) {
  double pap = S[S_PAP];
  if (bad(pap)) flag(S, FLAG_NONFINITE);
  else if (pap <= 0) flag(S, FLAG_BREAKDOWN);
  double a = S[S_FLAG] == FLAG_OK ? S[S_RR] / pap : 0;
  S[S_ALPHA] = a; S[S_ALPHA + 1] = 0;
  S[S_NALPHA] = -a; S[S_NALPHA + 1] = 0;
}
// beta = rr_new / rr
__global__ void k_cg2(double* S, double* mirror, int which, int it) {
  double rn = S[S_RN];
  if (bad(rn)) flag(S, FLAG_NONFINITE);
  double b = (S[S_FLAG] == FLAG_OK && S[S_RR] > 0) ? rn / S[S_RR] : 0;
  S[S_BETA] = b; S[S_BETA + 1] = 0;
  if (S[S_FLAG] == FLAG_OK) S[S_RR] = rn;
  mirror[4 * which + 0] = rn;
  mirror[4 * which + 1] = S[S_FLAG];
  mirror[4 * which + 2] = it;
}

// GCR: gamma_k = ||z_k||, 1/gamma_k; move beta_{0,k} (a cdot result) into its slot
__global__ void k_gcr_gamma(double* S, int k) {
  double zz = S[S_ZZ];
  if (bad(zz)) flag(S, FLAG_NONFINITE);
  else if (zz <= 0) flag(S, FLAG_BREAKDOWN);
  double g = S[S_FLAG] == FLAG_OK ? sqrt(zz) : 1;
  S[S_GG + 4 * k] = g;
  S[S_INVG] = S[S_FLAG] == FLAG_OK ? 1.0 / g : 0;
  S[S_INVG + 1] = 0;
  if (k > 0) {
    S[S_GB + 4 * (0 * KMAX + k) + 1] = S[S_B0];
    S[S_GB + 4 * (0 * KMAX + k) + 2] = S[S_B0 + 1];
  }
}
// back-substitution of Algorithm 1: gamma_l chi_l + sum_{i>l} beta_{l,i} chi_i = alpha_l
__global__ void k_gcr_backsub(double* S, int k) {
  for (int l = k - 1; l >= 0; --l) {
    double sr = S[S_GA + 4 * l], si = S[S_GA + 4 * l + 1];
    for (int i = l + 1; i < k; ++i) {
      double br = S[S_GB + 4 * (l * KMAX + i) + 1], bi = S[S_GB + 4 * (l * KMAX + i) + 2];
      double cr = S[S_GC + 4 * i], ci = S[S_GC + 4 * i + 1];
      sr -= br * cr - bi * ci;
      si -= br * ci + bi * cr;
    }
    double g = S[S_GG + 4 * l];
    S[S_GC + 4 * l] = sr / g;
    S[S_GC + 4 * l + 1] = si / g;
  }
}

// Multi-shift CG (Eq. 4). The base system is the smallest shift j0, solved by CG on
// A' = A + sigma_j0. The residuals of a shifted system A' + s (s = sigma_j - sigma_j0)
// are zeta_j times the base residuals (same Krylov space, both orthogonal to it);
// equating the CG three-term recurrences of the two systems gives
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} / (a_{k-1} zeta_{k-1} (1 + s a_k)
//                                            + a_k b_{k-1} (zeta_{k-1} - zeta_k)),
//   a_j = a_k zeta_{k+1} / zeta_k,   b_j = b_k (zeta_{k+1} / zeta_k)^2,
// with zeta_{-1} = zeta_0 = 1, a_{-1} = 1, b_{-1} = 0.
struct ShiftTable { double v[KSH]; };
__global__ void k_ms_init(double* S, int n, ShiftTable sh) {
  for (int j = 0; j < KSH; ++j) {
    S[S_MSSH + j] = j < n ? sh.v[j] : 0;
    S[S_MSZ + j] = 1;
    S[S_MSZP + j] = 1;
    S[S_MSCV + j] = 0;
    S[S_MSC + 4 * j + 0] = 0;
    S[S_MSC + 4 * j + 1] = 1;
    S[S_MSC + 4 * j + 2] = 0;
    S[S_MSC + 4 * j + 3] = j < n ? 1 : 0;
  }
  S[S_MSAB] = 1;      // a_{-1}
  S[S_MSAB + 1] = 0;  // b_{-1}
}
// base system: alpha = rr / (p, (A + sigma_0) p)
__global__ void k_ms1(double* S) {
  double pap = S[S_PAP];
  if (bad(pap)) flag(S, FLAG_NONFINITE);
  else if (pap <= 0) flag(S, FLAG_BREAKDOWN);
  double a = S[S_FLAG] == FLAG_OK ? S[S_RR] / pap : 0;
  S[S_ALPHA] = a;
  S[S_NALPHA] = -a; S[S_NALPHA + 1] = 0;
}
// every shift: zeta_{k+1}, a_j, b_j; retire systems that converged last time
__global__ void k_ms2(double* S, int n, int j0, double tol2bb, double* mirror, int which, int it) {
  const double a = S[S_ALPHA], rr = S[S_RR], rn = S[S_RN];
  if (bad(rn)) flag(S, FLAG_NONFINITE);
  const double bk = (S[S_FLAG] == FLAG_OK && rr > 0) ? rn / rr : 0;
  const double ap = S[S_MSAB], bp = S[S_MSAB + 1], s0 = S[S_MSSH + j0];
  double worst = 0;
  int nact = 0;
  for (int j = 0; j < n; ++j) {
    if (S[S_MSCV + j] != 0) S[S_MSC + 4 * j + 3] = 0;
    if (S[S_MSC + 4 * j + 3] == 0) continue;
    const double z = S[S_MSZ + j], zp = S[S_MSZP + j];
    double zn = 1;
    if (j != j0) {
      const double sh = S[S_MSSH + j] - s0;
      const double den = ap * zp * (1 + sh * a) + a * bp * (zp - z);
      zn = den != 0 ? z * zp * ap / den : 0;
    }
    if (bad(zn) || z == 0) {
      flag(S, FLAG_NONFINITE);
      S[S_MSC + 4 * j + 3] = 0;
      continue;
    }
    S[S_MSC + 4 * j + 0] = a * zn / z;
    S[S_MSC + 4 * j + 1] = zn;
    S[S_MSC + 4 * j + 2] = bk * (zn / z) * (zn / z);
    S[S_MSZP + j] = z;
    S[S_MSZ + j] = zn;
    const double res = zn * zn * rn;
    if (res <= tol2bb) S[S_MSCV + j] = 1;  // this update is its last
    else {
      ++nact;
      worst = res > worst ? res : worst;
    }
  }
  S[S_MSAB] = a;
  S[S_MSAB + 1] = bk;
  if (S[S_FLAG] == FLAG_OK) S[S_RR] = rn;
  mirror[4 * which + 0] = worst;
  mirror[4 * which + 1] = S[S_FLAG];
  mirror[4 * which + 2] = it;
  mirror[4 * which + 3] = nact;
}

// --------------------------------------------------------------- host side
struct Ctx {
  dirac_ctx* c;
  cudaStream_t st;
  int parity;   // -1 full, 0 even (CG_EVEN_NORMAL)
  int which;    // operator: 0 = M, 2 = normal
  int next = 0;
  dirac_solver_stats* stats;
  double flops_per_apply = 0;
  double shift = 0;           // A = M^dagger M + shift for the normal-operator solvers
  double* S = nullptr;        // device scalar slots
  double* mirror = nullptr;   // device alias of the mapped host mirror
  volatile double* hmirror = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool graphs = false;        // GCR: replay captured steps (needs a capturable stream)

  char* get(int prec) {
    size_t bytes = (parity < 0 ? 2 : 1) * spinor_half_bytes(prec, c->nr, c->Vh);
    int i = next++;
    if (i >= 48) return nullptr;
    if (c->work_bytes[i] < bytes) {
      if (c->work[i]) cudaFree(c->work[i]);
      c->work[i] = nullptr;
      c->work_bytes[i] = 0;
      if (cudaMalloc(&c->work[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        c->work[i] = nullptr;
        return nullptr;
      }
      c->work_bytes[i] = bytes;
    }
    return c->work[i];
  }
  FieldRef f(const void* p, int prec) const { return field_ref(c, p, prec, parity); }
  int A(char* out, const char* in, int prec) {
    stats->dslash_calls += 1;
    stats->flops += flops_per_apply;
    return apply_op(c, out, in, parity, prec, which, st, which == 2 ? shift : 0.0);
  }
  double* slot(int s) const { return S + s; }
  // record the end of iteration `it`; its mirror entry is it % 2
  int mark(int it) { return cudaEventRecord(ev[it & 1], st) == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA; }
  // wait for iteration `it` and return its mirrored {value, flag}
  int read(int it, double* v, int* fl) {
    if (cudaEventSynchronize(ev[it & 1]) != cudaSuccess) return DIRAC_ERR_CUDA;
    *v = hmirror[4 * (it & 1) + 0];
    *fl = (int)hmirror[4 * (it & 1) + 1];
    return DIRAC_OK;
  }
};

#define TRY(expr)                   \
  do {                              \
    int _rc = (expr);               \
    if (_rc) return _rc;            \
  } while (0)

int blas_fail(Ctx& S, int rc) {
  if (rc) S.c->err = blas_error(S.c->blas);
  return rc;
}
#define BT(expr) TRY(blas_fail(S, (expr)))
#define KC(launch)                                                          \
  do {                                                                      \
    launch;                                                                 \
    if (cudaGetLastError() != cudaSuccess)                                  \
      return set_err(S.c, DIRAC_ERR_CUDA, "solver scalar kernel launch");   \
  } while (0)

bool finite(double v) { return std::isfinite(v); }

int flag_error(Ctx& S, int fl, const char* who) {
  if (fl == FLAG_BREAKDOWN) return set_err(S.c, DIRAC_ERR_BREAKDOWN, std::string(who) + ": a Krylov denominator vanished");
  return set_err(S.c, DIRAC_ERR_NONFINITE, std::string(who) + ": non-finite scalar");
}

// The sloppy solution correction between reliable updates is accumulated in at least
// FP32: with 16-bit storage the late, small updates of a cycle would fall below the
// 11-bit resolution of the accumulated correction and be lost.
int accum_prec(int sp) { return sp == P16 ? P32 : sp; }

// A x for the true residual: FP64 fields; for the Wilson-clover M (or M^dagger M) on the
// whole lattice the operator runs in double-single arithmetic unless switched off
// (dirac_set_ds_residual), otherwise in FP64
int residual_operator(Ctx& S, char* out, const char* x, bool* ds) {
  dirac_ctx* c = S.c;
  *ds = c->ds_residual && S.parity < 0 && (S.which == 0 || S.which == 2) && ds_available(c);
  if (!*ds) return S.A(out, x, P64);
  S.stats->dslash_calls += 1;
  S.stats->flops += S.flops_per_apply;
  if (S.which == 0) return wilson_M_ds(c, out, x, false, S.st);
  TRY(ensure_tmp(c, P64));
  TRY(wilson_M_ds(c, c->tmp[P64], x, false, S.st));
  TRY(wilson_M_ds(c, out, c->tmp[P64], true, S.st));
  if (S.shift != 0.0) BT(blas_axpby(c->blas, cval(S.shift), S.f(x, P64), cval(1), S.f(out, P64), S.st));
  return DIRAC_OK;
}

// r = b - A x in FP64 storage, returns ||r||^2 (host, synchronising). A residual that the
// double-single operator puts below `target` (a convergence decision) is recomputed with
// the FP64 operator, which then decides.
int true_residual(Ctx& S, char* r, const char* x, const char* b, double* rr, double target = -1.0) {
  Range range("true residual (FP64)");
  bool ds = false;
  TRY(residual_operator(S, r, x, &ds));
  BT(blas_xmy_norm(S.c->blas, S.f(b, P64), S.f(r, P64), rr, S.st));
  if (ds && *rr < target) {
    TRY(S.A(r, x, P64));
    BT(blas_xmy_norm(S.c->blas, S.f(b, P64), S.f(r, P64), rr, S.st));
  }
  return DIRAC_OK;
}

int start_residual(Ctx& S, char* x, const char* b, char* r, const dirac_solver_params& P, double bb,
                   double* rr) {
  if (P.use_x0) return true_residual(S, r, x, b, rr, P.tol * P.tol * bb);
  BT(blas_zero(S.c->blas, S.f(x, P64), S.st));
  BT(blas_copy(S.c->blas, S.f(r, P64), S.f(b, P64), S.st));
  *rr = bb;
  return DIRAC_OK;
}

// ------------------------------------------------------------------ CG (Sec. 3.1)
int solve_cg(Ctx& S, char* x, const char* b, const dirac_solver_params& P) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy, ap = accum_prec(sp);
  char *r = S.get(P64), *rs = S.get(sp), *p = S.get(sp), *Ap = S.get(sp), *xs = S.get(ap);
  if (!r || !rs || !p || !Ap || !xs) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (!finite(bb)) return set_err(S.c, DIRAC_ERR_NONFINITE, "non-finite source");
  if (bb == 0.0) {
    BT(blas_zero(B, S.f(x, P64), S.st));
    return DIRAC_OK;
  }
  const double target = P.tol * P.tol * bb, d2 = P.delta * P.delta;
  double rr;
  TRY(start_residual(S, x, b, r, P, bb, &rr));
  if (rr < target) return DIRAC_OK;
  BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
  BT(blas_copy(B, S.f(p, sp), S.f(rs, sp), S.st));
  BT(blas_zero(B, S.f(xs, ap), S.st));
  KC((k_init<<<1, 1, 0, S.st>>>(S.S)));
  KC((k_set<<<1, 1, 0, S.st>>>(S.S, S_RR, rr, 0)));
  double rmax = rr;
  int it = 0;
  bool converged = false;
  while (S.stats->iters < P.max_iter) {
    TRY(S.A(Ap, p, sp));
    BT(blas_cdot_norm(B, S.f(p, sp), S.f(Ap, sp), nullptr, S.st, S.slot(S_PAP)));
    KC((k_cg1<<<1, 1, 0, S.st>>>(S.S)));
    BT(blas_cg_update(B, cptr(S.slot(S_ALPHA)), S.f(p, sp), cptr(S.slot(S_NALPHA)), S.f(Ap, sp),
                      S.f(xs, ap), S.f(rs, sp), nullptr, S.st, S.slot(S_RN)));
    KC((k_cg2<<<1, 1, 0, S.st>>>(S.S, S.mirror, it & 1, it)));
    BT(blas_axpby(B, cval(1), S.f(rs, sp), cptr(S.slot(S_BETA)), S.f(p, sp), S.st));
    TRY(S.mark(it));
    S.stats->iters++;
    if (it > 0) {  // decisions from the previous iteration
      double rp;
      int fl;
      TRY(S.read(it - 1, &rp, &fl));
      if (fl != FLAG_OK) return flag_error(S, fl, "CG");
      if ((d2 > 0 && rp < d2 * rmax) || rp < target) {
        // reliable update: fold the sloppy correction into x, recompute r in FP64
        BT(blas_axpby(B, cval(1), S.f(xs, ap), cval(1), S.f(x, P64), S.st));
        BT(blas_zero(B, S.f(xs, ap), S.st));
        TRY(true_residual(S, r, x, b, &rr, target));
        S.stats->reliable_updates++;
        if (rr < target) { converged = true; break; }
        BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
        KC((k_set<<<1, 1, 0, S.st>>>(S.S, S_RR, rr, 0)));
        rmax = rr;
        it = -1;  // the mirror of the iteration before the update is stale
      }
    }
    ++it;
  }
  if (!converged) BT(blas_axpby(B, cval(1), S.f(xs, ap), cval(1), S.f(x, P64), S.st));
  return DIRAC_OK;
}

// ------------------------------------------------------------------ BiCGstab (Sec. 3.1)
// Replay of solver steps as CUDA graphs. A step whose launches depend only on a small
// key (the Krylov index of GCR, the mirror slot of BiCGstab) runs directly the first time
// (allocations and one-time attributes happen then), is captured the second time and
// replayed afterwards; the statistics it adds on the host are recorded at capture and
// added on replay.
struct StepGraphs {
  struct G {
    cudaGraphExec_t exec = nullptr;
    int state = 0;  // 0: not run, 1: run once directly, 2: captured
    dirac_solver_stats delta{};
  };
  std::vector<G> g;
  bool on;
  StepGraphs(int n, bool enable) : g(n), on(enable) {}
  ~StepGraphs() {
    for (auto& x : g)
      if (x.exec) cudaGraphExecDestroy(x.exec);
  }
  template <class F>
  int run(Ctx& S, int key, F&& step) {
    G& e = g[key];
    if (!on || e.state == 0) {
      e.state = 1;
      return step();
    }
    if (e.state == 2) {
      if (cudaGraphLaunch(e.exec, S.st) != cudaSuccess) return set_err(S.c, DIRAC_ERR_CUDA, "graph launch");
      S.stats->dslash_calls += e.delta.dslash_calls;
      S.stats->precond_calls += e.delta.precond_calls;
      S.stats->flops += e.delta.flops;
      return DIRAC_OK;
    }
    const dirac_solver_stats before = *S.stats;
    if (cudaStreamBeginCapture(S.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return set_err(S.c, DIRAC_ERR_CUDA, "graph capture");
    const int rc = step();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(S.st, &graph);
    if (rc || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : set_err(S.c, DIRAC_ERR_CUDA, "graph capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return set_err(S.c, DIRAC_ERR_CUDA, "graph instantiate");
    e.delta.dslash_calls = S.stats->dslash_calls - before.dslash_calls;
    e.delta.precond_calls = S.stats->precond_calls - before.precond_calls;
    e.delta.flops = S.stats->flops - before.flops;
    e.state = 2;
    if (cudaGraphLaunch(e.exec, S.st) != cudaSuccess) return set_err(S.c, DIRAC_ERR_CUDA, "graph launch");
    return DIRAC_OK;
  }
};

int solve_bicgstab(Ctx& S, char* x, const char* b, const dirac_solver_params& P) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy, ap = accum_prec(sp);
  char *r = S.get(P64), *rs = S.get(sp), *r0 = S.get(sp), *p = S.get(sp), *v = S.get(sp),
       *t = S.get(sp), *xs = S.get(ap);
  if (!r || !rs || !r0 || !p || !v || !t || !xs) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (!finite(bb)) return set_err(S.c, DIRAC_ERR_NONFINITE, "non-finite source");
  if (bb == 0.0) {
    BT(blas_zero(B, S.f(x, P64), S.st));
    return DIRAC_OK;
  }
  const double target = P.tol * P.tol * bb, d2 = P.delta * P.delta;
  double rr;
  TRY(start_residual(S, x, b, r, P, bb, &rr));
  if (rr < target) return DIRAC_OK;
  BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
  BT(blas_copy(B, S.f(r0, sp), S.f(rs, sp), S.st));
  BT(blas_zero(B, S.f(p, sp), S.st));
  BT(blas_zero(B, S.f(v, sp), S.st));
  BT(blas_zero(B, S.f(xs, ap), S.st));
  KC((k_init<<<1, 1, 0, S.st>>>(S.S)));
  BT(blas_cdot(B, S.f(r0, sp), S.f(rs, sp), nullptr, S.st, S.slot(S_RHO)));
  double rmax = rr;
  int it = 0;
  bool converged = false;
  // one iteration; its launches depend only on the mirror slot it & 1
  auto step = [&](int slot) -> int {
    Range range("BiCGstab iteration");
    KC((k_bicg1<<<1, 1, 0, S.st>>>(S.S)));
    // p = r + beta (p - omega v)
    BT(blas_pupdate(B, S.f(rs, sp), cptr(S.slot(S_BETA)), cptr(S.slot(S_NBW)), S.f(v, sp), S.f(p, sp), S.st));
    TRY(S.A(v, p, sp));
    BT(blas_cdot(B, S.f(r0, sp), S.f(v, sp), nullptr, S.st, S.slot(S_SIGMA)));
    KC((k_bicg2<<<1, 1, 0, S.st>>>(S.S)));
    // s = r - alpha v (in rs)
    BT(blas_caxpy_norm(B, cptr(S.slot(S_NALPHA)), S.f(v, sp), S.f(rs, sp), nullptr, S.st, S.slot(S_TMP)));
    TRY(S.A(t, rs, sp));
    BT(blas_cdot_norm(B, S.f(t, sp), S.f(rs, sp), nullptr, S.st, S.slot(S_TS)));
    KC((k_bicg3<<<1, 1, 0, S.st>>>(S.S)));
    // xs += alpha p + omega s; r = s - omega t; ||r||^2, (r0, r)
    BT(blas_bicg_xr(B, cptr(S.slot(S_ALPHA)), S.f(p, sp), cptr(S.slot(S_OMEGA)), S.f(rs, sp),
                    cptr(S.slot(S_NOMEGA)), S.f(t, sp), S.f(xs, ap), S.f(r0, sp), nullptr, S.st,
                    S.slot(S_RN)));
    KC((k_bicg4<<<1, 1, 0, S.st>>>(S.S, S.mirror, slot, slot)));
    return DIRAC_OK;
  };
  StepGraphs graphs(2, S.graphs);
  while (S.stats->iters < P.max_iter) {
    TRY(graphs.run(S, it & 1, [&] { return step(it & 1); }));
    TRY(S.mark(it));
    S.stats->iters++;
    if (it > 0) {
      double rp;
      int fl;
      TRY(S.read(it - 1, &rp, &fl));
      if (fl != FLAG_OK) return flag_error(S, fl, "BiCGstab");
      if ((d2 > 0 && rp < d2 * rmax) || rp < target) {
        BT(blas_axpby(B, cval(1), S.f(xs, ap), cval(1), S.f(x, P64), S.st));
        BT(blas_zero(B, S.f(xs, ap), S.st));
        TRY(true_residual(S, r, x, b, &rr, target));
        S.stats->reliable_updates++;
        if (rr < target) { converged = true; break; }
        BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
        BT(blas_cdot(B, S.f(r0, sp), S.f(rs, sp), nullptr, S.st, S.slot(S_TMP)));
        KC((k_bicg_rho<<<1, 1, 0, S.st>>>(S.S)));
        rmax = rr;
        it = -1;
      }
    }
    ++it;
  }
  if (!converged) BT(blas_axpby(B, cval(1), S.f(xs, ap), cval(1), S.f(x, P64), S.st));
  return DIRAC_OK;
}

// ------------------------------------------------------------------ GCR (Algorithm 1)
// Preconditioner K of the flexible GCR: none, the Schwarz preconditioner (runs in
// prec_precond) or the attached PTC network (runs in FP32). A preconditioner whose
// precision differs from the sloppy one gets its input and output converted.
enum : int { K_NONE = 0, K_SCHWARZ = 1, K_PTC = 2, K_SELECT = 3 };

struct Precond {
  char* in[3] = {};
  char* out[3] = {};
  double flops[3] = {};
};

int precond_apply(Ctx& S, Precond& K, int kind, char* out, const char* in, int sp, int pp) {
  Range range(kind == K_PTC ? "preconditioner (PTC)" : "preconditioner (Schwarz)");
  Blas* B = S.c->blas;
  const int kp = kind == K_PTC ? P32 : pp;
  S.stats->precond_calls++;
  S.stats->flops += K.flops[kind];
  auto run = [&](char* o, const char* i) -> int {
    return kind == K_PTC ? ptc_apply_internal(S.c->ptc_attached, o, i, S.st) : schwarz_apply(S.c, o, i, kp, S.st);
  };
  if (kp == sp) return run(out, in);
  BT(blas_copy(B, S.f(K.in[kp], kp), S.f(in, sp), S.st));
  TRY(run(K.out[kp], K.in[kp]));
  BT(blas_copy(B, S.f(out, sp), S.f(K.out[kp], kp), S.st));
  return DIRAC_OK;
}

int solve_gcr(Ctx& S, char* x, const char* b, const dirac_solver_params& P, int precond) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy, pp = P.prec_precond;
  const int kmax = P.k_max;
  if (kmax < 1 || kmax > KMAX) return set_err(S.c, DIRAC_ERR_ARG, "k_max must be in [1, 20]");
  if (precond == K_SELECT && !S.c->ptc_attached)
    return set_err(S.c, DIRAC_ERR_STATE, "GCR_PTC: no PTC network attached");
  char* r = S.get(P64);
  char* rh = S.get(sp);
  std::vector<char*> pv(kmax), zv(kmax);
  for (int i = 0; i < kmax; ++i) {
    pv[i] = S.get(sp);
    zv[i] = S.get(sp);
  }
  Precond K;
  K.flops[K_SCHWARZ] = (double)S.c->V * S.c->p.mr_steps * (1872.0 + 192.0);
  if (precond == K_SELECT) K.flops[K_PTC] = ptc_flops_per_apply(S.c->ptc_attached);
  for (int kind : {K_SCHWARZ, K_PTC}) {
    if (precond == K_NONE || (precond != K_SELECT && precond != kind)) continue;
    const int kp = kind == K_PTC ? P32 : pp;
    if (kp == sp || K.in[kp]) continue;
    K.in[kp] = S.get(kp);
    K.out[kp] = S.get(kp);
    if (!K.in[kp] || !K.out[kp]) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  }
  if (!r || !rh) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  for (int i = 0; i < kmax; ++i)
    if (!pv[i] || !zv[i]) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");

  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (!finite(bb)) return set_err(S.c, DIRAC_ERR_NONFINITE, "non-finite source");
  if (bb == 0.0) {
    BT(blas_zero(B, S.f(x, P64), S.st));
    return DIRAC_OK;
  }
  const double target = P.tol * P.tol * bb, d2 = P.delta * P.delta;
  double r0n2;
  TRY(start_residual(S, x, b, r, P, bb, &r0n2));
  BT(blas_copy(B, S.f(rh, sp), S.f(r, P64), S.st));
  int kind = precond;
  if (precond == K_SELECT && S.c->ptc_force) {
    kind = K_PTC;
  } else if (precond == K_SELECT) {
    // keep the preconditioner with the smaller ||r0 - M K r0|| on this source
    for (int k2 : {K_SCHWARZ, K_PTC}) {
      double e2;
      TRY(precond_apply(S, K, k2, pv[0], rh, sp, pp));
      TRY(S.A(zv[0], pv[0], sp));
      BT(blas_xmy_norm(B, S.f(rh, sp), S.f(zv[0], sp), &e2, S.st));
      S.stats->precond_reduction[k2 - 1] = r0n2 > 0 ? std::sqrt(e2 / r0n2) : 0.0;
    }
    const double* red = S.stats->precond_reduction;
    kind = finite(red[1]) && red[1] < red[0] ? K_PTC : K_SCHWARZ;
  }
  S.stats->precond_kind = kind;
  KC((k_init<<<1, 1, 0, S.st>>>(S.S)));
  auto gb = [&](int i, int k) { return S.slot(S_GB + 4 * (i * KMAX + k) + 1); };
  // One GCR step at Krylov index k: p_k = K r_k, z_k = M p_k, orthogonalisation, the
  // residual update. Its launches depend only on k, so from the second restart cycle on
  // each step replays a CUDA graph captured the cycle before.
  auto step = [&](int k) -> int {
    Range range("GCR step");
    // p_k = K r_k
    if (kind != K_NONE) {
      TRY(precond_apply(S, K, kind, pv[k], rh, sp, pp));
    } else {
      BT(blas_copy(B, S.f(pv[k], sp), S.f(rh, sp), S.st));
    }
    // z_k = M p_k
    TRY(S.A(zv[k], pv[k], sp));
    // modified Gram-Schmidt: beta_ik = (z_i, z_k); z_k -= beta_ik z_i. Each pass
    // subtracts the previous projection and forms the next inner product.
    if (k == 0) {
      BT(blas_norm2(B, S.f(zv[0], sp), nullptr, S.st, S.slot(S_ZZ)));
    } else {
      BT(blas_cdot(B, S.f(zv[0], sp), S.f(zv[k], sp), nullptr, S.st, S.slot(S_B0)));
      for (int i = 1; i < k; ++i) {
        const double* bprev = i == 1 ? S.slot(S_B0) : gb(i - 1, k);
        BT(blas_caxpy_norm_dot(B, cptr(bprev, -1), S.f(zv[i - 1], sp), S.f(zv[k], sp), S.f(zv[i], sp),
                               nullptr, S.st, gb(i, k) - 1));
      }
      const double* blast = k == 1 ? S.slot(S_B0) : gb(k - 1, k);
      BT(blas_caxpy_norm(B, cptr(blast, -1), S.f(zv[k - 1], sp), S.f(zv[k], sp), nullptr, S.st, S.slot(S_ZZ)));
    }
    KC((k_gcr_gamma<<<1, 1, 0, S.st>>>(S.S, k)));
    // z_k /= gamma_k ; alpha_k = (z_k, r_k) ; r_{k+1} = r_k - alpha_k z_k
    BT(blas_scale_cdot(B, cptr(S.slot(S_INVG)), S.f(zv[k], sp), S.f(rh, sp), nullptr, S.st, S.slot(S_GA + 4 * k)));
    BT(blas_caxpy_norm(B, cptr(S.slot(S_GA + 4 * k), -1), S.f(zv[k], sp), S.f(rh, sp), nullptr, S.st,
                       S.slot(S_RH)));
    KC((k_mirror<<<1, 1, 0, S.st>>>(S.S, S_RH, S.mirror, k & 1, k)));
    return DIRAC_OK;
  };
  // Each preconditioner has its own captured steps. With K_SELECT (not forced) the choice
  // is revisited at every restart: the residual reduction per second of the cycle just
  // finished (natural log of ||r|| per second of wall time) is kept per preconditioner;
  // the other one is tried once (if its one-step test reduced the residual at all), and
  // afterwards whichever has the higher last measured rate runs the next cycle (flexible
  // GCR admits a change of K at a restart).
  StepGraphs cap_n(kmax, S.graphs), cap_s(kmax, S.graphs), cap_p(kmax, S.graphs);
  StepGraphs* caps[3] = {&cap_n, &cap_s, &cap_p};
  const bool adaptive = precond == K_SELECT && !S.c->ptc_force;
  double rate[3] = {-1.0, -1.0, -1.0};
  auto cycle_t0 = std::chrono::steady_clock::now();
  double cycle_r0 = r0n2;
  int k = 0;
  while (r0n2 > target && S.stats->iters < P.max_iter) {
    TRY(caps[kind]->run(S, k, [&] { return step(k); }));
    TRY(S.mark(k));
    ++k;
    S.stats->iters++;
    bool restart = k == kmax || S.stats->iters >= P.max_iter;
    if (!restart && k >= 2) {  // the previous step's residual, one iteration behind
      double rp;
      int fl;
      TRY(S.read(k - 2, &rp, &fl));
      if (fl != FLAG_OK) return flag_error(S, fl, "GCR");
      restart = (d2 > 0 && rp < d2 * r0n2) || rp < target;
    }
    if (restart) {
      double rp;
      int fl;
      TRY(S.read(k - 1, &rp, &fl));
      if (fl != FLAG_OK) return flag_error(S, fl, "GCR");
      KC((k_gcr_backsub<<<1, 1, 0, S.st>>>(S.S, k)));
      std::vector<Cf> cf(k);
      std::vector<FieldRef> xs(k);
      for (int i = 0; i < k; ++i) {
        cf[i] = cptr(S.slot(S_GC + 4 * i));
        xs[i] = S.f(pv[i], sp);
      }
      BT(blas_multi_caxpy(B, k, cf.data(), xs.data(), S.f(x, P64), S.st));
      TRY(true_residual(S, r, x, b, &r0n2, target));
      if (!finite(r0n2)) return set_err(S.c, DIRAC_ERR_NONFINITE, "GCR: non-finite true residual");
      BT(blas_copy(B, S.f(rh, sp), S.f(r, P64), S.st));
      S.stats->restarts++;
      k = 0;
      if (adaptive) {
        const auto now = std::chrono::steady_clock::now();
        const double secs = std::chrono::duration<double>(now - cycle_t0).count();
        if (secs > 0 && r0n2 > 0 && cycle_r0 > 0) rate[kind] = 0.5 * std::log(cycle_r0 / r0n2) / secs;
        const int other = kind == K_SCHWARZ ? K_PTC : K_SCHWARZ;
        // a preconditioner whose one-step test reduced nothing (||r0 - M K r0|| >= ||r0||,
        // e.g. an untrained network with K = 0) is never tried: its GCR step would break down
        const double red_other = S.stats->precond_reduction[other - 1];
        const bool usable = finite(red_other) && red_other < 1.0;
        if (usable && (rate[other] < 0 || rate[other] > rate[kind])) {
          kind = other;
          S.stats->precond_switches++;
        }
        S.stats->precond_rate[0] = rate[K_SCHWARZ];
        S.stats->precond_rate[1] = rate[K_PTC];
        cycle_t0 = now;
        cycle_r0 = r0n2;
      }
    }
  }
  S.stats->precond_kind = kind;
  return DIRAC_OK;
}

// ------------------------------------------------------------------ multi-shift CG
// Sec. 8.2: multi-shift CG in the sloppy precision for every shift at once, then
// mixed-precision CG refinement of each x_j on its own system (warm start).
int solve_ms_stage(Ctx& S, char* const* xout, const char* b, const double* shifts, int n,
                   const dirac_solver_params& P, double ms_tol) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy, ap = accum_prec(sp);
  int j0 = 0;
  for (int j = 1; j < n; ++j)
    if (shifts[j] < shifts[j0]) j0 = j;
  char *rs = S.get(sp), *Ap = S.get(sp);
  std::vector<FieldRef> xs(n), ps(n);
  for (int j = 0; j < n; ++j) {
    char* xp = S.get(ap);
    char* pp = S.get(sp);
    if (!xp || !pp) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
    xs[j] = S.f(xp, ap);
    ps[j] = S.f(pp, sp);
  }
  if (!rs || !Ap) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (!finite(bb)) return set_err(S.c, DIRAC_ERR_NONFINITE, "non-finite source");
  if (bb == 0.0) {
    for (int j = 0; j < n; ++j) BT(blas_zero(B, S.f(xout[j], P64), S.st));
    return DIRAC_OK;
  }
  BT(blas_copy(B, S.f(rs, sp), S.f(b, P64), S.st));
  for (int j = 0; j < n; ++j) {
    BT(blas_copy(B, ps[j], S.f(rs, sp), S.st));
    BT(blas_zero(B, xs[j], S.st));
  }
  ShiftTable tab{};
  for (int j = 0; j < n; ++j) tab.v[j] = shifts[j];
  KC((k_init<<<1, 1, 0, S.st>>>(S.S)));
  KC((k_ms_init<<<1, 1, 0, S.st>>>(S.S, n, tab)));
  BT(blas_norm2(B, S.f(rs, sp), nullptr, S.st, S.slot(S_RR)));
  const double tol2bb = ms_tol * ms_tol * bb;
  S.shift = shifts[j0];
  int it = 0, last = -1;
  while (S.stats->iters < P.max_iter) {
    last = it;
    TRY(S.A(Ap, ps[j0].p, sp));
    BT(blas_cdot_norm(B, ps[j0], S.f(Ap, sp), nullptr, S.st, S.slot(S_PAP)));
    KC((k_ms1<<<1, 1, 0, S.st>>>(S.S)));
    BT(blas_caxpy_norm(B, cptr(S.slot(S_NALPHA)), S.f(Ap, sp), S.f(rs, sp), nullptr, S.st, S.slot(S_RN)));
    KC((k_ms2<<<1, 1, 0, S.st>>>(S.S, n, j0, tol2bb, S.mirror, it & 1, it)));
    BT(blas_multishift_update(B, n, xs.data(), ps.data(), S.f(rs, sp), S.slot(S_MSC), S.st));
    TRY(S.mark(it));
    S.stats->iters++;
    if (it > 0) {
      double worst;
      int fl;
      TRY(S.read(it - 1, &worst, &fl));
      if (fl != FLAG_OK) return flag_error(S, fl, "multi-shift CG");
      if (S.hmirror[4 * ((it - 1) & 1) + 3] == 0) break;  // every shift converged
    }
    ++it;
  }
  if (last >= 0) {
    double worst;
    int fl;
    TRY(S.read(last, &worst, &fl));
    if (fl != FLAG_OK) return flag_error(S, fl, "multi-shift CG");
  }
  for (int j = 0; j < n; ++j) BT(blas_copy(B, S.f(xout[j], P64), xs[j], S.st));
  return DIRAC_OK;
}

int ensure_scalars(dirac_ctx* c) {
  if (!c->dscal && cudaMalloc(&c->dscal, sizeof(double) * S_END) != cudaSuccess) {
    cudaGetLastError();
    c->dscal = nullptr;
    return set_err(c, DIRAC_ERR_OOM, "solver scalars");
  }
  if (!c->hmirror) {
    if (cudaHostAlloc(&c->hmirror, sizeof(double) * 16, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&c->dmirror, c->hmirror, 0) != cudaSuccess) {
      cudaGetLastError();
      if (c->hmirror) cudaFreeHost(c->hmirror);
      c->hmirror = nullptr;
      return set_err(c, DIRAC_ERR_OOM, "solver mirror");
    }
  }
  return DIRAC_OK;
}

// operator flops per application (Wilson-clover 1872/site, plain Wilson 1368/site,
// asqtad hopping term 1146/output site plus the diagonal)
double op_flops(const dirac_ctx* c, int which, int parity) {
  if (c->p.kind == DIRAC_WILSON_CLOVER && which >= 3)  // Schur: 2 hops + Ahat + Ahat^-1
    return (double)c->Vh * (2 * 1320.0 + (c->p.csw != 0 ? 2 * 504.0 : 0.0) + 48.0);
  if (c->p.kind == DIRAC_WILSON_CLOVER)
    return (double)c->V * (c->p.csw != 0 ? 1872.0 : 1368.0) * (which == 2 ? 2 : 1);
  return which == 2 ? (parity >= 0 ? 2.0 * 1146.0 * c->Vh + 12.0 * c->Vh : 2.0 * 1158.0 * c->V)
                    : 1158.0 * c->V;
}

// final FP64 true residual ||b - A x|| / ||b|| into stats; NOT_CONVERGED above tol
int finish_stats(Ctx& S, const char* x, const char* b, double tol) {
  S.next = 0;
  char* r = S.get(P64);
  if (!r) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  double rr = 0, bb = 0;
  int rc = blas_norm2(S.c->blas, S.f(b, P64), &bb, S.st);
  if (rc) return set_err(S.c, rc, blas_error(S.c->blas));
  TRY(S.A(r, x, P64));
  S.stats->dslash_calls -= 1;
  S.stats->flops -= S.flops_per_apply;
  rc = blas_xmy_norm(S.c->blas, S.f(b, P64), S.f(r, P64), &rr, S.st);
  if (rc) return set_err(S.c, rc, blas_error(S.c->blas));
  if (!std::isfinite(bb) || !std::isfinite(rr)) {
    S.stats->true_rel_resid = NAN;
    return set_err(S.c, DIRAC_ERR_NONFINITE, "non-finite true residual");
  }
  S.stats->true_rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  if (!std::isfinite(S.stats->true_rel_resid)) return set_err(S.c, DIRAC_ERR_NONFINITE, "non-finite true residual");
  if (S.stats->true_rel_resid > tol) return set_err(S.c, DIRAC_ERR_NOT_CONVERGED, "max_iter reached");
  return DIRAC_OK;
}

}  // namespace

}  // namespace dirac

using namespace dirac;

extern "C" int solve_multishift(dirac_ctx* c, void* const* x, const void* b, const double* shifts, int nshift,
                                const dirac_solver_params* params, dirac_solver_stats* stats, void* stream) {
  if (!c || !x || !b || !shifts || !params || nshift < 1 || nshift > KSH)
    return set_err(c, DIRAC_ERR_ARG, "bad multi-shift arguments (1..16 shifts)");
  const dirac_solver_params& P = *params;
  for (int j = 0; j < nshift; ++j) {
    if (!x[j] || x[j] == b) return set_err(c, DIRAC_ERR_ARG, "null or aliased solution field");
    if (!(shifts[j] >= 0) || !std::isfinite(shifts[j])) return set_err(c, DIRAC_ERR_ARG, "shifts must be >= 0");
    for (int i = 0; i < j; ++i)
      if (x[i] == x[j]) return set_err(c, DIRAC_ERR_ARG, "solution fields must be distinct");
  }
  int parity;
  if (P.alg == DIRAC_SOLVER_CG_NORMAL) parity = -1;
  else if (P.alg == DIRAC_SOLVER_CG_EVEN_NORMAL && c->p.kind == DIRAC_ASQTAD) parity = 0;
  else return set_err(c, DIRAC_ERR_UNSUPPORTED, "multi-shift needs CG_NORMAL or asqtad CG_EVEN_NORMAL");
  if (!(P.tol > 0) || P.max_iter < 0 || P.delta < 0) return set_err(c, DIRAC_ERR_ARG, "bad tolerances");
  int rc;
  if ((rc = check_op(c, P64, false))) return rc;
  if ((rc = check_op(c, P.prec_sloppy, false))) return rc;
  if ((rc = ensure_scalars(c))) return rc;
  std::vector<dirac_solver_stats> local(nshift + 1);
  dirac_solver_stats* st = stats ? stats : local.data();
  for (int j = 0; j <= nshift; ++j) st[j] = dirac_solver_stats{};
  cudaStream_t s = (cudaStream_t)stream;
  Ctx S{c, s, parity, 2, 0, st, 0};
  S.S = c->dscal;
  S.mirror = c->dmirror;
  S.hmirror = c->hmirror;
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&S.ev[i], cudaEventDisableTiming) != cudaSuccess)
      return set_err(c, DIRAC_ERR_CUDA, "cudaEventCreate");
  S.flops_per_apply = op_flops(c, 2, parity);
  // stage 1: the multi-shift solve in the sloppy precision, as far as it can resolve
  const double ms_tol = P.prec_sloppy == DIRAC_PREC_F64 ? P.tol
                       : std::max(P.tol, P.prec_sloppy == DIRAC_PREC_F32 ? 1e-6 : 1e-3);
  auto t0 = std::chrono::steady_clock::now();
  rc = solve_ms_stage(S, (char* const*)x, (const char*)b, shifts, nshift, P, ms_tol);
  cudaStreamSynchronize(s);
  st[0].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // stage 2: refine each x_j with mixed-precision CG on its own shifted system
  for (int j = 0; rc == DIRAC_OK && j < nshift; ++j) {
    S.stats = &st[1 + j];
    S.shift = shifts[j];
    S.next = 0;
    auto t1 = std::chrono::steady_clock::now();
    dirac_solver_params Pj = P;
    Pj.use_x0 = 1;
    rc = solve_cg(S, (char*)x[j], (const char*)b, Pj);
    if (rc == DIRAC_OK) rc = finish_stats(S, (const char*)x[j], (const char*)b, P.tol);
    cudaStreamSynchronize(s);
    st[1 + j].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
  }
  cudaError_t e = cudaStreamSynchronize(s);
  for (int i = 0; i < 2; ++i) cudaEventDestroy(S.ev[i]);
  if (rc == DIRAC_OK && e != cudaSuccess) rc = set_err(c, DIRAC_ERR_CUDA, cudaGetErrorString(e));
  return rc;
}

extern "C" int solve(dirac_ctx* c, void* x, const void* b, const dirac_solver_params* params,
                     dirac_solver_stats* stats, void* stream) {
  Range range("solve");
  if (!c || !x || !b || !params || x == b) return set_err(c, DIRAC_ERR_ARG, "bad solve arguments");
  const dirac_solver_params& P = *params;
  const bool wil = c->p.kind == DIRAC_WILSON_CLOVER;
  int parity = -1, which = 0;
  bool eo = false;
  switch (P.alg) {
    case DIRAC_SOLVER_BICGSTAB_EO:
    case DIRAC_SOLVER_GCR_EO:
      if (!wil) return set_err(c, DIRAC_ERR_UNSUPPORTED, "even-odd solvers need the Wilson-clover operator");
      which = 3; parity = 0; eo = true; break;
    case DIRAC_SOLVER_CG_NORMAL: which = 2; break;
    case DIRAC_SOLVER_CG_EVEN_NORMAL:
      if (wil) return set_err(c, DIRAC_ERR_UNSUPPORTED, "CG_EVEN_NORMAL needs the asqtad operator");
      which = 2; parity = 0; break;
    case DIRAC_SOLVER_BICGSTAB:
    case DIRAC_SOLVER_GCR: which = 0; break;
    case DIRAC_SOLVER_GCR_DD:
    case DIRAC_SOLVER_GCR_PTC:
      if (!wil) return set_err(c, DIRAC_ERR_UNSUPPORTED, "GCR_DD / GCR_PTC need the Wilson-clover operator");
      which = 0; break;
    default: return set_err(c, DIRAC_ERR_ARG, "unknown solver");
  }
  if (!(P.tol > 0) || P.max_iter < 0 || P.delta < 0) return set_err(c, DIRAC_ERR_ARG, "bad tolerances");
  int rc;
  if ((rc = check_op(c, P64, false))) return rc;
  if ((rc = check_op(c, P.prec_sloppy, false))) return rc;
  if ((P.alg == DIRAC_SOLVER_GCR_DD || P.alg == DIRAC_SOLVER_GCR_PTC) && (rc = check_op(c, P.prec_precond, false)))
    return rc;
  if (P.alg == DIRAC_SOLVER_GCR_PTC && (rc = check_op(c, P32, false))) return rc;
  if ((rc = ensure_scalars(c))) return rc;
  dirac_solver_stats local{};
  dirac_solver_stats* st = stats ? stats : &local;
  *st = dirac_solver_stats{};
  st->precond_rate[0] = st->precond_rate[1] = -1.0;
  // The solve runs on the context's own non-blocking stream, ordered after the caller's
  // stream: GCR captures its steps as CUDA graphs, which the legacy default stream
  // cannot do. The call returns after the solve finished (synchronously).
  cudaStream_t caller = (cudaStream_t)stream;
  if (!c->solve_stream && cudaStreamCreateWithFlags(&c->solve_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c->solve_stream = nullptr;
    return set_err(c, DIRAC_ERR_CUDA, "solver stream");
  }
  if (!c->solve_event && cudaEventCreateWithFlags(&c->solve_event, cudaEventDisableTiming) != cudaSuccess) {
    c->solve_event = nullptr;
    return set_err(c, DIRAC_ERR_CUDA, "solver event");
  }
  cudaEventRecord(c->solve_event, caller);
  cudaStreamWaitEvent(c->solve_stream, c->solve_event, 0);
  cudaStream_t s = c->solve_stream;
  Ctx S{c, s, parity, which, 0, st, 0};
  S.graphs = true;
  S.S = c->dscal;
  S.mirror = c->dmirror;
  S.hmirror = c->hmirror;
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&S.ev[i], cudaEventDisableTiming) != cudaSuccess)
      return set_err(c, DIRAC_ERR_CUDA, "cudaEventCreate");
  S.flops_per_apply = op_flops(c, which, parity);
  auto t0 = std::chrono::steady_clock::now();
  if (eo) {
    // Sec. 3.1: solve the Schur complement system on the even sites, then rebuild x_o.
    // The even half of the caller's full field x is the even half-field solved for.
    char* bhat = S.get(P64);
    if (!bhat) rc = set_err(c, DIRAC_ERR_OOM, "solver workspace");
    else rc = schur_source(c, bhat, (const char*)b, P64, s);
    if (rc == DIRAC_OK) {
      if (P.alg == DIRAC_SOLVER_BICGSTAB_EO) rc = solve_bicgstab(S, (char*)x, bhat, P);
      else rc = solve_gcr(S, (char*)x, bhat, P, K_NONE);
    }
    if (rc == DIRAC_OK) rc = schur_reconstruct(c, (char*)x, (const char*)b, P64, s);
    // the final check is on the full system M x = b
    S.which = 0;
    S.parity = -1;
    S.flops_per_apply = op_flops(c, 0, -1);
  } else {
    switch (P.alg) {
      case DIRAC_SOLVER_CG_NORMAL:
      case DIRAC_SOLVER_CG_EVEN_NORMAL: rc = solve_cg(S, (char*)x, (const char*)b, P); break;
      case DIRAC_SOLVER_BICGSTAB: rc = solve_bicgstab(S, (char*)x, (const char*)b, P); break;
      case DIRAC_SOLVER_GCR_DD: rc = solve_gcr(S, (char*)x, (const char*)b, P, K_SCHWARZ); break;
      case DIRAC_SOLVER_GCR_PTC: rc = solve_gcr(S, (char*)x, (const char*)b, P, K_SELECT); break;
      default: rc = solve_gcr(S, (char*)x, (const char*)b, P, K_NONE); break;
    }
  }
  if (rc == DIRAC_OK) rc = finish_stats(S, (const char*)x, (const char*)b, P.tol);
  cudaError_t e = cudaStreamSynchronize(s);
  st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < 2; ++i) cudaEventDestroy(S.ev[i]);
  if (rc == DIRAC_OK && e != cudaSuccess) rc = set_err(c, DIRAC_ERR_CUDA, cudaGetErrorString(e));
  return rc;
}
