// Krylov solvers behind solve(): CG on the normal equations, BiCGstab (Sec. 3.1) and
// the mixed-precision flexible GCR of Algorithm 1 with the Schwarz preconditioner
// (Sec. 8.1). The outer iterate x, the source b and the restart / reliable-update
// residual live in FP64; the Krylov vectors and the inner operator use the sloppy
// precision; the preconditioner runs in its own precision. Scalars are computed on
// the host from FP64-accumulated device reductions.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace dirac {

using cplx = std::complex<double>;

namespace {

struct Ctx {
  dirac_ctx* c;
  cudaStream_t st;
  int parity;   // -1 full, 0 even (CG_EVEN_NORMAL)
  int which;    // operator: 0 = M, 2 = normal
  int next = 0;
  dirac_solver_stats* stats;
  double flops_per_apply = 0;

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
    return apply_op(c, out, in, parity, prec, which, st);
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

bool finite(double v) { return std::isfinite(v); }

// The sloppy solution correction between reliable updates is accumulated in at least
// FP32: with 16-bit storage the late, small updates of a cycle would fall below the
// 11-bit resolution of the accumulated correction and be lost.
int accum_prec(int sp) { return sp == P16 ? P32 : sp; }

// r = b - A x in FP64, returns ||r||^2
int true_residual(Ctx& S, char* r, const char* x, const char* b, double* rr) {
  TRY(S.A(r, x, P64));
  BT(blas_xmy_norm(S.c->blas, S.f(b, P64), S.f(r, P64), rr, S.st));
  return DIRAC_OK;
}

// ------------------------------------------------------------------ CG (Sec. 3.1)
int solve_cg(Ctx& S, char* x, const char* b, const dirac_solver_params& P) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy;
  const int ap = accum_prec(sp);
  char *r = S.get(P64), *rs = S.get(sp), *p = S.get(sp), *Ap = S.get(sp), *xs = S.get(ap);
  if (!r || !rs || !p || !Ap || !xs) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (bb == 0.0) {
    BT(blas_zero(B, S.f(x, P64), S.st));
    return DIRAC_OK;
  }
  const double target = P.tol * P.tol * bb;
  double rr;
  if (P.use_x0) {
    TRY(true_residual(S, r, x, b, &rr));
  } else {
    BT(blas_zero(B, S.f(x, P64), S.st));
    BT(blas_copy(B, S.f(r, P64), S.f(b, P64), S.st));
    rr = bb;
  }
  BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
  BT(blas_copy(B, S.f(p, sp), S.f(rs, sp), S.st));
  BT(blas_zero(B, S.f(xs, ap), S.st));
  double rr_s = rr, rmax = rr;
  const double d2 = P.delta * P.delta;
  bool converged = rr < target;
  while (!converged && S.stats->iters < P.max_iter) {
    TRY(S.A(Ap, p, sp));
    double pAp[3];
    BT(blas_cdot_norm(B, S.f(p, sp), S.f(Ap, sp), pAp, S.st));
    if (!finite(pAp[0])) return set_err(S.c, DIRAC_ERR_NONFINITE, "CG: non-finite (p, Ap)");
    if (pAp[0] <= 0.0) return set_err(S.c, DIRAC_ERR_BREAKDOWN, "CG: (p, Ap) <= 0");
    const double alpha = rr_s / pAp[0];
    BT(blas_axpby(B, alpha, 0, S.f(p, sp), 1, 0, S.f(xs, ap), S.st));
    double rr_new;
    BT(blas_caxpy_norm(B, -alpha, 0, S.f(Ap, sp), S.f(rs, sp), &rr_new, S.st));
    S.stats->iters++;
    if (!finite(rr_new)) return set_err(S.c, DIRAC_ERR_NONFINITE, "CG: non-finite residual");
    if ((d2 > 0 && rr_new < d2 * rmax) || rr_new < target) {
      // reliable update: fold the sloppy correction into x, recompute r in FP64
      BT(blas_axpby(B, 1, 0, S.f(xs, ap), 1, 0, S.f(x, P64), S.st));
      BT(blas_zero(B, S.f(xs, ap), S.st));
      TRY(true_residual(S, r, x, b, &rr));
      S.stats->reliable_updates++;
      if (rr < target) { converged = true; break; }
      BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
      rr_new = rr;
      rmax = rr;
    }
    const double beta = rr_new / rr_s;
    BT(blas_axpby(B, 1, 0, S.f(rs, sp), beta, 0, S.f(p, sp), S.st));
    rr_s = rr_new;
  }
  if (!converged) {
    BT(blas_axpby(B, 1, 0, S.f(xs, ap), 1, 0, S.f(x, P64), S.st));
  }
  return DIRAC_OK;
}

// ------------------------------------------------------------------ BiCGstab (Sec. 3.1)
int solve_bicgstab(Ctx& S, char* x, const char* b, const dirac_solver_params& P) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy;
  const int ap = accum_prec(sp);
  char *r = S.get(P64), *rs = S.get(sp), *r0 = S.get(sp), *p = S.get(sp), *v = S.get(sp),
       *t = S.get(sp), *xs = S.get(ap);
  if (!r || !rs || !r0 || !p || !v || !t || !xs) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (bb == 0.0) {
    BT(blas_zero(B, S.f(x, P64), S.st));
    return DIRAC_OK;
  }
  const double target = P.tol * P.tol * bb;
  double rr;
  if (P.use_x0) {
    TRY(true_residual(S, r, x, b, &rr));
  } else {
    BT(blas_zero(B, S.f(x, P64), S.st));
    BT(blas_copy(B, S.f(r, P64), S.f(b, P64), S.st));
    rr = bb;
  }
  BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
  BT(blas_copy(B, S.f(r0, sp), S.f(rs, sp), S.st));
  BT(blas_zero(B, S.f(p, sp), S.st));
  BT(blas_zero(B, S.f(v, sp), S.st));
  BT(blas_zero(B, S.f(xs, ap), S.st));
  cplx rho(1, 0), alpha(1, 0), omega(1, 0), rho_new;
  {
    double d[2];
    BT(blas_cdot(B, S.f(r0, sp), S.f(rs, sp), d, S.st));
    rho_new = cplx(d[0], d[1]);
  }
  double rmax = rr;
  const double d2 = P.delta * P.delta;
  bool converged = rr < target;
  while (!converged && S.stats->iters < P.max_iter) {
    if (std::abs(rho_new) == 0.0) return set_err(S.c, DIRAC_ERR_BREAKDOWN, "BiCGstab: rho = 0");
    const cplx beta = (rho_new / rho) * (alpha / omega);
    // p = r + beta (p - omega v)
    BT(blas_axpby(B, 1, 0, S.f(rs, sp), beta.real(), beta.imag(), S.f(p, sp), S.st));
    const cplx bw = -beta * omega;
    BT(blas_axpby(B, bw.real(), bw.imag(), S.f(v, sp), 1, 0, S.f(p, sp), S.st));
    TRY(S.A(v, p, sp));
    double sg[2];
    BT(blas_cdot(B, S.f(r0, sp), S.f(v, sp), sg, S.st));
    const cplx sigma(sg[0], sg[1]);
    if (!finite(sg[0]) || !finite(sg[1])) return set_err(S.c, DIRAC_ERR_NONFINITE, "BiCGstab: non-finite");
    if (std::abs(sigma) == 0.0) return set_err(S.c, DIRAC_ERR_BREAKDOWN, "BiCGstab: (r0, v) = 0");
    alpha = rho_new / sigma;
    double ss;  // s = r - alpha v (in rs)
    BT(blas_caxpy_norm(B, -alpha.real(), -alpha.imag(), S.f(v, sp), S.f(rs, sp), &ss, S.st));
    TRY(S.A(t, rs, sp));
    double ts[3];
    BT(blas_cdot_norm(B, S.f(t, sp), S.f(rs, sp), ts, S.st));
    if (ts[2] == 0.0) return set_err(S.c, DIRAC_ERR_BREAKDOWN, "BiCGstab: (t, t) = 0");
    omega = cplx(ts[0], ts[1]) / ts[2];
    BT(blas_axpbz_add(B, alpha.real(), alpha.imag(), S.f(p, sp), omega.real(), omega.imag(), S.f(rs, sp),
                      S.f(xs, ap), S.st));
    double out[3];  // r = s - omega t ; ||r||^2 ; (r0, r)
    BT(blas_caxpy_norm_dot(B, -omega.real(), -omega.imag(), S.f(t, sp), S.f(rs, sp), S.f(r0, sp), out, S.st));
    rho = rho_new;
    rho_new = cplx(out[1], out[2]);
    double rr_new = out[0];
    S.stats->iters++;
    if (!finite(rr_new)) return set_err(S.c, DIRAC_ERR_NONFINITE, "BiCGstab: non-finite residual");
    if ((d2 > 0 && rr_new < d2 * rmax) || rr_new < target) {
      BT(blas_axpby(B, 1, 0, S.f(xs, ap), 1, 0, S.f(x, P64), S.st));
      BT(blas_zero(B, S.f(xs, ap), S.st));
      TRY(true_residual(S, r, x, b, &rr));
      S.stats->reliable_updates++;
      if (rr < target) { converged = true; break; }
      BT(blas_copy(B, S.f(rs, sp), S.f(r, P64), S.st));
      double d[2];
      BT(blas_cdot(B, S.f(r0, sp), S.f(rs, sp), d, S.st));
      rho_new = cplx(d[0], d[1]);
      rmax = rr;
    }
  }
  if (!converged) {
    BT(blas_axpby(B, 1, 0, S.f(xs, ap), 1, 0, S.f(x, P64), S.st));
  }
  return DIRAC_OK;
}

// ------------------------------------------------------------------ GCR (Algorithm 1)
int solve_gcr(Ctx& S, char* x, const char* b, const dirac_solver_params& P, bool precond) {
  Blas* B = S.c->blas;
  const int sp = P.prec_sloppy, pp = P.prec_precond;
  const int kmax = P.k_max;
  if (kmax < 1 || kmax > 20) return set_err(S.c, DIRAC_ERR_ARG, "k_max must be in [1, 20]");
  char* r = S.get(P64);
  char* rh = S.get(sp);
  std::vector<char*> pv(kmax), zv(kmax);
  for (int i = 0; i < kmax; ++i) {
    pv[i] = S.get(sp);
    zv[i] = S.get(sp);
  }
  char *pin = nullptr, *pout = nullptr;
  if (precond && pp != sp) {
    pin = S.get(pp);
    pout = S.get(pp);
    if (!pin || !pout) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  }
  if (!r || !rh) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");
  for (int i = 0; i < kmax; ++i)
    if (!pv[i] || !zv[i]) return set_err(S.c, DIRAC_ERR_OOM, "solver workspace");

  double bb;
  BT(blas_norm2(B, S.f(b, P64), &bb, S.st));
  if (bb == 0.0) {
    BT(blas_zero(B, S.f(x, P64), S.st));
    return DIRAC_OK;
  }
  const double target = P.tol * P.tol * bb;
  double r0n2;
  if (P.use_x0) {
    TRY(true_residual(S, r, x, b, &r0n2));
  } else {
    BT(blas_zero(B, S.f(x, P64), S.st));
    BT(blas_copy(B, S.f(r, P64), S.f(b, P64), S.st));
    r0n2 = bb;
  }
  BT(blas_copy(B, S.f(rh, sp), S.f(r, P64), S.st));
  std::vector<cplx> beta(kmax * kmax), alpha(kmax), chi(kmax);
  std::vector<double> gamma(kmax);
  const double d2 = P.delta * P.delta;
  const double kflops = (double)S.c->V * P.k_max * 0;  // BLAS flops not counted
  (void)kflops;
  const double sflops = (double)S.c->V * S.c->p.mr_steps * (1872.0 + 192.0);
  int k = 0;
  while (r0n2 > target && S.stats->iters < P.max_iter) {
    // p_k = K r_k
    if (precond) {
      S.stats->precond_calls++;
      S.stats->flops += sflops;
      if (pp == sp) {
        TRY(schwarz_apply(S.c, pv[k], rh, sp, S.st));
      } else {
        BT(blas_copy(B, S.f(pin, pp), S.f(rh, sp), S.st));
        TRY(schwarz_apply(S.c, pout, pin, pp, S.st));
        BT(blas_copy(B, S.f(pv[k], sp), S.f(pout, pp), S.st));
      }
    } else {
      BT(blas_copy(B, S.f(pv[k], sp), S.f(rh, sp), S.st));
    }
    // z_k = M p_k
    TRY(S.A(zv[k], pv[k], sp));
    // modified Gram-Schmidt: beta_ik = (z_i, z_k); z_k -= beta_ik z_i. Each pass
    // subtracts the previous projection and forms the next inner product.
    double zz;
    if (k == 0) {
      BT(blas_norm2(B, S.f(zv[0], sp), &zz, S.st));
    } else {
      double d[2];
      BT(blas_cdot(B, S.f(zv[0], sp), S.f(zv[k], sp), d, S.st));
      beta[0 * kmax + k] = cplx(d[0], d[1]);
      for (int i = 1; i < k; ++i) {
        const cplx bm = -beta[(i - 1) * kmax + k];
        double o[3];
        BT(blas_caxpy_norm_dot(B, bm.real(), bm.imag(), S.f(zv[i - 1], sp), S.f(zv[k], sp), S.f(zv[i], sp), o,
                               S.st));
        beta[i * kmax + k] = cplx(o[1], o[2]);
      }
      const cplx bm = -beta[(k - 1) * kmax + k];
      BT(blas_caxpy_norm(B, bm.real(), bm.imag(), S.f(zv[k - 1], sp), S.f(zv[k], sp), &zz, S.st));
    }
    if (!finite(zz)) return set_err(S.c, DIRAC_ERR_NONFINITE, "GCR: non-finite ||z||");
    if (zz <= 0.0) return set_err(S.c, DIRAC_ERR_BREAKDOWN, "GCR: z_k vanished after orthogonalisation");
    gamma[k] = std::sqrt(zz);
    double a2[2];
    BT(blas_scale_cdot(B, 1.0 / gamma[k], S.f(zv[k], sp), S.f(rh, sp), a2, S.st));
    alpha[k] = cplx(a2[0], a2[1]);
    double rr;
    BT(blas_caxpy_norm(B, -a2[0], -a2[1], S.f(zv[k], sp), S.f(rh, sp), &rr, S.st));
    ++k;
    S.stats->iters++;
    if (!finite(rr)) return set_err(S.c, DIRAC_ERR_NONFINITE, "GCR: non-finite residual");
    if (k == kmax || (d2 > 0 && rr < d2 * r0n2) || rr < target || S.stats->iters >= P.max_iter) {
      // back-substitution: gamma_l chi_l + sum_{i>l} beta_li chi_i = alpha_l
      for (int l = k - 1; l >= 0; --l) {
        cplx s = alpha[l];
        for (int i = l + 1; i < k; ++i) s -= beta[l * kmax + i] * chi[i];
        chi[l] = s / gamma[l];
      }
      std::vector<double> cr(k), ci(k);
      std::vector<FieldRef> xs(k);
      for (int i = 0; i < k; ++i) {
        cr[i] = chi[i].real();
        ci[i] = chi[i].imag();
        xs[i] = S.f(pv[i], sp);
      }
      BT(blas_multi_caxpy(B, k, cr.data(), ci.data(), xs.data(), S.f(x, P64), S.st));
      TRY(true_residual(S, r, x, b, &r0n2));
      if (!finite(r0n2)) return set_err(S.c, DIRAC_ERR_NONFINITE, "GCR: non-finite true residual");
      BT(blas_copy(B, S.f(rh, sp), S.f(r, P64), S.st));
      S.stats->restarts++;
      k = 0;
    }
  }
  return DIRAC_OK;
}

}  // namespace

}  // namespace dirac

using namespace dirac;

extern "C" int solve(dirac_ctx* c, void* x, const void* b, const dirac_solver_params* params,
                     dirac_solver_stats* stats, void* stream) {
  if (!c || !x || !b || !params || x == b) return set_err(c, DIRAC_ERR_ARG, "bad solve arguments");
  const dirac_solver_params& P = *params;
  const bool wil = c->p.kind == DIRAC_WILSON_CLOVER;
  int parity = -1, which = 0;
  switch (P.alg) {
    case DIRAC_SOLVER_CG_NORMAL: which = 2; break;
    case DIRAC_SOLVER_CG_EVEN_NORMAL:
      if (wil) return set_err(c, DIRAC_ERR_UNSUPPORTED, "CG_EVEN_NORMAL needs the asqtad operator");
      which = 2; parity = 0; break;
    case DIRAC_SOLVER_BICGSTAB:
    case DIRAC_SOLVER_GCR: which = 0; break;
    case DIRAC_SOLVER_GCR_DD:
      if (!wil) return set_err(c, DIRAC_ERR_UNSUPPORTED, "GCR_DD needs the Wilson-clover operator");
      which = 0; break;
    default: return set_err(c, DIRAC_ERR_ARG, "unknown solver");
  }
  if (!(P.tol > 0) || P.max_iter < 0 || P.delta < 0) return set_err(c, DIRAC_ERR_ARG, "bad tolerances");
  int rc;
  if ((rc = check_op(c, P64, false))) return rc;
  if ((rc = check_op(c, P.prec_sloppy, false))) return rc;
  if (P.alg == DIRAC_SOLVER_GCR_DD && (rc = check_op(c, P.prec_precond, false))) return rc;
  dirac_solver_stats local{};
  dirac_solver_stats* st = stats ? stats : &local;
  *st = dirac_solver_stats{};
  cudaStream_t s = (cudaStream_t)stream;
  Ctx S{c, s, parity, which, 0, st, 0};
  // operator flops per application (counts in the design doc)
  if (wil) S.flops_per_apply = (double)c->V * (c->p.csw != 0 ? 1872.0 : 1368.0) * (which == 2 ? 2 : 1);
  else S.flops_per_apply = which == 2 ? (parity >= 0 ? 2.0 * 1146.0 * c->Vh + 12.0 * c->Vh : 2.0 * 1158.0 * c->V)
                                      : 1158.0 * c->V;
  auto t0 = std::chrono::steady_clock::now();
  switch (P.alg) {
    case DIRAC_SOLVER_CG_NORMAL:
    case DIRAC_SOLVER_CG_EVEN_NORMAL: rc = solve_cg(S, (char*)x, (const char*)b, P); break;
    case DIRAC_SOLVER_BICGSTAB: rc = solve_bicgstab(S, (char*)x, (const char*)b, P); break;
    case DIRAC_SOLVER_GCR_DD: rc = solve_gcr(S, (char*)x, (const char*)b, P, true); break;
    default: rc = solve_gcr(S, (char*)x, (const char*)b, P, false); break;
  }
  if (rc == DIRAC_OK) {
    // final FP64 true residual ||b - A x|| / ||b||
    S.next = 0;
    char* r = S.get(P64);
    double rr = 0, bb = 0;
    if (!r) return set_err(c, DIRAC_ERR_OOM, "solver workspace");
    if ((rc = blas_norm2(c->blas, S.f(b, P64), &bb, s))) return set_err(c, rc, blas_error(c->blas));
    if ((rc = S.A(r, (const char*)x, P64))) return rc;
    st->dslash_calls -= 1;
    st->flops -= S.flops_per_apply;
    if ((rc = blas_xmy_norm(c->blas, S.f(b, P64), S.f(r, P64), &rr, s))) return set_err(c, rc, blas_error(c->blas));
    st->true_rel_resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    if (!std::isfinite(st->true_rel_resid)) rc = set_err(c, DIRAC_ERR_NONFINITE, "non-finite true residual");
    else if (st->true_rel_resid > P.tol) rc = set_err(c, DIRAC_ERR_NOT_CONVERGED, "max_iter reached");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == DIRAC_OK && e != cudaSuccess) rc = set_err(c, DIRAC_ERR_CUDA, cudaGetErrorString(e));
  return rc;
}
