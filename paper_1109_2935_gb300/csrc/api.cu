// The C ABI of libdirac (declared in include/dirac.h): context lifecycle, gauge and
// spinor loading, operator application, the Schwarz preconditioner and BLAS-1.
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"
#include "wilson.cuh"

using namespace dirac;

namespace dirac {

int set_err(dirac_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(dirac_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(c, DIRAC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return DIRAC_OK;
}

static int dalloc(dirac_ctx* c, char** p, size_t bytes) {
  if (*p) return DIRAC_OK;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(c, DIRAC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  return DIRAC_OK;
}

FieldRef field_ref(const dirac_ctx* c, const void* p, int prec, int parity) {
  FieldRef f;
  f.p = (char*)p;
  f.prec = prec;
  f.nr = c->nr;
  f.Vh = (int)c->Vh;
  f.npar = parity < 0 ? 2 : 1;
  f.hb = spinor_half_bytes(prec, c->nr, c->Vh);
  return f;
}

static bool valid_prec(int p) { return p == P64 || p == P32 || p == P16; }

int check_op(dirac_ctx* c, int prec, bool need_schwarz) {
  if (!c) return DIRAC_ERR_ARG;
  if (!valid_prec(prec)) return set_err(c, DIRAC_ERR_ARG, "unknown precision");
  if (!(c->mask & (1u << prec))) return set_err(c, DIRAC_ERR_UNSUPPORTED, "precision not in prec_mask");
  if (c->p.kind == DIRAC_WILSON_CLOVER && !c->have_gauge)
    return set_err(c, DIRAC_ERR_STATE, "gauge field not loaded");
  if (c->p.kind == DIRAC_ASQTAD && !(c->have_fat && c->have_long))
    return set_err(c, DIRAC_ERR_STATE, "fat and long links not loaded");
  (void)need_schwarz;
  return DIRAC_OK;
}

int ensure_tmp(dirac_ctx* c, int prec) {
  size_t b = 2 * spinor_half_bytes(prec, c->nr, c->Vh);
  int rc = dalloc(c, &c->tmp[prec], b);
  if (rc) return rc;
  return dalloc(c, &c->tmp2[prec], b);
}

static void wilson_launch(int prec, int recon, bool fullm, const WilsonArg& a, cudaStream_t st) {
  if (prec == P64) launch_wilson_p64(recon, fullm, a, st);
  else if (prec == P32) launch_wilson_p32(recon, fullm, a, st);
  else launch_wilson_p16(recon, fullm, a, st);
}

// Wilson: full M (or M^dagger) on full fields.
int wilson_M(dirac_ctx* c, char* out, const char* in, int prec, bool dag, cudaStream_t st) {
  WilsonArg a;
  size_t hb = spinor_half_bytes(prec, 24, c->Vh);
  a.out[0] = out; a.out[1] = out + hb;
  a.in[0] = in; a.in[1] = in + hb;
  a.gauge = c->gauge[prec];
  a.clover = c->p.csw != 0.0 ? c->clover[prec] : nullptr;
  a.g = c->g;
  a.kappa = c->p.kappa;
  a.dagger = dag;
  a.out_parity = 0;
  wilson_launch(prec, c->p.recon[prec], true, a, st);
  return cuda_check(c, "wilson M kernel");
}

// Wilson, half-fields: out_p = Cpost (Cself self_p + s D_{p,1-p} in_{1-p}) (defaults:
// the plain hopping block out_p = D_{p,1-p} in_{1-p}).
int wilson_hop(dirac_ctx* c, char* out, const char* in, int parity, int prec, bool dag, cudaStream_t st,
               double s, const char* self, const char* c_self, const char* c_post) {
  WilsonArg a;
  a.out[0] = a.out[1] = out;
  a.in[0] = a.in[1] = in;
  a.gauge = c->gauge[prec];
  a.clover = nullptr;
  a.g = c->g;
  a.kappa = c->p.kappa;
  a.dagger = dag;
  a.out_parity = parity;
  a.s = s;
  a.self = self;
  a.c_self = c_self;
  a.c_post = c_post;
  wilson_launch(prec, c->p.recon[prec], false, a, st);
  return cuda_check(c, "wilson dslash kernel");
}

// clover-format matrices for parity p (null = identity when c_sw = 0)
static const char* clov(dirac_ctx* c, int prec) { return c->p.csw != 0.0 ? c->clover[prec] : nullptr; }
static const char* clov_inv(dirac_ctx* c, int prec) { return c->p.csw != 0.0 ? c->clover_inv[prec] : nullptr; }

// Even-odd (Schur complement) operator on even half-fields (Sec. 3.1):
//   Mhat in_e = Ahat_ee in_e - kappa^2 D_eo Ahat_oo^-1 D_oe in_e
int schur_apply(dirac_ctx* c, char* out, const char* in, int prec, bool dag, cudaStream_t st) {
  int rc;
  if ((rc = ensure_tmp(c, prec))) return rc;
  char* t = c->tmp[prec];  // odd half-field
  if ((rc = wilson_hop(c, t, in, 1, prec, dag, st, 1.0, nullptr, nullptr, clov_inv(c, prec)))) return rc;
  const double k2 = c->p.kappa * c->p.kappa;
  return wilson_hop(c, out, t, 0, prec, dag, st, -k2, in, clov(c, prec), nullptr);
}

// bhat_e = b_e + kappa D_eo Ahat_oo^-1 b_o   (b full field; bhat even half-field)
int schur_source(dirac_ctx* c, char* bhat, const char* b, int prec, cudaStream_t st) {
  int rc;
  if ((rc = ensure_tmp(c, prec))) return rc;
  const size_t hb = spinor_half_bytes(prec, 24, c->Vh);
  char* t = c->tmp[prec];
  if ((rc = wilson_hop(c, t, b, 1, prec, false, st, 0.0, b + hb, clov_inv(c, prec), nullptr))) return rc;
  return wilson_hop(c, bhat, t, 0, prec, false, st, c->p.kappa, b, nullptr, nullptr);
}

// x_o = Ahat_oo^-1 (b_o + kappa D_oe x_e)   (x full field whose even half is solved)
int schur_reconstruct(dirac_ctx* c, char* x, const char* b, int prec, cudaStream_t st) {
  const size_t hb = spinor_half_bytes(prec, 24, c->Vh);
  return wilson_hop(c, x + hb, x, 1, prec, false, st, c->p.kappa, b + hb, nullptr, clov_inv(c, prec));
}

// Asqtad: out_p = a x_p + b D_{p,1-p} in_{1-p}
int stag_hop(dirac_ctx* c, char* out, const char* in, const char* x, int parity, int prec, double a,
             double b, cudaStream_t st) {
  launch_staggered(prec, c->p.recon[prec], out, in, x, c->fat[prec], c->gauge[prec], c->g, parity, a, b, st);
  return cuda_check(c, "asqtad dslash kernel");
}

// A x for the operator family; `which`: 0 = M, 1 = M^dagger, 2 = M^dagger M.
// parity: FULL, or EVEN/ODD (hopping block for M/M^dagger; (M^dagger M)_pp for asqtad).
int apply_op(dirac_ctx* c, char* out, const char* in, int parity, int prec, int which, cudaStream_t st,
             double shift) {
  const bool wil = c->p.kind == DIRAC_WILSON_CLOVER;
  const size_t hb = spinor_half_bytes(prec, c->nr, c->Vh);
  int rc;
  if (which == 2) {  // M^dagger M + shift
    if ((rc = ensure_tmp(c, prec))) return rc;
    char* t = c->tmp[prec];
    if (wil) {
      if (parity >= 0) return set_err(c, DIRAC_ERR_UNSUPPORTED, "Wilson normal operator is full-lattice only");
      if ((rc = wilson_M(c, t, in, prec, false, st))) return rc;
      if ((rc = wilson_M(c, out, t, prec, true, st))) return rc;
      if (shift != 0.0)
        return blas_axpby(c->blas, cval(shift), field_ref(c, in, prec, -1), cval(1), field_ref(c, out, prec, -1), st);
      return DIRAC_OK;
    }
    const double m2 = c->p.mass * c->p.mass + shift;
    if (parity >= 0) {  // (M^dagger M)_pp = m^2 - 1/4 D_{p,1-p} D_{1-p,p}
      if ((rc = stag_hop(c, t, in, nullptr, 1 - parity, prec, 0.0, 1.0, st))) return rc;
      return stag_hop(c, out, t, in, parity, prec, m2, -0.25, st);
    }
    for (int p = 0; p < 2; ++p)  // t = D in
      if ((rc = stag_hop(c, t + p * hb, in + (1 - p) * hb, nullptr, p, prec, 0.0, 1.0, st))) return rc;
    for (int p = 0; p < 2; ++p)  // out = m^2 in - 1/4 D t
      if ((rc = stag_hop(c, out + p * hb, t + (1 - p) * hb, in + p * hb, p, prec, m2, -0.25, st))) return rc;
    return DIRAC_OK;
  }
  if (which == 3 || which == 4) {  // even-odd Schur operator (4: adjoint), even half-fields
    if (!wil || parity != 0) return set_err(c, DIRAC_ERR_UNSUPPORTED, "Schur operator: Wilson-clover, even sites");
    return schur_apply(c, out, in, prec, which == 4, st);
  }
  const bool dag = which == 1;
  if (wil) {
    if (parity < 0) return wilson_M(c, out, in, prec, dag, st);
    return wilson_hop(c, out, in, parity, prec, dag, st, 1.0, nullptr, nullptr, nullptr);
  }
  if (parity >= 0) return stag_hop(c, out, in, nullptr, parity, prec, 0.0, dag ? -1.0 : 1.0, st);
  for (int p = 0; p < 2; ++p)  // M = m - D/2, M^dagger = m + D/2
    if ((rc = stag_hop(c, out + p * hb, in + (1 - p) * hb, in + p * hb, p, prec, c->p.mass, dag ? 0.5 : -0.5, st)))
      return rc;
  return DIRAC_OK;
}

void launch_wilson_ds(const WilsonArg& a, cudaStream_t st);

bool ds_available(const dirac_ctx* c) {
  return c->p.kind == DIRAC_WILSON_CLOVER && c->p.recon[P64] == 18 && c->gauge[P64] != nullptr &&
         (c->p.csw == 0.0 || c->clover[P64] != nullptr);
}

int wilson_M_ds(dirac_ctx* c, char* out, const char* in, bool dag, cudaStream_t st) {
  if (!ds_available(c))
    return set_err(c, DIRAC_ERR_UNSUPPORTED, "double-single operator: Wilson-clover with 18-real FP64 links");
  WilsonArg a;
  const size_t hb = spinor_half_bytes(P64, 24, c->Vh);
  a.out[0] = out; a.out[1] = out + hb;
  a.in[0] = in; a.in[1] = in + hb;
  a.gauge = c->gauge[P64];
  a.clover = c->p.csw != 0.0 ? c->clover[P64] : nullptr;
  a.g = c->g;
  a.kappa = c->p.kappa;
  a.dagger = dag;
  a.out_parity = 0;
  launch_wilson_ds(a, st);
  return cuda_check(c, "double-single wilson M kernel");
}

int schwarz_apply(dirac_ctx* c, char* out, const char* in, int prec, cudaStream_t st) {
  int rc = launch_schwarz(prec, c->p.recon[prec], out, in, c->gauge[prec], c->clover[prec], c->g,
                          c->p.block, c->p.mr_steps, c->p.kappa, st);
  if (rc) return set_err(c, rc, std::string("schwarz kernel: ") + cudaGetErrorString(cudaGetLastError()));
  return cuda_check(c, "schwarz kernel");
}

}  // namespace dirac

// ======================================================================== C ABI
extern "C" {

int dirac_create(const dirac_params* params, dirac_ctx** out) {
  if (!params || !out) return DIRAC_ERR_ARG;
  *out = nullptr;
  const dirac_params& p = *params;
  if (p.kind != DIRAC_WILSON_CLOVER && p.kind != DIRAC_ASQTAD) return DIRAC_ERR_ARG;
  int64_t V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (p.dims[mu] < 2 || (p.dims[mu] & 1)) return DIRAC_ERR_ARG;
    V *= p.dims[mu];
  }
  if (V / 2 > (int64_t)0x3fffffff) return DIRAC_ERR_ARG;
  unsigned mask = p.prec_mask ? p.prec_mask : 7u;
  if (mask & ~7u) return DIRAC_ERR_ARG;
  for (int q = 0; q < 3; ++q) {
    int r = p.recon[q] ? p.recon[q] : 18;
    if (r != 18 && r != 12 && r != 8) return DIRAC_ERR_ARG;
  }
  if (p.kind == DIRAC_WILSON_CLOVER) {
    int nbs = 1;
    for (int mu = 0; mu < 4; ++mu) {
      int b = p.block[mu] ? p.block[mu] : 1;
      if (b < 1 || p.dims[mu] % b) return DIRAC_ERR_ARG;
      nbs *= b;
    }
    if (nbs > 256) return DIRAC_ERR_ARG;
    if (p.mr_steps < 0) return DIRAC_ERR_ARG;
  }
  dirac_ctx* c = new dirac_ctx();
  c->p = p;
  for (int q = 0; q < 3; ++q) c->p.recon[q] = p.recon[q] ? p.recon[q] : 18;
  for (int mu = 0; mu < 4; ++mu) {
    if (!c->p.block[mu]) c->p.block[mu] = 1;
    c->g.L[mu] = p.dims[mu];
  }
  c->g.Lxh = p.dims[0] / 2;
  c->V = V;
  c->Vh = V / 2;
  c->g.Vh = (int)c->Vh;
  c->g.apbc = p.t_antiperiodic ? 1 : 0;
  c->nr = p.kind == DIRAC_WILSON_CLOVER ? 24 : 6;
  c->mask = mask;
  c->blas = blas_create();
  if (!c->blas) {
    delete c;
    return DIRAC_ERR_CUDA;
  }
  *out = c;
  return DIRAC_OK;
}

int dirac_destroy(dirac_ctx* c) {
  if (!c) return DIRAC_ERR_ARG;
  bool ok = true;
  for (dirac_ptc* n : c->ptcs) ptc_release(n);
  c->ptcs.clear();
  c->ptc_attached = nullptr;
  auto fr = [&](void* p) { if (p && cudaFree(p) != cudaSuccess) ok = false; };
  for (int q = 0; q < 3; ++q)
    for (char* p : {c->gauge[q], c->fat[q], c->clover[q], c->clover_inv[q], c->tmp[q], c->tmp2[q]}) fr(p);
  for (int i = 0; i < 48; ++i) fr(c->work[i]);
  fr(c->staging);
  fr(c->dscal);
  if (c->hmirror && cudaFreeHost(c->hmirror) != cudaSuccess) ok = false;
  if (c->solve_stream && cudaStreamDestroy(c->solve_stream) != cudaSuccess) ok = false;
  if (c->solve_event && cudaEventDestroy(c->solve_event) != cudaSuccess) ok = false;
  blas_destroy(c->blas);
  delete c;
  cudaGetLastError();  // leave no pending error behind for later contexts
  return ok ? DIRAC_OK : DIRAC_ERR_CUDA;
}

const char* dirac_last_error(const dirac_ctx* c) { return c ? c->err.c_str() : "null context"; }

size_t dirac_field_bytes(const dirac_ctx* c, dirac_prec prec, dirac_parity parity) {
  if (!c || !valid_prec(prec)) return 0;
  return (parity == DIRAC_PARITY_FULL ? 2 : 1) * spinor_half_bytes(prec, c->nr, c->Vh);
}

int dirac_load_gauge(dirac_ctx* c, const double* links, int which, int on_device, void* stream) {
  if (!c || !links || which < 0 || which > 2) return set_err(c, DIRAC_ERR_ARG, "bad load_gauge arguments");
  const bool wil = c->p.kind == DIRAC_WILSON_CLOVER;
  if ((wil && which != 0) || (!wil && which == 0))
    return set_err(c, DIRAC_ERR_ARG, "link field does not match the operator kind");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nat = (size_t)c->V * 72 * sizeof(double);
  const double* src = links;
  char* staging = nullptr;
  int rc;
  if (!on_device) {
    if ((rc = dalloc(c, &staging, nat))) return rc;
    cudaMemcpyAsync(staging, links, nat, cudaMemcpyHostToDevice, st);
    src = (const double*)staging;
  }
  for (int q = 0; q < 3; ++q) {
    if (!(c->mask & (1u << q))) continue;
    int recon = which == 1 ? 18 : c->p.recon[q];
    char** dst = which == 1 ? &c->fat[q] : &c->gauge[q];
    if ((rc = dalloc(c, dst, link_bytes(q, recon, c->Vh)))) break;
    launch_pack_links(q, recon, *dst, src, c->g, st);
    if ((rc = cuda_check(c, "pack links"))) break;
  }
  if (!rc && which == 0) {
    const bool inv = c->p.csw != 0.0;
    for (int q = 0; q < 3 && !rc; ++q)
      if (c->mask & (1u << q)) {
        rc = dalloc(c, &c->clover[q], 2 * clover_parity_bytes(q, c->Vh));
        if (!rc && inv) rc = dalloc(c, &c->clover_inv[q], 2 * clover_parity_bytes(q, c->Vh));
      }
    if (!rc) {
      launch_build_clover(src, c->g, c->p.kappa, c->p.csw, c->clover, inv ? c->clover_inv : nullptr, c->mask, st);
      rc = cuda_check(c, "build clover");
    }
  }
  if (staging) {
    cudaStreamSynchronize(st);
    cudaFree(staging);
  }
  if (rc) return rc;
  if (which == 0) c->have_gauge = true;
  if (which == 1) c->have_fat = true;
  if (which == 2) c->have_long = true;
  return cuda_check(c, "load gauge");
}

static int spinor_xfer(dirac_ctx* c, bool import, void* dev, dirac_prec prec, dirac_parity parity,
                       double* nat_ptr, int nat_on_device, cudaStream_t st) {
  if (!c || !dev || !nat_ptr || !valid_prec(prec) || parity < -1 || parity > 1)
    return set_err(c, DIRAC_ERR_ARG, "bad spinor transfer arguments");
  const size_t nat = (size_t)c->V * c->nr * sizeof(double);
  double* d = nat_ptr;
  char* staging = nullptr;
  int rc;
  // Page-locked host memory (and, on systems where the GPU shares the host's page
  // tables, any host memory) is read and written in place over the host link by
  // coalesced conversion kernels (FP64 / FP32 storage): no staging copy, one pass.
  bool direct = false;
  if (!nat_on_device && (int)prec != P16) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, nat_ptr) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
      d = (double*)pa.devicePointer;
      direct = true;
    } else {
      cudaGetLastError();
      int dev = 0, pageable = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
      direct = pageable != 0;
    }
  }
  if (!nat_on_device && !direct) {
    if (c->staging_bytes < nat) {
      if (c->staging) cudaFree(c->staging);
      c->staging = nullptr;
      c->staging_bytes = 0;
      if ((rc = dalloc(c, &c->staging, nat))) return rc;
      c->staging_bytes = nat;
    }
    staging = c->staging;
    d = (double*)staging;
    // an export of one parity copies the host array in first so the other parity's
    // sites come back unchanged
    if (import || parity != DIRAC_PARITY_FULL) cudaMemcpyAsync(d, nat_ptr, nat, cudaMemcpyHostToDevice, st);
  }
  if (direct) launch_host_spinor(import, prec, c->nr, (char*)dev, parity, d, c->g, st);
  else if (import) launch_import_spinor(prec, c->nr, (char*)dev, parity, d, c->g, st);
  else launch_export_spinor(prec, c->nr, d, parity, (const char*)dev, c->g, st);
  rc = cuda_check(c, import ? "import spinor" : "export spinor");
  if (direct) {
    cudaStreamSynchronize(st);  // the host buffer is read / written on return
    if (!rc) rc = cuda_check(c, "spinor host access");
  }
  if (staging) {
    if (!import && !rc) cudaMemcpyAsync(nat_ptr, d, nat, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);  // the host buffer is free for reuse on return
    if (!rc) rc = cuda_check(c, "spinor staging copy");
  }
  return rc;
}

int dirac_import_spinor(dirac_ctx* c, void* dst, dirac_prec prec, dirac_parity parity,
                        const double* src, int src_on_device, void* stream) {
  return spinor_xfer(c, true, dst, prec, parity, (double*)src, src_on_device, (cudaStream_t)stream);
}

int dirac_export_spinor(dirac_ctx* c, double* dst, int dst_on_device, const void* src,
                        dirac_prec prec, dirac_parity parity, void* stream) {
  return spinor_xfer(c, false, (void*)src, prec, parity, dst, dst_on_device, (cudaStream_t)stream);
}

static int apply_entry(dirac_ctx* c, void* out, const void* in, dirac_parity parity, dirac_prec prec,
                       int which, void* stream) {
  int rc = check_op(c, prec, false);
  if (rc) return rc;
  if (!out || !in || out == in) return set_err(c, DIRAC_ERR_ARG, "null or aliased fields");
  if (parity < -1 || parity > 1) return set_err(c, DIRAC_ERR_ARG, "bad parity");
  return apply_op(c, (char*)out, (const char*)in, parity, prec, which, (cudaStream_t)stream);
}

int dirac_apply(dirac_ctx* c, void* out, const void* in, dirac_parity parity, dirac_prec prec, void* stream) {
  return apply_entry(c, out, in, parity, prec, 0, stream);
}
int dirac_apply_dagger(dirac_ctx* c, void* out, const void* in, dirac_parity parity, dirac_prec prec,
                       void* stream) {
  return apply_entry(c, out, in, parity, prec, 1, stream);
}
int dirac_apply_ds(dirac_ctx* c, void* out, const void* in, int dagger, void* stream) {
  int rc = check_op(c, P64, false);
  if (rc) return rc;
  if (!out || !in || out == in) return set_err(c, DIRAC_ERR_ARG, "bad field pointers");
  return wilson_M_ds(c, (char*)out, (const char*)in, dagger != 0, (cudaStream_t)stream);
}

int dirac_set_ds_residual(dirac_ctx* c, int on) {
  if (!c) return DIRAC_ERR_ARG;
  c->ds_residual = on != 0;
  return DIRAC_OK;
}

int dirac_apply_normal(dirac_ctx* c, void* out, const void* in, dirac_parity parity, dirac_prec prec,
                       void* stream) {
  return apply_entry(c, out, in, parity, prec, 2, stream);
}

int dirac_apply_eo(dirac_ctx* c, void* out, const void* in, dirac_prec prec, int dagger, void* stream) {
  int rc = check_op(c, prec, false);
  if (rc) return rc;
  if (c->p.kind != DIRAC_WILSON_CLOVER)
    return set_err(c, DIRAC_ERR_UNSUPPORTED, "the even-odd operator is defined for Wilson-clover");
  if (!out || !in || out == in) return set_err(c, DIRAC_ERR_ARG, "null or aliased fields");
  return apply_op(c, (char*)out, (const char*)in, 0, prec, dagger ? 4 : 3, (cudaStream_t)stream);
}

int schwarz_precondition(dirac_ctx* c, void* out, const void* in, dirac_prec prec, void* stream) {
  int rc = check_op(c, prec, false);
  if (rc) return rc;
  if (c->p.kind != DIRAC_WILSON_CLOVER)
    return set_err(c, DIRAC_ERR_UNSUPPORTED, "Schwarz preconditioner is defined for Wilson-clover");
  if (!out || !in || out == in) return set_err(c, DIRAC_ERR_ARG, "null or aliased fields");
  return schwarz_apply(c, (char*)out, (const char*)in, prec, (cudaStream_t)stream);
}

static int blas_rc(dirac_ctx* c, int rc) {
  if (rc) c->err = blas_error(c->blas);
  return rc;
}

int dirac_norm2(dirac_ctx* c, const void* x, dirac_prec prec, dirac_parity parity, double* result,
                void* stream) {
  if (!c || !x || !result || !valid_prec(prec)) return set_err(c, DIRAC_ERR_ARG, "bad norm2 arguments");
  return blas_rc(c, blas_norm2(c->blas, field_ref(c, x, prec, parity), result, (cudaStream_t)stream));
}

int dirac_cdot(dirac_ctx* c, const void* x, const void* y, dirac_prec prec, dirac_parity parity,
               double result[2], void* stream) {
  if (!c || !x || !y || !result || !valid_prec(prec)) return set_err(c, DIRAC_ERR_ARG, "bad cdot arguments");
  return blas_rc(c, blas_cdot(c->blas, field_ref(c, x, prec, parity), field_ref(c, y, prec, parity), result,
                              (cudaStream_t)stream));
}

int dirac_caxpy_norm(dirac_ctx* c, double ar, double ai, const void* x, void* y, dirac_prec prec,
                     dirac_parity parity, double* result, void* stream) {
  if (!c || !x || !y || !result || x == y || !valid_prec(prec))
    return set_err(c, DIRAC_ERR_ARG, "bad caxpy_norm arguments");
  return blas_rc(c, blas_caxpy_norm(c->blas, cval(ar, ai), field_ref(c, x, prec, parity),
                                    field_ref(c, y, prec, parity), result, (cudaStream_t)stream));
}

int dirac_convert(dirac_ctx* c, void* dst, dirac_prec dprec, const void* src, dirac_prec sprec,
                  dirac_parity parity, void* stream) {
  if (!c || !dst || !src || !valid_prec(dprec) || !valid_prec(sprec) || dst == src)
    return set_err(c, DIRAC_ERR_ARG, "bad convert arguments");
  return blas_rc(c, blas_copy(c->blas, field_ref(c, dst, dprec, parity), field_ref(c, src, sprec, parity),
                              (cudaStream_t)stream));
}

}  // extern "C"
