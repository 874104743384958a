// Host-side internals of libdirac: the context behind the opaque dirac_ctx handle,
// field descriptors and the kernel launchers shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dirac.h"
#include "field.cuh"

struct dirac_ctx;

namespace dirac {

// ---------------------------------------------------------------- field geometry
inline size_t spinor_half_bytes(int prec, int nr, int64_t Vh) {
  if (prec == P64) return (size_t)nr * 8 * Vh;
  if (prec == P32) return (size_t)nr * 4 * Vh;
  return (size_t)nr * 2 * Vh + (size_t)4 * Vh;
}
inline size_t link_bytes(int prec, int recon, int64_t Vh) {
  int w = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
  return (size_t)8 * recon * w * Vh;  // 4 directions x 2 parities
}
inline size_t clover_parity_bytes(int prec, int64_t Vh) {
  return prec == P64 ? (size_t)576 * Vh : (prec == P32 ? (size_t)288 * Vh : (size_t)148 * Vh);
}

// A spinor field view used by the BLAS kernels: `npar` consecutive half-fields
// starting at parity `par0`.
struct FieldRef {
  char* p;
  int prec;
  int nr;      // reals per site: 24 Wilson, 6 staggered
  int Vh;
  int npar;    // 1 (half-field) or 2 (full field)
  size_t hb;   // bytes per half-field
};

// ---------------------------------------------------------------- launchers
struct WilsonArg;
void launch_wilson_p64(int recon, bool fullm, const WilsonArg& a, cudaStream_t st);
void launch_wilson_p32(int recon, bool fullm, const WilsonArg& a, cudaStream_t st);
void launch_wilson_p16(int recon, bool fullm, const WilsonArg& a, cudaStream_t st);

void launch_staggered(int prec, int recon, char* out, const char* in, const char* x,
                      const char* fat, const char* lng, const Geom& g, int out_parity, double a,
                      double b, cudaStream_t st);

// natural FP64 <-> device layout
void launch_import_spinor(int prec, int nr, char* dst, int parity, const double* src, const Geom& g,
                          cudaStream_t st);
void launch_export_spinor(int prec, int nr, double* dst, int parity, const char* src, const Geom& g,
                          cudaStream_t st);
void launch_pack_links(int prec, int recon, char* dst, const double* src, const Geom& g,
                       cudaStream_t st);
// natural FP64 array in host memory the GPU can access <-> device layout, coalesced over
// the host link (FP64 / FP32 storage; returns false for FP16, which uses a staging copy)
bool launch_host_spinor(bool import, int prec, int nr, char* dev, int parity, double* nat, const Geom& g,
                        cudaStream_t st);
// Ahat = 1 + 2 kappa A into dst[p]; Ahat^-1 into inv[p] when inv is not null
void launch_build_clover(const double* links, const Geom& g, double kappa, double csw,
                         char* const dst[3], char* const inv[3], unsigned prec_mask, cudaStream_t st);

// Schwarz block-MR preconditioner
int launch_schwarz(int prec, int recon, char* out, const char* in, const char* gauge,
                   const char* clover, const Geom& g, const int block[4], int mr_steps,
                   double kappa, cudaStream_t st);

// ---------------------------------------------------------------- BLAS (blas.cu)
// A complex coefficient: the host value (r, i), or s * (p[0], p[1]) read on the device
// when p is set (written there by an earlier reduction or a solver's scalar kernel).
struct Cf {
  double r = 0, i = 0;
  const double* p = nullptr;
  double s = 1;
};
inline Cf cval(double r, double i = 0) { Cf c; c.r = r; c.i = i; return c; }
inline Cf cptr(const double* p, double s = 1) { Cf c; c.p = p; c.s = s; return c; }

struct Blas;  // reduction scratch + pinned result slots
Blas* blas_create();
void blas_destroy(Blas*);
// Reductions return their result on the host after a stream synchronisation, or, when
// `dres` (3 doubles of device memory) is given, leave it there without synchronising.
int blas_copy(Blas*, const FieldRef& dst, const FieldRef& src, cudaStream_t st);
int blas_zero(Blas*, const FieldRef& x, cudaStream_t st);
// y = a x + b y
int blas_axpby(Blas*, Cf a, const FieldRef& x, Cf b, const FieldRef& y, cudaStream_t st);
// p = r + b p + c v
int blas_pupdate(Blas*, const FieldRef& r, Cf b, Cf c, const FieldRef& v, const FieldRef& p, cudaStream_t st);
int blas_norm2(Blas*, const FieldRef& x, double* out, cudaStream_t st, double* dres = nullptr);
int blas_cdot(Blas*, const FieldRef& x, const FieldRef& y, double out[2], cudaStream_t st,
              double* dres = nullptr);
// out = {Re (x,y), Im (x,y), ||x||^2}
int blas_cdot_norm(Blas*, const FieldRef& x, const FieldRef& y, double out[3], cudaStream_t st,
                   double* dres = nullptr);
// y += a x; out = ||y||^2
int blas_caxpy_norm(Blas*, Cf a, const FieldRef& x, const FieldRef& y, double* out, cudaStream_t st,
                    double* dres = nullptr);
// y += a x; out = {||y||^2, Re (w,y), Im (w,y)}
int blas_caxpy_norm_dot(Blas*, Cf a, const FieldRef& x, const FieldRef& y, const FieldRef& w,
                        double out[3], cudaStream_t st, double* dres = nullptr);
// xs += a p + b s; s += c t; out = {||s||^2, Re (w,s), Im (w,s)}
int blas_bicg_xr(Blas*, Cf a, const FieldRef& p, Cf b, const FieldRef& s, Cf c, const FieldRef& t,
                 const FieldRef& xs, const FieldRef& w, double out[3], cudaStream_t st,
                 double* dres = nullptr);
// xs += a p; r += c Ap; out = ||r||^2
int blas_cg_update(Blas*, Cf a, const FieldRef& p, Cf c, const FieldRef& Ap, const FieldRef& xs,
                   const FieldRef& r, double* out, cudaStream_t st, double* dres = nullptr);
// x *= Re s; out = (x, y) after scaling
int blas_scale_cdot(Blas*, Cf s, const FieldRef& x, const FieldRef& y, double out[2], cudaStream_t st,
                    double* dres = nullptr);
// y = b - y ; out = ||y||^2   (residual r = b - Ax with Ax held in y)
int blas_xmy_norm(Blas*, const FieldRef& b, const FieldRef& y, double* out, cudaStream_t st,
                  double* dres = nullptr);
// y += sum_i c_i x_i
int blas_multi_caxpy(Blas*, int n, const Cf* c, const FieldRef* xs, const FieldRef& y, cudaStream_t st);
// multi-shift CG: x_j += a_j p_j; p_j = z_j r + b_j p_j for the active j (coef on device,
// 4 doubles per shift: a, z, b, active), n <= 16
int blas_multishift_update(Blas*, int n, const FieldRef* xs, const FieldRef* ps, const FieldRef& r,
                           const double* coef, cudaStream_t st);
const char* blas_error(Blas*);

// ---------------------------------------------------------------- api.cu helpers
int set_err(dirac_ctx* c, int code, const std::string& msg);
int cuda_check(dirac_ctx* c, const char* what);
FieldRef field_ref(const dirac_ctx* c, const void* p, int prec, int parity);
int check_op(dirac_ctx* c, int prec, bool need_schwarz);
int ensure_tmp(dirac_ctx* c, int prec);
// which: 0 = M, 1 = M^dagger, 2 = M^dagger M (+ shift), 3 / 4 = even-odd Schur operator /
// its adjoint (Wilson-clover, parity EVEN); parity FULL(-1) / EVEN / ODD
int apply_op(dirac_ctx* c, char* out, const char* in, int parity, int prec, int which, cudaStream_t st,
             double shift = 0.0);
int schwarz_apply(dirac_ctx* c, char* out, const char* in, int prec, cudaStream_t st);
// the Wilson-clover M (dag: M^dagger) on FP64 full fields in double-single arithmetic
// (wilson_ds.cu); DIRAC_ERR_UNSUPPORTED unless Wilson-clover with 18-real FP64 links
int wilson_M_ds(dirac_ctx* c, char* out, const char* in, bool dag, cudaStream_t st);
bool ds_available(const dirac_ctx* c);
// even-odd form (Wilson-clover): bhat_e = b_e + kappa D_eo Ahat_oo^-1 b_o and
// x_o = Ahat_oo^-1 (b_o + kappa D_oe x_e); which = 3 / 4 in apply_op is the Schur
// operator / its adjoint on even half-fields
int schur_source(dirac_ctx* c, char* bhat, const char* b, int prec, cudaStream_t st);
int schur_reconstruct(dirac_ctx* c, char* x, const char* b, int prec, cudaStream_t st);

// ---------------------------------------------------------------- batched operator (batch.cu)
// dirac_batch_create with a tuning level: 2 = every tile shape and the tensor-core kernel
// timed (the public call), 1 = the default shape timed against the tensor-core kernel,
// 0 = no timing (default shape; the tensor-core kernel where it exists), -1 = no timing and
// the CUDA-core kernel only (default shape; for plans that will be masked)
// (ds: FP64 fields, 18-real links, arithmetic in double-single as dirac_apply_ds)
int batch_create(dirac_ctx* const* ctxs, int nlat, void* const* out, const void* const* in, const int* nrhs,
                 int prec, cudaStream_t stream, dirac_batch** plan, int tune, bool ds = false);
// skip the right-hand sides whose mask[rhs * stride] is 0 (read at every launch); a masked
// plan runs the CUDA-core kernel
int batch_set_mask(dirac_batch* b, const double* mask, int stride, cudaStream_t st);

// ---------------------------------------------------------------- PTC network (ptc.cu)
// out = K in on FP32 full fields; flops of one application; free a network
int ptc_apply_internal(dirac_ptc* n, char* out, const char* in, cudaStream_t st);
double ptc_flops_per_apply(const dirac_ptc* n);
void ptc_release(dirac_ptc* n);
// tensor-core inference layer (ptc_tc.cu): BF16 weight image of a layer, its size, and
// one layer out[c] = sum W T in[c'] on FP32 full fields
size_t ptc_tc_image_bytes(int cin, int cout);
void ptc_tc_pack(int cin, int cout, const float2* w, void* img, cudaStream_t st);
int ptc_tc_layer(int cin, int cout, int recon, const char* const* in, char* const* out, const char* gauge,
                 const void* img, const Geom& g, int* err, uint64_t wait_ns, int stall, cudaStream_t st);

}  // namespace dirac

// ---------------------------------------------------------------- the context
struct dirac_ctx {
  dirac_params p;
  dirac::Geom g;
  int64_t V, Vh;
  int nr;                      // reals per site
  unsigned mask;               // precisions kept
  // library-owned operator storage per precision
  char* gauge[3] = {nullptr, nullptr, nullptr};   // Wilson U or asqtad long links
  char* fat[3] = {nullptr, nullptr, nullptr};     // asqtad fat links
  char* clover[3] = {nullptr, nullptr, nullptr};  // Wilson-clover Ahat
  char* clover_inv[3] = {nullptr, nullptr, nullptr};  // Ahat^-1 (c_sw != 0)
  bool have_gauge = false, have_fat = false, have_long = false;
  // scratch spinors for composite operators, per precision (full fields)
  char* tmp[3] = {nullptr, nullptr, nullptr};
  char* tmp2[3] = {nullptr, nullptr, nullptr};
  dirac::Blas* blas = nullptr;
  // solver work fields (solvers.cu), grown on demand and kept until destroy
  char* work[48] = {};
  size_t work_bytes[48] = {};
  // solver scalars: device slots, a mapped host mirror of per-iteration residuals
  double* dscal = nullptr;
  double* hmirror = nullptr;
  double* dmirror = nullptr;
  // device staging for natural-layout spinors passed from host memory
  char* staging = nullptr;
  size_t staging_bytes = 0;
  // PTC networks created on this context (freed by dirac_destroy) and the one
  // DIRAC_SOLVER_GCR_PTC uses
  std::vector<dirac_ptc*> ptcs;
  dirac_ptc* ptc_attached = nullptr;
  int ptc_force = 0;
  // solve(): private stream (graph capture needs a non-default stream) and the event that
  // orders it after the caller's stream
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t solve_event = nullptr;
  // solve(): FP64 true residuals of restarts / reliable updates in double-single arithmetic
  // (the final check and any convergence decision are confirmed in FP64). Off by default:
  // measured slower than the FP64 operator on this part (dirac_set_ds_residual)
  int ds_residual = 0;
  std::string err;
};
