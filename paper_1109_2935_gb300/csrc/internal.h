// Host-side internals of libdirac: the context behind the opaque dirac_ctx handle,
// field descriptors and the kernel launchers shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

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
void launch_build_clover(const double* links, const Geom& g, double kappa, double csw,
                         char* const dst[3], unsigned prec_mask, cudaStream_t st);

// Schwarz block-MR preconditioner
int launch_schwarz(int prec, int recon, char* out, const char* in, const char* gauge,
                   const char* clover, const Geom& g, const int block[4], int mr_steps,
                   double kappa, cudaStream_t st);

// ---------------------------------------------------------------- BLAS (blas.cu)
struct Blas;  // reduction scratch + pinned result slots
Blas* blas_create();
void blas_destroy(Blas*);
// All scalars are host values; reductions synchronise the stream and return on host.
int blas_copy(Blas*, const FieldRef& dst, const FieldRef& src, cudaStream_t st);
int blas_zero(Blas*, const FieldRef& x, cudaStream_t st);
// y = a x + b y (complex a, b)
int blas_axpby(Blas*, double ar, double ai, const FieldRef& x, double br, double bi,
               const FieldRef& y, cudaStream_t st);
// z = x + a y  (z may alias x or y)
int blas_xpay_to(Blas*, const FieldRef& x, double ar, double ai, const FieldRef& y,
                 const FieldRef& z, cudaStream_t st);
// y += a x + b z
int blas_axpbz_add(Blas*, double ar, double ai, const FieldRef& x, double br, double bi,
                   const FieldRef& z, const FieldRef& y, cudaStream_t st);
int blas_norm2(Blas*, const FieldRef& x, double* out, cudaStream_t st);
int blas_cdot(Blas*, const FieldRef& x, const FieldRef& y, double out[2], cudaStream_t st);
// out = {Re (x,y), Im (x,y), ||x||^2}
int blas_cdot_norm(Blas*, const FieldRef& x, const FieldRef& y, double out[3], cudaStream_t st);
// y += a x; out = ||y||^2
int blas_caxpy_norm(Blas*, double ar, double ai, const FieldRef& x, const FieldRef& y,
                    double* out, cudaStream_t st);
// y += a x; out = {||y||^2, Re (w,y), Im (w,y)}
int blas_caxpy_norm_dot(Blas*, double ar, double ai, const FieldRef& x, const FieldRef& y,
                        const FieldRef& w, double out[3], cudaStream_t st);
// x *= s (real); out = (x, y) after scaling
int blas_scale_cdot(Blas*, double s, const FieldRef& x, const FieldRef& y, double out[2],
                    cudaStream_t st);
// y = b - y ; out = ||y||^2   (residual r = b - Ax with Ax held in y)
int blas_xmy_norm(Blas*, const FieldRef& b, const FieldRef& y, double* out, cudaStream_t st);
// y += sum_i c_i x_i (n <= 32 vectors of one precision), complex coefficients
int blas_multi_caxpy(Blas*, int n, const double* c_re, const double* c_im, const FieldRef* xs,
                     const FieldRef& y, cudaStream_t st);
const char* blas_error(Blas*);

// ---------------------------------------------------------------- api.cu helpers
int set_err(dirac_ctx* c, int code, const std::string& msg);
int cuda_check(dirac_ctx* c, const char* what);
FieldRef field_ref(const dirac_ctx* c, const void* p, int prec, int parity);
int check_op(dirac_ctx* c, int prec, bool need_schwarz);
int ensure_tmp(dirac_ctx* c, int prec);
// which: 0 = M, 1 = M^dagger, 2 = M^dagger M; parity FULL(-1) / EVEN / ODD
int apply_op(dirac_ctx* c, char* out, const char* in, int parity, int prec, int which, cudaStream_t st);
int schwarz_apply(dirac_ctx* c, char* out, const char* in, int prec, cudaStream_t st);

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
  bool have_gauge = false, have_fat = false, have_long = false;
  // scratch spinors for composite operators, per precision (full fields)
  char* tmp[3] = {nullptr, nullptr, nullptr};
  char* tmp2[3] = {nullptr, nullptr, nullptr};
  dirac::Blas* blas = nullptr;
  // solver work fields (solvers.cu), grown on demand and kept until destroy
  char* work[48] = {};
  size_t work_bytes[48] = {};
  // device staging for natural-layout spinors passed from host memory
  char* staging = nullptr;
  size_t staging_bytes = 0;
  std::string err;
};
