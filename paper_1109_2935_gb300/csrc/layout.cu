// Conversion between the host applications' natural FP64 layout and the device
// layout (Sec. 5: fields reordered for coalescing; Sec. 6.1: parity-split fields of
// Vh sites), including the gauge compression to 12 or 8 reals (Sec. 5 strategy (a)).
#include "internal.h"

namespace dirac {

__device__ __forceinline__ int64_t lex_index(const Geom& g, const int x[4]) {
  return (((int64_t)x[3] * g.L[2] + x[2]) * g.L[1] + x[1]) * g.L[0] + x[0];
}

template <int PREC, int NR>
__global__ void import_spinor_kernel(char* dst, int par0, int npar, const double* src, Geom g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)npar * g.Vh) return;
  int q = (int)(i / g.Vh), cb = (int)(i - (int64_t)q * g.Vh);
  int par = par0 + q;
  int x[4];
  cb_coords(g, cb, par, x);
  const double* s = src + lex_index(g, x) * NR;
  using T = typename Real<PREC>::T;
  T v[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) v[k] = (T)s[k];
  SpinorIO<PREC, NR>::store(dst + (size_t)q * SpinorIO<PREC, NR>::half_bytes(g.Vh), g.Vh, cb, v);
}

template <int PREC, int NR>
__global__ void export_spinor_kernel(double* dst, int par0, int npar, const char* src, Geom g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)npar * g.Vh) return;
  int q = (int)(i / g.Vh), cb = (int)(i - (int64_t)q * g.Vh);
  int par = par0 + q;
  int x[4];
  cb_coords(g, cb, par, x);
  using T = typename Real<PREC>::T;
  T v[NR];
  SpinorIO<PREC, NR>::load(src + (size_t)q * SpinorIO<PREC, NR>::half_bytes(g.Vh), g.Vh, cb, v);
  double* d = dst + lex_index(g, x) * NR;
#pragma unroll
  for (int k = 0; k < NR; ++k) d[k] = (double)v[k];
}

template <int PREC, int R>
__global__ void pack_links_kernel(char* dst, const double* src, Geom g) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * (int64_t)g.Vh) return;
  int par = (int)(i / g.Vh), cb = (int)(i - (int64_t)par * g.Vh);
  int x[4];
  cb_coords(g, cb, par, x);
  const double* s = src + lex_index(g, x) * 72;
  for (int mu = 0; mu < 4; ++mu) {
    double u[18];
    for (int k = 0; k < 18; ++k) u[k] = s[mu * 18 + k];
    LinkIO<PREC, R>::store(dst, g.Vh, mu, par, cb, u);
  }
}

static inline dim3 grid_for(int64_t n) { return dim3((unsigned)((n + 255) / 256)); }

// parity: -1 full, 0 even, 1 odd
void launch_import_spinor(int prec, int nr, char* dst, int parity, const double* src, const Geom& g,
                          cudaStream_t st) {
  int par0 = parity < 0 ? 0 : parity, npar = parity < 0 ? 2 : 1;
  dim3 grid = grid_for((int64_t)npar * g.Vh), block(256);
  if (nr == 24) {
    if (prec == P64) import_spinor_kernel<P64, 24><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else if (prec == P32) import_spinor_kernel<P32, 24><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else import_spinor_kernel<P16, 24><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
  } else {
    if (prec == P64) import_spinor_kernel<P64, 6><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else if (prec == P32) import_spinor_kernel<P32, 6><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else import_spinor_kernel<P16, 6><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
  }
}

void launch_export_spinor(int prec, int nr, double* dst, int parity, const char* src, const Geom& g,
                          cudaStream_t st) {
  int par0 = parity < 0 ? 0 : parity, npar = parity < 0 ? 2 : 1;
  dim3 grid = grid_for((int64_t)npar * g.Vh), block(256);
  if (nr == 24) {
    if (prec == P64) export_spinor_kernel<P64, 24><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else if (prec == P32) export_spinor_kernel<P32, 24><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else export_spinor_kernel<P16, 24><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
  } else {
    if (prec == P64) export_spinor_kernel<P64, 6><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else if (prec == P32) export_spinor_kernel<P32, 6><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
    else export_spinor_kernel<P16, 6><<<grid, block, 0, st>>>(dst, par0, npar, src, g);
  }
}

template <int PREC>
static void pack_links_prec(int recon, char* dst, const double* src, const Geom& g, cudaStream_t st) {
  dim3 grid = grid_for(2 * (int64_t)g.Vh), block(256);
  if (recon == 18) pack_links_kernel<PREC, 18><<<grid, block, 0, st>>>(dst, src, g);
  else if (recon == 12) pack_links_kernel<PREC, 12><<<grid, block, 0, st>>>(dst, src, g);
  else pack_links_kernel<PREC, 8><<<grid, block, 0, st>>>(dst, src, g);
}

void launch_pack_links(int prec, int recon, char* dst, const double* src, const Geom& g,
                       cudaStream_t st) {
  if (prec == P64) pack_links_prec<P64>(recon, dst, src, g, st);
  else if (prec == P32) pack_links_prec<P32>(recon, dst, src, g, st);
  else pack_links_prec<P16>(recon, dst, src, g, st);
}

}  // namespace dirac
