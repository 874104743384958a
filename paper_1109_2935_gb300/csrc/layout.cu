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

// Host-resident natural arrays (FP64 / FP32 storage): one thread per 16-byte piece (two
// reals) of the natural array, so every warp reads or writes 512 contiguous bytes over
// the host link; the device side of each piece is a whole chunk (FP64, or FP32
// staggered) or half a chunk (FP32 Wilson).
template <int PREC, int NR>
__device__ __forceinline__ void piece_place(const Geom& g, int64_t i, int& par, int& cb, int& chunk, int& half) {
  constexpr int NP = NR / 2;
  const int64_t s = i / NP;
  const int j = (int)(i - s * NP);
  int r = (int)s, x[4];
  x[0] = r % g.L[0]; r /= g.L[0];
  x[1] = r % g.L[1]; r /= g.L[1];
  x[2] = r % g.L[2];
  x[3] = r / g.L[2];
  par = (x[0] + x[1] + x[2] + x[3]) & 1;
  cb = (int)(s >> 1);
  if (PREC == P32 && NR == 24) { chunk = j >> 1; half = j & 1; }
  else { chunk = j; half = 0; }
}

// Each thread moves HP consecutive pieces, its host loads issued together so that more
// requests are in flight over the long-latency host link.
constexpr int HP = 4;

template <int PREC, int NR>
__device__ __forceinline__ void piece_store(char* dst, int par0, const Geom& g, int64_t i, double2 v) {
  int par, cb, chunk, half;
  piece_place<PREC, NR>(g, i, par, cb, chunk, half);
  char* base = dst + (size_t)(par - par0) * SpinorIO<PREC, NR>::half_bytes(g.Vh);
  if constexpr (PREC == P64) {
    reinterpret_cast<double2*>(base)[(size_t)chunk * g.Vh + cb] = v;
  } else if constexpr (NR == 24) {
    reinterpret_cast<float2*>(base + ((size_t)chunk * g.Vh + cb) * 16)[half] = make_float2((float)v.x, (float)v.y);
  } else {
    reinterpret_cast<float2*>(base)[(size_t)chunk * g.Vh + cb] = make_float2((float)v.x, (float)v.y);
  }
}

template <int PREC, int NR>
__device__ __forceinline__ double2 piece_load(const char* src, int par0, const Geom& g, int64_t i) {
  int par, cb, chunk, half;
  piece_place<PREC, NR>(g, i, par, cb, chunk, half);
  const char* base = src + (size_t)(par - par0) * SpinorIO<PREC, NR>::half_bytes(g.Vh);
  if constexpr (PREC == P64) {
    return reinterpret_cast<const double2*>(base)[(size_t)chunk * g.Vh + cb];
  } else if constexpr (NR == 24) {
    const float2 f = reinterpret_cast<const float2*>(base + ((size_t)chunk * g.Vh + cb) * 16)[half];
    return make_double2(f.x, f.y);
  } else {
    const float2 f = reinterpret_cast<const float2*>(base)[(size_t)chunk * g.Vh + cb];
    return make_double2(f.x, f.y);
  }
}

template <int PREC, int NR>
__device__ __forceinline__ bool piece_in(const Geom& g, int64_t i, int par0, int npar) {
  int par, cb, chunk, half;
  piece_place<PREC, NR>(g, i, par, cb, chunk, half);
  return par >= par0 && par < par0 + npar;
}

// piece i of thread t in block b: i = (b * HP + h) * blockDim + t, so every load
// instruction of a warp still covers 512 contiguous bytes
template <int PREC, int NR>
__global__ void import_host_kernel(char* dst, int par0, int npar, const double2* src, Geom g) {
  const int64_t n = (int64_t)g.Vh * NR;  // 2 Vh sites x NR / 2 pieces
  const int64_t i0 = (int64_t)blockIdx.x * HP * blockDim.x + threadIdx.x;
  double2 v[HP];
  bool use[HP];
#pragma unroll
  for (int h = 0; h < HP; ++h) {
    const int64_t i = i0 + (int64_t)h * blockDim.x;
    use[h] = i < n && piece_in<PREC, NR>(g, i, par0, npar);
    if (use[h]) v[h] = src[i];
  }
#pragma unroll
  for (int h = 0; h < HP; ++h)
    if (use[h]) piece_store<PREC, NR>(dst, par0, g, i0 + (int64_t)h * blockDim.x, v[h]);
}

template <int PREC, int NR>
__global__ void export_host_kernel(double2* dst, int par0, int npar, const char* src, Geom g) {
  const int64_t n = (int64_t)g.Vh * NR;
  const int64_t i0 = (int64_t)blockIdx.x * HP * blockDim.x + threadIdx.x;
  double2 v[HP];
  bool use[HP];
#pragma unroll
  for (int h = 0; h < HP; ++h) {
    const int64_t i = i0 + (int64_t)h * blockDim.x;
    use[h] = i < n && piece_in<PREC, NR>(g, i, par0, npar);
    if (use[h]) v[h] = piece_load<PREC, NR>(src, par0, g, i);
  }
#pragma unroll
  for (int h = 0; h < HP; ++h)
    if (use[h]) dst[i0 + (int64_t)h * blockDim.x] = v[h];
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

bool launch_host_spinor(bool import, int prec, int nr, char* dev, int parity, double* nat, const Geom& g,
                        cudaStream_t st) {
  if (prec == P16) return false;  // the per-site norm needs the whole site in one thread
  int par0 = parity < 0 ? 0 : parity, npar = parity < 0 ? 2 : 1;
  const int64_t n = (int64_t)g.Vh * nr;
  dim3 grid((unsigned)((n + 256 * HP - 1) / (256 * HP))), block(256);
  double2* h = reinterpret_cast<double2*>(nat);
  if (import) {
    if (nr == 24) {
      if (prec == P64) import_host_kernel<P64, 24><<<grid, block, 0, st>>>(dev, par0, npar, h, g);
      else import_host_kernel<P32, 24><<<grid, block, 0, st>>>(dev, par0, npar, h, g);
    } else {
      if (prec == P64) import_host_kernel<P64, 6><<<grid, block, 0, st>>>(dev, par0, npar, h, g);
      else import_host_kernel<P32, 6><<<grid, block, 0, st>>>(dev, par0, npar, h, g);
    }
  } else {
    if (nr == 24) {
      if (prec == P64) export_host_kernel<P64, 24><<<grid, block, 0, st>>>(h, par0, npar, dev, g);
      else export_host_kernel<P32, 24><<<grid, block, 0, st>>>(h, par0, npar, dev, g);
    } else {
      if (prec == P64) export_host_kernel<P64, 6><<<grid, block, 0, st>>>(h, par0, npar, dev, g);
      else export_host_kernel<P32, 6><<<grid, block, 0, st>>>(h, par0, npar, dev, g);
    }
  }
  return true;
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
