// Improved staggered (asqtad) stencil (Eq. 3), one thread per output site of one
// parity. Read as the anti-Hermitian staggered operator with the phases
// eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) applied in the kernel to phase-free links:
//
//   D psi(x) = sum_mu eta_mu(x) [ F_mu(x) psi(x+mu)  - F_mu(x-mu)^dagger  psi(x-mu)
//                                + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^dagger psi(x-3mu) ]
//
// with F the fat links (18 reals, not unitary) and L the long links (18/12/8 reals).
// All hops are odd, so D maps one parity to the other. The kernel computes
//   out_p = a * x_p + b * D_{p,1-p} in_{1-p}
// which covers the hopping block (a = 0), M = m - D/2 per parity and the second half
// of the even-site normal operator m^2 - 1/4 D_eo D_oe.
#include "field.cuh"
#include "internal.h"

namespace dirac {

struct StagArg {
  char* out;             // half-field of parity out_parity
  const char* in;        // half-field of parity 1 - out_parity
  const char* x;         // half-field of parity out_parity for the a*x term, or null
  const char* fat;
  const char* lng;
  Geom g;
  int out_parity;
  double a, b;
};

__device__ __forceinline__ int stag_shift(int v, int n, int L, int& wraps) {
  v += n;
  wraps = 0;
  while (v >= L) { v -= L; ++wraps; }
  while (v < 0) { v += L; ++wraps; }
  return v;
}

// A neighbour spinor and the factor its link product is multiplied by: with FP16 storage
// the per-site norm is left out of the 6 values and folded into that factor.
template <int PREC, typename T>
__device__ __forceinline__ T load_stag_spinor(const char* src, int Vh, int cb, T v[6]) {
  if constexpr (PREC == P16) {
    return SpinorIO<P16, 6>::load_raw(src, Vh, cb, v);
  } else {
    SpinorIO<PREC, 6>::load(src, Vh, cb, v);
    return (T)1;
  }
}

template <int PREC, int RL>
__global__ void __launch_bounds__(128) staggered_kernel(const StagArg a) {
  using T = typename Real<PREC>::T;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= Vh) return;
  const int par = a.out_parity;
  int x[4];
  cb_coords(g, cb, par, x);
  C<T> acc[3] = {{0, 0}, {0, 0}, {0, 0}};
  int esum = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const T eta = (esum & 1) ? (T)-1 : (T)1;
    esum += x[mu];
#pragma unroll
    for (int hop = 0; hop < 2; ++hop) {
      const int n = hop == 0 ? 1 : 3;
      const char* links = hop == 0 ? a.fat : a.lng;
      // forward: link at x, neighbour x + n mu
      {
        int y[4] = {x[0], x[1], x[2], x[3]}, w;
        y[mu] = stag_shift(x[mu], n, g.L[mu], w);
        T bc = (mu == 3 && g.apbc && (w & 1)) ? (T)-1 : (T)1;
        T v[6];
        const T nrm = load_stag_spinor<PREC, T>(a.in, Vh, cb_index(g, y), v);
        C<T> h[3] = {{v[0], v[1]}, {v[2], v[3]}, {v[4], v[5]}}, r[3];
        Link<T> U;
        if (hop == 0) LinkIO<PREC, 18>::load(links, Vh, mu, par, cb, U);
        else LinkIO<PREC, RL>::load(links, Vh, mu, par, cb, U);
        su3_mv(U, h, r);
        const T f = eta * bc * nrm;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = acc[c] + f * r[c];
      }
      // backward: link at x - n mu, neighbour x - n mu
      {
        int y[4] = {x[0], x[1], x[2], x[3]}, w;
        y[mu] = stag_shift(x[mu], -n, g.L[mu], w);
        T bc = (mu == 3 && g.apbc && (w & 1)) ? (T)-1 : (T)1;
        int ycb = cb_index(g, y);
        T v[6];
        const T nrm = load_stag_spinor<PREC, T>(a.in, Vh, ycb, v);
        C<T> h[3] = {{v[0], v[1]}, {v[2], v[3]}, {v[4], v[5]}}, r[3];
        Link<T> U;
        if (hop == 0) LinkIO<PREC, 18>::load(links, Vh, mu, 1 - par, ycb, U);
        else LinkIO<PREC, RL>::load(links, Vh, mu, 1 - par, ycb, U);
        su3_mv_dag(U, h, r);
        const T f = -eta * bc * nrm;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = acc[c] + f * r[c];
      }
    }
  }
  T out[6];
  const T bb = (T)a.b;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    out[2 * c] = bb * acc[c].r;
    out[2 * c + 1] = bb * acc[c].i;
  }
  if (a.x) {
    T s[6];
    SpinorIO<PREC, 6>::load(a.x, Vh, cb, s);
    const T aa = (T)a.a;
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k] = fma(aa, s[k], out[k]);
  }
  SpinorIO<PREC, 6>::store(a.out, Vh, cb, out);
}

template <int PREC>
static void launch_stag_prec(int recon, const StagArg& a, cudaStream_t st) {
  dim3 block(128), grid((a.g.Vh + 127) / 128);
  if (recon == 18) staggered_kernel<PREC, 18><<<grid, block, 0, st>>>(a);
  else if (recon == 12) staggered_kernel<PREC, 12><<<grid, block, 0, st>>>(a);
  else staggered_kernel<PREC, 8><<<grid, block, 0, st>>>(a);
}

void launch_staggered(int prec, int recon, char* out, const char* in, const char* x,
                      const char* fat, const char* lng, const Geom& g, int out_parity, double a,
                      double b, cudaStream_t st) {
  StagArg arg{out, in, x, fat, lng, g, out_parity, a, b};
  if (prec == P64) launch_stag_prec<P64>(recon, arg, st);
  else if (prec == P32) launch_stag_prec<P32>(recon, arg, st);
  else launch_stag_prec<P16>(recon, arg, st);
}

}  // namespace dirac
