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

// ---------------------------------------------------------------- 16-bit hops
// r = U chi (dag: U^dagger chi) from stored binary16 values: a link of R = 18 reals (all
// 9 entries, one complex per word, row-major) or R = 12 (rows 0 and 1; row 2 =
// conj(row0 x row1) is rebuilt in FP32) and a binary16 colour vector (3 words). Products
// of two binary16 values are exact, so each term is one fma.rn.f32.f16 into the FP32
// accumulator; only row 2 of a 12-real link needs the vector in FP32.
template <int R>
__device__ __forceinline__ void stag_mv_h(const uint32_t* uw, const uint32_t chi[3], bool dag, C<float> r[3]) {
  constexpr int NR = R / 6;  // rows stored
  uint32_t nchi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) nchi[b] = chi[b] ^ 0x80008000u;
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = C<float>{0.f, 0.f};
  if (!dag) {
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const uint32_t u = uw[3 * a + b];
        r[a].r = fma_hh<1, 1>(u, nchi[b], fma_hh<0, 0>(u, chi[b], r[a].r));
        r[a].i = fma_hh<1, 0>(u, chi[b], fma_hh<0, 1>(u, chi[b], r[a].i));
      }
  } else {
#pragma unroll
    for (int b = 0; b < NR; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const uint32_t u = uw[3 * b + a];
        r[a].r = fma_hh<1, 1>(u, chi[b], fma_hh<0, 0>(u, chi[b], r[a].r));
        r[a].i = fma_hh<1, 0>(u, nchi[b], fma_hh<0, 1>(u, chi[b], r[a].i));
      }
  }
  if constexpr (R == 12) {
    // row 2: c_j = conj(a_p b_q - a_q b_p), p = j + 1, q = j + 2 (mod 3), a / b rows 0 / 1
    C<float> c[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int p = (j + 1) % 3, q = (j + 2) % 3;
      const uint32_t ap = uw[p], aq = uw[q], bp = uw[3 + p], bq = uw[3 + q];
      const uint32_t nap = ap ^ 0x80008000u, naq = aq ^ 0x80008000u;
      float cr = fma_hh<0, 0>(ap, bq, 0.f);
      cr = fma_hh<1, 1>(nap, bq, cr);
      cr = fma_hh<0, 0>(naq, bp, cr);
      cr = fma_hh<1, 1>(aq, bp, cr);
      float ci = fma_hh<0, 1>(ap, bq, 0.f);
      ci = fma_hh<1, 0>(ap, bq, ci);
      ci = fma_hh<0, 1>(naq, bp, ci);
      ci = fma_hh<1, 0>(naq, bp, ci);
      c[j] = C<float>{cr, -ci};
    }
    C<float> x[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&chi[b]));
      x[b] = C<float>{f.x, f.y};
    }
    if (!dag) {
#pragma unroll
      for (int b = 0; b < 3; ++b) cmac(r[2], c[b], x[b]);
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) cmacc(r[a], c[a], x[2]);
    }
  }
}

// a 16-bit colour vector (3 binary16 words) and its norm
__device__ __forceinline__ float load_stag_h(const char* src, int Vh, int cb, uint32_t chi[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) chi[k] = __ldg(reinterpret_cast<const uint32_t*>(src + ((size_t)k * Vh + cb) * 4));
  return __ldg(reinterpret_cast<const float*>(src + (size_t)12 * Vh) + cb);
}
// the stored words of a 16-bit link with R = 18 (9 words) or 12 (6 words) reals
template <int R>
__device__ __forceinline__ void load_link_h(const char* base, int Vh, int mu, int par, int cb, uint32_t uw[9]) {
  const char* plane = base + (size_t)(mu * 2 + par) * link_plane_bytes(R, 2, Vh);
  if constexpr (R == 18) {
#pragma unroll
    for (int k = 0; k < 9; ++k) uw[k] = __ldg(reinterpret_cast<const uint32_t*>(plane + ((size_t)k * Vh + cb) * 4));
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint2 q = __ldg(reinterpret_cast<const uint2*>(plane + ((size_t)k * Vh + cb) * 8));
      uw[2 * k] = q.x;
      uw[2 * k + 1] = q.y;
    }
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
        C<T> r[3];
        T nrm;
        if constexpr (PREC == P16 && RL != 8) {
          uint32_t chi[3], uw[9];
          nrm = load_stag_h(a.in, Vh, cb_index(g, y), chi);
          if (hop == 0) {
            load_link_h<18>(links, Vh, mu, par, cb, uw);
            stag_mv_h<18>(uw, chi, false, r);
          } else {
            load_link_h<RL>(links, Vh, mu, par, cb, uw);
            stag_mv_h<RL>(uw, chi, false, r);
          }
        } else {
          T v[6];
          nrm = load_stag_spinor<PREC, T>(a.in, Vh, cb_index(g, y), v);
          C<T> h[3] = {{v[0], v[1]}, {v[2], v[3]}, {v[4], v[5]}};
          Link<T> U;
          if (hop == 0) LinkIO<PREC, 18>::load(links, Vh, mu, par, cb, U);
          else LinkIO<PREC, RL>::load(links, Vh, mu, par, cb, U);
          su3_mv(U, h, r);
        }
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
        C<T> r[3];
        T nrm;
        if constexpr (PREC == P16 && RL != 8) {
          uint32_t chi[3], uw[9];
          nrm = load_stag_h(a.in, Vh, ycb, chi);
          if (hop == 0) {
            load_link_h<18>(links, Vh, mu, 1 - par, ycb, uw);
            stag_mv_h<18>(uw, chi, true, r);
          } else {
            load_link_h<RL>(links, Vh, mu, 1 - par, ycb, uw);
            stag_mv_h<RL>(uw, chi, true, r);
          }
        } else {
          T v[6];
          nrm = load_stag_spinor<PREC, T>(a.in, Vh, ycb, v);
          C<T> h[3] = {{v[0], v[1]}, {v[2], v[3]}, {v[4], v[5]}};
          Link<T> U;
          if (hop == 0) LinkIO<PREC, 18>::load(links, Vh, mu, 1 - par, ycb, U);
          else LinkIO<PREC, RL>::load(links, Vh, mu, 1 - par, ycb, U);
          su3_mv_dag(U, h, r);
        }
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
