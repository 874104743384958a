// Wilson-clover stencil (Eq. 2), one thread per output site.
//
//   hopping term  D psi(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                     + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
//   kappa form    M psi    = Ahat psi - kappa D psi,  Ahat = 1 + 2 kappa A  (stored)
//   adjoint       M^dagger = Ahat - kappa D^dagger, D^dagger swaps the projectors.
//
// Spin basis: chiral, gamma_mu = [[0, B_mu], [B_mu^dagger, 0]] with
//   B_x = [[0, i], [i, 0]], B_y = [[0, -1], [1, 0]], B_z = [[i, 0], [0, -i]], B_t = 1.
// For P = 1 + s gamma_mu (s = -1 forward, +1 backward; flipped for the adjoint):
//   P psi = [h ; s B^dagger h]  with  h = psi_up + s B psi_low,
// so every hop multiplies only the 2-spin half spinor h by the link (Sec. 5:
// "similarity transforms to increase the sparsity of the Dirac matrices").
#pragma once
#include "field.cuh"

namespace dirac {

struct WilsonArg {
  char* out[2];          // output half-field base for each parity
  const char* in[2];     // input half-field base for each parity
  const char* gauge;     // links of this precision, [mu][parity][chunk][Vh]
  const char* clover;    // Ahat of this precision, [parity][chunk][Vh]; null: Ahat = 1
  Geom g;
  double kappa;
  int dagger;            // 1: apply the adjoint
  int out_parity;        // hop mode: parity of the output half-field
  // hop mode: out_p = Cpost (Cself self_p + s D_{p,1-p} in_{1-p}); a null matrix is the
  // identity, a null self drops that term, s = 0 skips the hopping term. Cself / Cpost
  // are clover-format fields ([parity][chunk][Vh]: Ahat or Ahat^-1).
  const char* self = nullptr;
  const char* c_self = nullptr;
  const char* c_post = nullptr;
  double s = 1.0;
};

// A neighbour spinor for wilson_hop and the factor that multiplies its projection: with
// FP16 storage the per-site norm is left out of the 24 values and folded into that
// factor (one multiply per projected component instead of one per stored value).
template <int PREC, typename T>
__device__ __forceinline__ T load_hop_spinor(const char* src, int Vh, int cb, T psi[24], T bc) {
  if constexpr (PREC == P16) {
    return bc * SpinorIO<P16, 24>::load_raw(src, Vh, cb, psi);
  } else {
    SpinorIO<PREC, 24>::load(src, Vh, cb, psi);
    return bc;
  }
}

// The spin projection of one hop: h = psi_up + s B_mu psi_low (two spin components,
// 3 colours each). Shared by the stencil and by the face packing of the domain
// decomposition, so that a projected face equals the stencil's own projection bit for bit.
template <int MU, typename T>
__device__ __forceinline__ void wilson_project(const T* psi, T s, C<T> h0[3], C<T> h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C<T> u0 = {psi[2 * c], psi[2 * c + 1]};
    C<T> u1 = {psi[6 + 2 * c], psi[6 + 2 * c + 1]};
    C<T> l0 = {psi[12 + 2 * c], psi[12 + 2 * c + 1]};
    C<T> l1 = {psi[18 + 2 * c], psi[18 + 2 * c + 1]};
    if (MU == 0) {        // B l = (i l1, i l0)
      h0[c] = u0 + s * times_i(l1);
      h1[c] = u1 + s * times_i(l0);
    } else if (MU == 1) { // B l = (-l1, l0)
      h0[c] = u0 - s * l1;
      h1[c] = u1 + s * l0;
    } else if (MU == 2) { // B l = (i l0, -i l1)
      h0[c] = u0 + s * times_i(l0);
      h1[c] = u1 - s * times_i(l1);
    } else {              // B l = l
      h0[c] = u0 + s * l0;
      h1[c] = u1 + s * l1;
    }
  }
}

// The rest of a hop after the projection: v = U h (U^dagger h for a backward hop), then
// acc += bc P-reconstruction of v.
template <int MU, typename T>
__device__ __forceinline__ void wilson_hop_proj(C<T> acc[4][3], const C<T> h0[3], const C<T> h1[3],
                                                const Link<T>& U, bool link_dag, T s, T bc) {
  C<T> v0[3], v1[3];
  if (link_dag) {
    su3_mv_dag(U, h0, v0);
    su3_mv_dag(U, h1, v1);
  } else {
    su3_mv(U, h0, v0);
    su3_mv(U, h1, v1);
  }
  // the hop's factor bc multiplies the accumulation (one fused multiply-add per real);
  // with bc = +-1 (FP32 / FP64 storage) this is exactly acc +- v
  const T ks = s * bc;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[0][c] = C<T>{fma(bc, v0[c].r, acc[0][c].r), fma(bc, v0[c].i, acc[0][c].i)};
    acc[1][c] = C<T>{fma(bc, v1[c].r, acc[1][c].r), fma(bc, v1[c].i, acc[1][c].i)};
    if (MU == 0) {        // B^dagger v = (-i v1, -i v0)
      acc[2][c] = C<T>{fma(ks, v1[c].i, acc[2][c].r), fma(-ks, v1[c].r, acc[2][c].i)};
      acc[3][c] = C<T>{fma(ks, v0[c].i, acc[3][c].r), fma(-ks, v0[c].r, acc[3][c].i)};
    } else if (MU == 1) { // B^dagger v = (v1, -v0)
      acc[2][c] = C<T>{fma(ks, v1[c].r, acc[2][c].r), fma(ks, v1[c].i, acc[2][c].i)};
      acc[3][c] = C<T>{fma(-ks, v0[c].r, acc[3][c].r), fma(-ks, v0[c].i, acc[3][c].i)};
    } else if (MU == 2) { // B^dagger v = (-i v0, i v1)
      acc[2][c] = C<T>{fma(ks, v0[c].i, acc[2][c].r), fma(-ks, v0[c].r, acc[2][c].i)};
      acc[3][c] = C<T>{fma(-ks, v1[c].i, acc[3][c].r), fma(ks, v1[c].r, acc[3][c].i)};
    } else {
      acc[2][c] = C<T>{fma(ks, v0[c].r, acc[2][c].r), fma(ks, v0[c].i, acc[2][c].i)};
      acc[3][c] = C<T>{fma(ks, v1[c].r, acc[3][c].r), fma(ks, v1[c].i, acc[3][c].i)};
    }
  }
}

template <int MU, typename T>
__device__ __forceinline__ void wilson_hop(C<T> acc[4][3], const T* psi, const Link<T>& U,
                                           bool link_dag, T s, T bc) {
  C<T> h0[3], h1[3];
  wilson_project<MU, T>(psi, s, h0, h1);
  wilson_hop_proj<MU, T>(acc, h0, h1, U, link_dag, s, bc);
}

// out[12] = Ahat(x) in[12] for the clover of precision PREC (block by block to bound
// register use).
template <int PREC, typename T>
__device__ __forceinline__ void apply_clover_site(const char* b, int Vh, int cb, const C<T> in[12],
                                                  C<T> out[12]) {
  if constexpr (PREC == P64 || PREC == P64DS) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      T v[36];
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        double2 q = ldg_chunk<double2>(b + ((size_t)(18 * blk + k) * Vh + cb) * 16);
        v[2 * k] = T(q.x); v[2 * k + 1] = T(q.y);
      }
      herm6_mv<T>(v, in + 6 * blk, out + 6 * blk);
    }
  } else if constexpr (PREC == P32) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      float v[36];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        float4 q = ldg_chunk<float4>(b + ((size_t)(9 * blk + k) * Vh + cb) * 16);
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
      }
      herm6_mv<T>(v, in + 6 * blk, out + 6 * blk);
    }
  } else {
    // 16-bit clover: the stored values times the per-site norm, which scales the 12
    // input components instead of the 72 entries
    float v[72];
    const float n = CloverIO<P16>::load_raw(b, Vh, cb, v);
    C<T> x[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = n * in[k];
    herm6_mv<T>(v, x, out);
    herm6_mv<T>(v + 36, x + 6, out + 6);
  }
}

// ---------------------------------------------------------------- 16-bit Ahat x self
// y = A x for one chirality block with the stored binary16 values of both: blk = the
// block's 18 half2 words (6 real diagonal entries in words 0..2, then L_ij, i > j, one
// complex per word), x = 6 complex binary16 words (re low, im high).
__device__ __forceinline__ void herm6_hh(const uint32_t blk[18], const uint32_t x[6], C<float> y[6]) {
  uint32_t nx[6];  // (-re, -im)
#pragma unroll
  for (int i = 0; i < 6; ++i) nx[i] = x[i] ^ 0x80008000u;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const uint32_t d = blk[i >> 1];
    if (i & 1) y[i] = C<float>{fma_hh<1, 0>(d, x[i], 0.f), fma_hh<1, 1>(d, x[i], 0.f)};
    else y[i] = C<float>{fma_hh<0, 0>(d, x[i], 0.f), fma_hh<0, 1>(d, x[i], 0.f)};
  }
  int w = 3;
#pragma unroll
  for (int i = 1; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const uint32_t l = blk[w++];
      // y_i += L x_j
      y[i].r = fma_hh<1, 1>(l, nx[j], fma_hh<0, 0>(l, x[j], y[i].r));
      y[i].i = fma_hh<1, 0>(l, x[j], fma_hh<0, 1>(l, x[j], y[i].i));
      // y_j += conj(L) x_i
      y[j].r = fma_hh<1, 1>(l, x[i], fma_hh<0, 0>(l, x[i], y[j].r));
      y[j].i = fma_hh<1, 0>(l, nx[i], fma_hh<0, 1>(l, x[i], y[j].i));
    }
  }
}

// av = Ahat self for 16-bit storage, from the stored binary16 values of the clover and of
// the site's own spinor; their two per-site norms scale the 12 results once.
__device__ __forceinline__ void clover_self_h(const char* clov, const char* self, int Vh, int cb, C<float> av[12]) {
  const float nc = __ldg(reinterpret_cast<const float*>(clov + (size_t)144 * Vh) + cb);
  const float ns = __ldg(reinterpret_cast<const float*>(self + (size_t)48 * Vh) + cb);
  uint32_t x[12];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int4 q = ldg_chunk<int4>(self + ((size_t)k * Vh + cb) * 16);
    x[4 * k] = (uint32_t)q.x; x[4 * k + 1] = (uint32_t)q.y; x[4 * k + 2] = (uint32_t)q.z; x[4 * k + 3] = (uint32_t)q.w;
  }
  // block 0: words 0..17 (chunks 0..3 and half of chunk 4); block 1: words 18..35
  uint32_t c[20];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int4 q = ldg_chunk<int4>(clov + ((size_t)k * Vh + cb) * 16);
    c[4 * k] = (uint32_t)q.x; c[4 * k + 1] = (uint32_t)q.y; c[4 * k + 2] = (uint32_t)q.z; c[4 * k + 3] = (uint32_t)q.w;
  }
  herm6_hh(c, x, av);
  c[0] = c[18];
  c[1] = c[19];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int4 q = ldg_chunk<int4>(clov + ((size_t)(5 + k) * Vh + cb) * 16);
    c[2 + 4 * k] = (uint32_t)q.x; c[3 + 4 * k] = (uint32_t)q.y; c[4 + 4 * k] = (uint32_t)q.z; c[5 + 4 * k] = (uint32_t)q.w;
  }
  herm6_hh(c, x + 6, av + 6);
  const float n = nc * ns;
#pragma unroll
  for (int k = 0; k < 12; ++k) av[k] = n * av[k];
}

// ---------------------------------------------------------------- 16-bit neighbours
// A 16-bit neighbour spinor for a hop: the upper two spin components converted (u, 12
// reals), the lower two kept as binary16 pairs (l, 6 words: spin 2 colours 0..2, spin 3
// colours 0..2, re low / im high); returns bc times the site norm, the hop's factor.
__device__ __forceinline__ float load_hop_h(const char* src, int Vh, int cb, float u[12], uint32_t l[6], float bc) {
  const float n = __ldg(reinterpret_cast<const float*>(src + (size_t)48 * Vh) + cb);
  uint32_t w[12];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int4 q = ldg_chunk<int4>(src + ((size_t)k * Vh + cb) * 16);
    w[4 * k] = (uint32_t)q.x; w[4 * k + 1] = (uint32_t)q.y; w[4 * k + 2] = (uint32_t)q.z; w[4 * k + 3] = (uint32_t)q.w;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
    u[2 * k] = f.x;
    u[2 * k + 1] = f.y;
    l[k] = w[6 + k];
  }
  return bc * n;
}

// The projection of wilson_project with binary16 lower components: each real is one
// fma of (s or -s) times a binary16 value into the FP32 upper value (sw: s in the low
// half, -s in the high half). s = +-1, so the result is round(u +- l), as in FP32.
template <int MU>
__device__ __forceinline__ void wilson_project_h(const float u[12], const uint32_t l[6], uint32_t sw,
                                                 C<float> h0[3], C<float> h1[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float u0r = u[2 * c], u0i = u[2 * c + 1], u1r = u[6 + 2 * c], u1i = u[7 + 2 * c];
    const uint32_t l0 = l[c], l1 = l[3 + c];
    if (MU == 0) {        // h = u + s (i l1, i l0)
      h0[c] = C<float>{fma_hh<1, 1>(sw, l1, u0r), fma_hh<0, 0>(sw, l1, u0i)};
      h1[c] = C<float>{fma_hh<1, 1>(sw, l0, u1r), fma_hh<0, 0>(sw, l0, u1i)};
    } else if (MU == 1) { // h = u + s (-l1, l0)
      h0[c] = C<float>{fma_hh<1, 0>(sw, l1, u0r), fma_hh<1, 1>(sw, l1, u0i)};
      h1[c] = C<float>{fma_hh<0, 0>(sw, l0, u1r), fma_hh<0, 1>(sw, l0, u1i)};
    } else if (MU == 2) { // h = u + s (i l0, -i l1)
      h0[c] = C<float>{fma_hh<1, 1>(sw, l0, u0r), fma_hh<0, 0>(sw, l0, u0i)};
      h1[c] = C<float>{fma_hh<0, 1>(sw, l1, u1r), fma_hh<1, 0>(sw, l1, u1i)};
    } else {              // h = u + s l
      h0[c] = C<float>{fma_hh<0, 0>(sw, l0, u0r), fma_hh<0, 1>(sw, l0, u0i)};
      h1[c] = C<float>{fma_hh<0, 0>(sw, l1, u1r), fma_hh<0, 1>(sw, l1, u1i)};
    }
  }
}
__device__ __forceinline__ uint32_t signs_h(float s) { return s > 0.f ? 0xBC003C00u : 0x3C00BC00u; }

template <int MU>
__device__ __forceinline__ void wilson_hop_h(C<float> acc[4][3], const float u[12], const uint32_t l[6],
                                             const Link<float>& U, bool link_dag, float s, float bc) {
  C<float> h0[3], h1[3];
  wilson_project_h<MU>(u, l, signs_h(s), h0, h1);
  wilson_hop_proj<MU, float>(acc, h0, h1, U, link_dag, s, bc);
}

// Launch shape per storage precision (threads per CTA, minimum resident CTAs per SM,
// which caps registers). FP32/FP16 are memory-latency bound and want many warps in
// flight; FP64 is FP64-ALU bound on this part.
#ifndef WILSON_INTERLEAVE
#define WILSON_INTERLEAVE 32
#endif
// Measured on GB300 at 24^3x128 (clover M): FP32 64x8 (128-register cap) 0.199 ms vs
// 128x1 (up to 255 registers) 0.288 ms; FP16 ~0.178 ms for every shape tried.
template <int PREC> struct WilsonShape { static constexpr int threads = 64, minb = 10; };
template <> struct WilsonShape<P32> { static constexpr int threads = 64, minb = 8; };
template <> struct WilsonShape<P64> { static constexpr int threads = 128, minb = 1; };
template <> struct WilsonShape<P64DS> { static constexpr int threads = 128, minb = 2; };

// One output site of the stencil: thread index idx over the Vh (hop mode) or 2 Vh
// (full operator) output sites. Shared by the single-RHS, multi-RHS and batched kernels.
template <int PREC, int R, bool FULLM>
__device__ __forceinline__ void wilson_site(const WilsonArg& a, int idx) {
  using T = typename Real<PREC>::T;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  int par, cb;
  if (FULLM) {
    // The two parities alternate every WILSON_INTERLEAVE threads (a warp: the parity
    // stays warp-uniform): the forward link U_mu(x) read by site x is read again as a
    // backward link by the neighbour x + mu of the other parity close in time, so it
    // comes from cache instead of a second DRAM pass over all links.
    if (idx >= 2 * Vh) return;
    constexpr int IL = WILSON_INTERLEAVE;
    const int grp = idx / (2 * IL), k = idx - grp * 2 * IL;
    if ((grp + 1) * IL <= Vh) {
      par = k >= IL;
      cb = grp * IL + k - par * IL;
    } else {  // last, incomplete pair of groups (Vh not a multiple of IL)
      const int half = Vh - grp * IL;
      par = k >= half;
      cb = grp * IL + k - par * half;
    }
  } else {
    if (idx >= Vh) return;
    par = a.out_parity;
    cb = idx;
  }
  int x[4];
  cb_coords(g, cb, par, x);
  // selects, not a runtime index into the parameter arrays (which would copy them
  // to local memory)
  const char* src = par ? a.in[0] : a.in[1];
  const char* self_in = par ? a.in[1] : a.in[0];
  char* dst = par ? a.out[1] : a.out[0];
  const T sf = a.dagger ? (T)1 : (T)-1;  // forward projector 1 - gamma (adjoint: 1 + gamma)
  const T sb = -sf;

  C<T> acc[4][3];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[s][c] = C<T>{0, 0};

#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (!FULLM && a.s == 0.0) break;  // hop mode without the hopping term
    // forward neighbour x + mu, link U_mu(x) stored at (mu, par, cb)
    {
      int y[4] = {x[0], x[1], x[2], x[3]};
      T bc = 1;
      if (++y[mu] == g.L[mu]) {
        y[mu] = 0;
        if (mu == 3 && g.apbc) bc = -1;
      }
      if constexpr (PREC == P16) {
        float u[12];
        uint32_t l[6];
        bc = load_hop_h(src, Vh, cb_index(g, y), u, l, bc);
        Link<T> U;
        LinkIO<PREC, R>::load(a.gauge, Vh, mu, par, cb, U);
        if (mu == 0) wilson_hop_h<0>(acc, u, l, U, false, sf, bc);
        if (mu == 1) wilson_hop_h<1>(acc, u, l, U, false, sf, bc);
        if (mu == 2) wilson_hop_h<2>(acc, u, l, U, false, sf, bc);
        if (mu == 3) wilson_hop_h<3>(acc, u, l, U, false, sf, bc);
      } else {
        T psi[24];
        bc = load_hop_spinor<PREC, T>(src, Vh, cb_index(g, y), psi, bc);
        Link<T> U;
        LinkIO<PREC, R>::load(a.gauge, Vh, mu, par, cb, U);
        if (mu == 0) wilson_hop<0>(acc, psi, U, false, sf, bc);
        if (mu == 1) wilson_hop<1>(acc, psi, U, false, sf, bc);
        if (mu == 2) wilson_hop<2>(acc, psi, U, false, sf, bc);
        if (mu == 3) wilson_hop<3>(acc, psi, U, false, sf, bc);
      }
    }
    // backward neighbour x - mu, link U_mu(x - mu) stored at (mu, 1 - par, cb(x - mu))
    {
      int y[4] = {x[0], x[1], x[2], x[3]};
      T bc = 1;
      if (y[mu]-- == 0) {
        y[mu] = g.L[mu] - 1;
        if (mu == 3 && g.apbc) bc = -1;
      }
      int ycb = cb_index(g, y);
      if constexpr (PREC == P16) {
        float u[12];
        uint32_t l[6];
        bc = load_hop_h(src, Vh, ycb, u, l, bc);
        Link<T> U;
        LinkIO<PREC, R>::load(a.gauge, Vh, mu, 1 - par, ycb, U);
        if (mu == 0) wilson_hop_h<0>(acc, u, l, U, true, sb, bc);
        if (mu == 1) wilson_hop_h<1>(acc, u, l, U, true, sb, bc);
        if (mu == 2) wilson_hop_h<2>(acc, u, l, U, true, sb, bc);
        if (mu == 3) wilson_hop_h<3>(acc, u, l, U, true, sb, bc);
      } else {
        T psi[24];
        bc = load_hop_spinor<PREC, T>(src, Vh, ycb, psi, bc);
        Link<T> U;
        LinkIO<PREC, R>::load(a.gauge, Vh, mu, 1 - par, ycb, U);
        if (mu == 0) wilson_hop<0>(acc, psi, U, true, sb, bc);
        if (mu == 1) wilson_hop<1>(acc, psi, U, true, sb, bc);
        if (mu == 2) wilson_hop<2>(acc, psi, U, true, sb, bc);
        if (mu == 3) wilson_hop<3>(acc, psi, U, true, sb, bc);
      }
    }
  }

  T out[24];
  bool clover_done = false;
  if constexpr (FULLM && PREC == P16) {
    if (a.clover) {  // Ahat self from the stored binary16 values (no conversions)
      C<float> av[12];
      clover_self_h(a.clover + (size_t)par * CloverIO<P16>::parity_bytes(Vh), self_in, Vh, cb, av);
      const float mk = -(float)a.kappa;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          out[6 * s + 2 * c] = fmaf(mk, acc[s][c].r, av[3 * s + c].r);
          out[6 * s + 2 * c + 1] = fmaf(mk, acc[s][c].i, av[3 * s + c].i);
        }
      clover_done = true;
    }
  }
  if (clover_done) {
  } else if (FULLM) {
    T self[24];
    C<T> sv[12], av[12];
    SpinorIO<PREC, 24>::load(self_in, Vh, cb, self);
#pragma unroll
    for (int k = 0; k < 12; ++k) sv[k] = C<T>{self[2 * k], self[2 * k + 1]};
    if (a.clover) {
      apply_clover_site<PREC, T>(a.clover + (size_t)par * CloverIO<PREC>::parity_bytes(Vh), Vh, cb, sv, av);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) av[k] = sv[k];
    }
    const T mk = -(T)a.kappa;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        out[6 * s + 2 * c] = fma(mk, acc[s][c].r, av[3 * s + c].r);
        out[6 * s + 2 * c + 1] = fma(mk, acc[s][c].i, av[3 * s + c].i);
      }
  } else {
    const T sc = (T)a.s;
    C<T> v[12];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[3 * s + c] = sc * acc[s][c];
    const size_t pb = CloverIO<PREC>::parity_bytes(Vh);
    if (a.self) {
      C<T> cv[12];
      bool done = false;
      if constexpr (PREC == P16) {
        if (a.c_self) {  // Cself self from the stored binary16 values
          clover_self_h(a.c_self + par * pb, a.self, Vh, cb, cv);
          done = true;
        }
      }
      if (!done) {
        T sl[24];
        SpinorIO<PREC, 24>::load(a.self, Vh, cb, sl);
        C<T> sv[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) sv[k] = C<T>{sl[2 * k], sl[2 * k + 1]};
        if (a.c_self) {
          apply_clover_site<PREC, T>(a.c_self + par * pb, Vh, cb, sv, cv);
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) cv[k] = sv[k];
        }
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = v[k] + cv[k];
    }
    if (a.c_post) {
      C<T> w[12];
      apply_clover_site<PREC, T>(a.c_post + par * pb, Vh, cb, v, w);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = w[k];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      out[2 * k] = v[k].r;
      out[2 * k + 1] = v[k].i;
    }
  }
  SpinorIO<PREC, 24>::store(dst, Vh, cb, out);
}

template <int PREC, int R, bool FULLM>
__global__ void __launch_bounds__(WilsonShape<PREC>::threads, WilsonShape<PREC>::minb)
    wilson_kernel(const WilsonArg a) {
  wilson_site<PREC, R, FULLM>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

template <int PREC>
void launch_wilson_prec(int recon, bool fullm, const WilsonArg& a, cudaStream_t st) {
  int n = fullm ? 2 * a.g.Vh : a.g.Vh;
  constexpr int T = WilsonShape<PREC>::threads;
  dim3 block(T), grid((n + T - 1) / T);
  if (recon == 18) {
    if (fullm) wilson_kernel<PREC, 18, true><<<grid, block, 0, st>>>(a);
    else wilson_kernel<PREC, 18, false><<<grid, block, 0, st>>>(a);
  } else if (recon == 12) {
    if (fullm) wilson_kernel<PREC, 12, true><<<grid, block, 0, st>>>(a);
    else wilson_kernel<PREC, 12, false><<<grid, block, 0, st>>>(a);
  } else {
    if (fullm) wilson_kernel<PREC, 8, true><<<grid, block, 0, st>>>(a);
    else wilson_kernel<PREC, 8, false><<<grid, block, 0, st>>>(a);
  }
}

}  // namespace dirac
