// Clover term of Eq. 2, built once per gauge field on the GPU in FP64.
//
// The paper gives only the structure of A_x (footnote to Eq. 2: Hermitian diagonal
// blocks, 72 reals). Reading used:
//   A(x) = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
//   sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],
//   F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger)/8 with the colour trace removed,
//   Q_{mu nu}(x) = sum of the four plaquette leaves around x (mu -> nu orientation).
// In the chiral basis gamma_mu = [[0, B_mu], [B_mu^dagger, 0]] sigma_{mu nu} is block
// diagonal: upper (i/2)(B_mu B_nu^dagger - B_nu B_mu^dagger), lower
// (i/2)(B_mu^dagger B_nu - B_nu^dagger B_mu). The stored field is
// Ahat = 1 + 2 kappa A, two Hermitian 6x6 blocks per site.
#include "internal.h"

namespace dirac {

using cd = C<double>;
struct M3 { cd m[3][3]; };

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cd s = {0, 0};
      for (int k = 0; k < 3; ++k) cmac(s, a.m[i][k], b.m[k][j]);
      c.m[i][j] = s;
    }
  return c;
}
__device__ __forceinline__ M3 dag(const M3& a) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.m[i][j] = conj(a.m[j][i]);
  return c;
}

struct NatLinks {
  const double* u;
  Geom g;
  __device__ M3 at(const int x[4], int mu) const {
    int64_t lex = (((int64_t)x[3] * g.L[2] + x[2]) * g.L[1] + x[1]) * g.L[0] + x[0];
    const double* p = u + (lex * 4 + mu) * 18;
    M3 r;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) r.m[i][j] = cd{p[6 * i + 2 * j], p[6 * i + 2 * j + 1]};
    return r;
  }
};

__device__ __forceinline__ void step(int y[4], const int x[4], const Geom& g, int mu, int dm, int nu, int dn) {
  for (int k = 0; k < 4; ++k) y[k] = x[k];
  y[mu] = (y[mu] + dm + g.L[mu]) % g.L[mu];
  y[nu] = (y[nu] + dn + g.L[nu]) % g.L[nu];
}

// 2x2 complex helpers for the spin blocks
struct M2 { cd m[2][2]; };
__device__ __forceinline__ M2 bmat(int mu) {
  M2 b;
  const cd z = {0, 0}, one = {1, 0}, mone = {-1, 0}, I = {0, 1}, mI = {0, -1};
  if (mu == 0) { b.m[0][0] = z; b.m[0][1] = I; b.m[1][0] = I; b.m[1][1] = z; }
  else if (mu == 1) { b.m[0][0] = z; b.m[0][1] = mone; b.m[1][0] = one; b.m[1][1] = z; }
  else if (mu == 2) { b.m[0][0] = I; b.m[0][1] = z; b.m[1][0] = z; b.m[1][1] = mI; }
  else { b.m[0][0] = one; b.m[0][1] = z; b.m[1][0] = z; b.m[1][1] = one; }
  return b;
}
__device__ __forceinline__ M2 mul2(const M2& a, const M2& b) {
  M2 c;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      cd s = {0, 0};
      for (int k = 0; k < 2; ++k) cmac(s, a.m[i][k], b.m[k][j]);
      c.m[i][j] = s;
    }
  return c;
}
__device__ __forceinline__ M2 dag2(const M2& a) {
  M2 c;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) c.m[i][j] = conj(a.m[j][i]);
  return c;
}

// Inverse of a 6x6 complex matrix by Gauss-Jordan elimination with partial pivoting.
// Returns false for a singular matrix.
__device__ bool invert6(cd M[6][6], cd Inv[6][6]) {
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) Inv[r][c] = cd{r == c ? 1.0 : 0.0, 0.0};
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    double best = M[col][col].r * M[col][col].r + M[col][col].i * M[col][col].i;
    for (int r = col + 1; r < 6; ++r) {
      double m = M[r][col].r * M[r][col].r + M[r][col].i * M[r][col].i;
      if (m > best) { best = m; piv = r; }
    }
    if (!(best > 0)) return false;
    if (piv != col)
      for (int c = 0; c < 6; ++c) {
        cd t = M[col][c]; M[col][c] = M[piv][c]; M[piv][c] = t;
        t = Inv[col][c]; Inv[col][c] = Inv[piv][c]; Inv[piv][c] = t;
      }
    // 1 / pivot
    const cd p = M[col][col];
    const double d = p.r * p.r + p.i * p.i;
    const cd ip = {p.r / d, -p.i / d};
    for (int c = 0; c < 6; ++c) {
      M[col][c] = ip * M[col][c];
      Inv[col][c] = ip * Inv[col][c];
    }
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      const cd f = M[r][col];
      for (int c = 0; c < 6; ++c) {
        M[r][c] = M[r][c] - f * M[col][c];
        Inv[r][c] = Inv[r][c] - f * Inv[col][c];
      }
    }
  }
  return true;
}

// pack a Hermitian 6x6 block: 6 real diagonal entries, then the 15 entries below the
// diagonal (row-major), symmetrised (the average of H_rc and conj(H_cr))
__device__ void pack_herm6(const cd H[6][6], double* o) {
  for (int r = 0; r < 6; ++r) o[r] = H[r][r].r;
  int k = 6;
  for (int r = 1; r < 6; ++r)
    for (int c = 0; c < r; ++c) {
      o[k++] = 0.5 * (H[r][c].r + H[c][r].r);
      o[k++] = 0.5 * (H[r][c].i - H[c][r].i);
    }
}

template <int NP>
__global__ void build_clover_kernel(const double* links, Geom g, double kappa, double csw,
                                    char* d64, char* d32, char* d16, char* i64, char* i32, char* i16) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * (int64_t)g.Vh) return;
  int par = (int)(i / g.Vh), cb = (int)(i - (int64_t)par * g.Vh);
  int x[4];
  cb_coords(g, cb, par, x);
  NatLinks U{links, g};
  // Ahat blocks accumulated as full complex 6x6 (index 3*s + c, s in {0,1} of the block)
  cd A[2][6][6];
  for (int b = 0; b < 2; ++b)
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) A[b][r][c] = cd{r == c ? 1.0 : 0.0, 0.0};
  const double coef = 2.0 * kappa * csw * 0.5;  // 2 kappa * c_sw/2; the i's are applied below
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu) {
      int y1[4], y2[4], y3[4];
      // (+mu, +nu): U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
      step(y1, x, g, mu, 1, nu, 0);
      step(y2, x, g, mu, 0, nu, 1);
      M3 Q = mul(mul(U.at(x, mu), U.at(y1, nu)), mul(dag(U.at(y2, mu)), dag(U.at(x, nu))));
      // (-mu, +nu): U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
      step(y1, x, g, mu, -1, nu, 1);
      step(y2, x, g, mu, -1, nu, 0);
      M3 t = mul(mul(U.at(x, nu), dag(U.at(y1, mu))), mul(dag(U.at(y2, nu)), U.at(y2, mu)));
      for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + t.m[a][b];
      // (-mu, -nu): U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
      step(y1, x, g, mu, -1, nu, 0);
      step(y2, x, g, mu, -1, nu, -1);
      step(y3, x, g, mu, 0, nu, -1);
      t = mul(mul(dag(U.at(y1, mu)), dag(U.at(y2, nu))), mul(U.at(y2, mu), U.at(y3, nu)));
      for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + t.m[a][b];
      // (+mu, -nu): U_nu(x-nu)^+ U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^+
      step(y1, x, g, mu, 0, nu, -1);
      step(y2, x, g, mu, 1, nu, -1);
      t = mul(mul(dag(U.at(y1, nu)), U.at(y1, mu)), mul(U.at(y2, nu), dag(U.at(x, mu))));
      for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Q.m[a][b] = Q.m[a][b] + t.m[a][b];
      // F = (Q - Q^+)/8, traceless
      M3 F;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) F.m[a][b] = 0.125 * (Q.m[a][b] - conj(Q.m[b][a]));
      cd tr = (1.0 / 3.0) * (F.m[0][0] + F.m[1][1] + F.m[2][2]);
      for (int a = 0; a < 3; ++a) F.m[a][a] = F.m[a][a] - tr;
      // spin blocks of sigma_{mu nu} without its factor i/2: S = [g_mu, g_nu]-block
      M2 Bm = bmat(mu), Bn = bmat(nu);
      M2 Su = mul2(Bm, dag2(Bn)), Su2 = mul2(Bn, dag2(Bm));
      M2 Sl = mul2(dag2(Bm), Bn), Sl2 = mul2(dag2(Bn), Bm);
      for (int blk = 0; blk < 2; ++blk)
        for (int s = 0; s < 2; ++s)
          for (int tt = 0; tt < 2; ++tt) {
            cd sg = blk == 0 ? Su.m[s][tt] - Su2.m[s][tt] : Sl.m[s][tt] - Sl2.m[s][tt];
            // A += coef * (i/2 * i) * sg (x) F  = coef * (-1/2) * sg (x) F
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) {
                cd v = sg * F.m[a][b];
                A[blk][3 * s + a][3 * tt + b] = A[blk][3 * s + a][3 * tt + b] + (-0.5 * coef) * v;
              }
          }
    }
  double v[72];
  for (int b = 0; b < 2; ++b) pack_herm6(A[b], v + 36 * b);
  if (d64) CloverIO<P64>::store(d64 + (size_t)par * CloverIO<P64>::parity_bytes(g.Vh), g.Vh, cb, v);
  if (d32) CloverIO<P32>::store(d32 + (size_t)par * CloverIO<P32>::parity_bytes(g.Vh), g.Vh, cb, v);
  if (d16) CloverIO<P16>::store(d16 + (size_t)par * CloverIO<P16>::parity_bytes(g.Vh), g.Vh, cb, v);
  if (i64 || i32 || i16) {
    // Ahat^-1 for the even-odd (Schur complement) operator; NaN marks a singular block
    for (int b = 0; b < 2; ++b) {
      cd Inv[6][6];
      if (!invert6(A[b], Inv))
        for (int r = 0; r < 6; ++r)
          for (int c = 0; c < 6; ++c) Inv[r][c] = cd{nan(""), nan("")};
      pack_herm6(Inv, v + 36 * b);
    }
    if (i64) CloverIO<P64>::store(i64 + (size_t)par * CloverIO<P64>::parity_bytes(g.Vh), g.Vh, cb, v);
    if (i32) CloverIO<P32>::store(i32 + (size_t)par * CloverIO<P32>::parity_bytes(g.Vh), g.Vh, cb, v);
    if (i16) CloverIO<P16>::store(i16 + (size_t)par * CloverIO<P16>::parity_bytes(g.Vh), g.Vh, cb, v);
  }
}

void launch_build_clover(const double* links, const Geom& g, double kappa, double csw,
                         char* const dst[3], char* const inv[3], unsigned prec_mask, cudaStream_t st) {
  int64_t n = 2 * (int64_t)g.Vh;
  dim3 grid((unsigned)((n + 127) / 128)), block(128);
  auto pick = [&](char* const* a, int q) { return (a && (prec_mask & (1u << q))) ? a[q] : nullptr; };
  build_clover_kernel<0><<<grid, block, 0, st>>>(links, g, kappa, csw, pick(dst, 0), pick(dst, 1),
                                                 pick(dst, 2), pick(inv, 0), pick(inv, 1), pick(inv, 2));
}

}  // namespace dirac
