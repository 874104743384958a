// Multi-right-hand-side Wilson-clover operator on the tensor cores (FP16 storage).
//
// With many right-hand sides on one lattice, the link-times-spinor product of every hop
// (Eq. 2) becomes a dense contraction: at a site x the 8 links are shared by all
// right-hand sides, so the hopping term of output spin s for right-hand side r is
//     (D psi_r)_s(x)[a] = sum over hops j and colours b of  h_{r,j}[.](b) W_j[a][b]
// a GEMM with rows = right-hand sides, K = (hop, colour) and columns = output colour.
// Each hop is spin-projected first (Sec. 5: the projectors of Eq. 2 leave two spin
// components), and the lower two output spins are phase multiples (+-1, +-i) of the
// upper ones, which are folded into two more variants of the link operand.
//
// Per site the products run as mma.sync m16n8k16 (FP16 operands, FP32 accumulation):
// rows = up to 16 right-hand sides, K = 24 complex (8 hops x 3 colours) = 48 reals in
// 3 k-tiles, columns = 3 colours x (re, im) (6 of 8 used). The clover term is one more
// k-tile per chirality: the 6x6 Hermitian block of Ahat acting on the site's own spinor.
//
// A CTA works through tiles of TS sites of one parity and all right-hand sides with two
// warp roles and two tile stages in shared memory:
//   producers (6 warps): the tile's links (forward and backward, decoded once, stored in
//     B-operand order) and stored clover; one thread per (site, right-hand side, half of
//     the hops) gathers its neighbour spinors, projects them in binary16 arithmetic and
//     writes the A rows. Neighbour indices come from a per-lattice table, fetched a tile
//     ahead, so each tile costs the producers one memory round trip. FP16 spinors carry per-site norms, so
//     each row is scaled to a common scale S (the largest norm among its terms), kept
//     beside it;
//   consumers (2 warps): one warp per site loads the A fragments (ldmatrix), builds the
//     B fragments from the staged links and clover, runs 16 MMAs (12 hopping, 4 clover),
//     re-encodes the outputs in FP16 with new per-site norms, and the 2 warps store the
//     tile's outputs coalesced. (The producers' gather is the longer half of the work:
//     measured with 4 + 4 warps, producers alone 1.20 ms, consumers alone 0.63 ms for
//     24^3x64 with 12 right-hand sides.)
// Named barriers hand each stage from producers to consumers and back; both roles walk
// the same tile sequence, so every barrier has its full count.
// Arithmetic: binary16 operands (spinor values relative to their row scale, links,
// clover), FP32 accumulation: results are within the FP16 storage bound of the
// single-right-hand-side operator, not bitwise equal to it.
#include <cstdint>
#include <cuda_fp16.h>

#include "internal.h"
#include "mrhs_tc.h"

namespace dirac {
namespace tc {

constexpr int TS = 8;           // sites per tile (one parity, consecutive cb)
constexpr int NT = 256;         // threads per CTA
constexpr int NPT = 192;        // producer threads (warps 0..5)
constexpr int NCW = 2;          // consumer warps (6..7)
constexpr int ROWS = 16;        // right-hand sides per tile (MMA rows)

constexpr int NST = 2;          // tile stages in flight
// named barriers (0 is __syncthreads)
constexpr int BAR_FULL = 1;     // + stage: producers arrive, consumers wait
constexpr int BAR_EMPTY = 4;    // + stage: consumers arrive, producers wait
constexpr int BAR_CONS = 8;     // consumers among themselves
// encoded outputs of site i staged in its A area: row r at byte 16 i + 80 r (12 binary16
// pairs, then the FP32 norm): 8 sites x 4 rows of a warp fall on distinct banks
constexpr int OUT_ROW_W = 20;   // words per output row

// One tile stage in shared memory.
//  A[site][spin-row s'][rhs][chunk]: 8 chunks of 16 bytes = 64 binary16 per row:
//    chunks 0..5: the 24 hop positions P = hop*3 + colour, hop = 2*mu + dir (dir 0 =
//    forward), each a (re, im) binary16 pair; chunks 6..7: the clover operand of
//    chirality s' (positions 4*j' + c', spin 2 s' + j', colour c'; c' = 3 zero).
//    The chunk index is XOR-swizzled with ((rhs ^ site) & 7): ldmatrix of 8 rows of one
//    site and the producers' stores of 8 sites of one row both hit 8 distinct bank groups.
//    After the MMAs the same bytes hold the site's encoded outputs (see OUT_ROW_W).
//  link[site][P*4 + a] = W_hop(P)[a][colour(P)] as a binary16 pair; W = U_mu(x) for a
//    forward hop, U_mu(x - mu)^dagger backward; a = 3 is zero (padding column).
//  craw[site]: the 72 stored binary16 values of Ahat (two packed Hermitian blocks).
struct Stage {
  uint4 A[TS][2][ROWS][8];
  uint32_t link[TS][100];       // 96 used; the padding spreads the sites over the banks
  uint32_t craw[TS][36];
  float S[TS][ROWS];
};
struct Smem {
  Stage st[NST];
};

// PRMT selectors picking a signed permutation of a binary16 pair w = (x, y) from the
// 8 bytes of (w, w ^ 0x80008000): F_reim(i^k W) = kSel[(k - reim) & 3] where
// F_0(v) = (Re v, -Im v) and F_1(v) = (Im v, Re v) are the two B-operand rows of a
// complex entry (column (a, re) and (a, im) of the real GEMM).
__constant__ uint32_t kSel[4] = {0x7610u, 0x5476u, 0x3254u, 0x1032u};

// Phase exponent k (c = i^k) of the lower output spin 2 + s' of a hop in direction mu,
// forward (dir 0, projector 1 - gamma) or backward (dir 1, 1 + gamma): the lower
// spins of (1 -/+ gamma_mu) are +-1 or +-i times one projected component (chiral basis).
__constant__ int kLowK[2][2][4] = {{{1, 2, 1, 2}, {1, 0, 3, 2}},   // forward: s' = 0, 1
                                   {{3, 0, 3, 0}, {3, 2, 1, 0}}};  // backward

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }
__device__ __forceinline__ __half2 hswap(__half2 h) { return __lowhigh2highlow(h); }

// Tile t of lattice L: parity, first checkerboard index, right-hand-side group.
struct TileRef {
  int par, cb0, rg, nrows;
};
__device__ __forceinline__ TileRef tile_ref(const TcLat& L, int t) {
  const int per_rg = 2 * L.ctiles;
  TileRef r;
  r.rg = t / per_rg;
  const int k = t - r.rg * per_rg;
  r.par = k & 1;
  r.cb0 = (k >> 1) * TS;
  r.nrows = min(ROWS, L.nrhs - r.rg * ROWS);
  return r;
}

__device__ __forceinline__ int lattice_of(const TcLat* lats, int nlat, int t) {
  int l = 0;
  while (l + 1 < nlat && t >= lats[l + 1].tile_begin) ++l;
  return l;
}

// ---------------------------------------------------------------- producers
// Raw stored reals of one link (FP16, R = 12 or 18), loaded before use.
template <int R> struct RawLink {
  uint32_t w[R / 2];
};
template <int R>
__device__ __forceinline__ void load_raw_link(const char* gauge, int Vh, int mu, int par, int cb, RawLink<R>& q) {
  const char* plane = gauge + (size_t)(mu * 2 + par) * (size_t)R * 2 * Vh;
  if constexpr (R == 18) {
#pragma unroll
    for (int k = 0; k < 9; ++k) q.w[k] = __ldg(reinterpret_cast<const uint32_t*>(plane + ((size_t)k * Vh + cb) * 4));
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(plane + ((size_t)k * Vh + cb) * 8));
      q.w[2 * k] = v.x;
      q.w[2 * k + 1] = v.y;
    }
  }
}

// the link in B-operand order: one 16-byte chunk per colour b = (W[0][b], W[1][b], W[2][b], 0)
template <int R>
__device__ __forceinline__ void store_link(const RawLink<R>& q, int dir, uint4* dst) {
  C<float> U[3][3];
#pragma unroll
  for (int e = 0; e < R / 2; ++e) {
    const float2 f = __half22float2(u2h(q.w[e]));
    U[e / 3][e % 3] = C<float>{f.x, f.y};
  }
  if constexpr (R == 12) {
    // third row = conj(row 0 x row 1) (unitarity, det = 1)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int a = (j + 1) % 3, b = (j + 2) % 3;
      U[2][j] = conj(U[0][a] * U[1][b] - U[0][b] * U[1][a]);
    }
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    uint32_t w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const C<float> e = dir == 0 ? U[a][b] : conj(U[b][a]);
      w[a] = h2u(__floats2half2_rn(e.r, e.i));
    }
    dst[b] = make_uint4(w[0], w[1], w[2], 0u);
  }
}

// projected pair h = u + s B l of hop direction MU (s = -1 forward, +1 backward),
// scaled by rr: the spin components of Eq. 2 after the projector, chiral basis
//   B_x l = (i l1, i l0), B_y l = (-l1, l0), B_z l = (i l0, -i l1), B_t l = (l0, l1)
template <int MU>
__device__ __forceinline__ void project(const uint32_t w[12], int dir, __half2 rr, uint32_t h0[3], uint32_t h1[3]) {
  const __half2 ur = rr;
  const __half2 sr = dir == 0 ? __hneg2(rr) : rr;                       // s * rr
  const __half2 im = __halves2half2(__float2half_rn(-1.0f), __float2half_rn(1.0f));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const __half2 u0 = __hmul2(u2h(w[c]), ur), u1 = __hmul2(u2h(w[3 + c]), ur);
    const __half2 l0 = u2h(w[6 + c]), l1 = u2h(w[9 + c]);
    if (MU == 0) {
      const __half2 k = __hmul2(sr, im);
      h0[c] = h2u(__hfma2(k, hswap(l1), u0));
      h1[c] = h2u(__hfma2(k, hswap(l0), u1));
    } else if (MU == 1) {
      h0[c] = h2u(__hfma2(__hneg2(sr), l1, u0));
      h1[c] = h2u(__hfma2(sr, l0, u1));
    } else if (MU == 2) {
      const __half2 k = __hmul2(sr, im);
      h0[c] = h2u(__hfma2(k, hswap(l0), u0));
      h1[c] = h2u(__hfma2(__hneg2(k), hswap(l1), u1));
    } else {
      h0[c] = h2u(__hfma2(sr, l0, u0));
      h1[c] = h2u(__hfma2(sr, l1, u1));
    }
  }
}

// the neighbour entry of hop h (runtime) from the two int4 of a site's table row
__device__ __forceinline__ int nbr_of(const int4& a, const int4& b, int h) {
  const int4 v = h < 4 ? a : b;
  const int k = h & 3;
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

template <int R>
__device__ void producer(Smem& sm, const TcLat* __restrict__ lats, int nlat, int ntiles) {
  const int tid = threadIdx.x;  // 0 .. NPT - 1
  // every item and link of this thread belongs to site my_i of the tile; its row of the
  // neighbour table is fetched one tile ahead, so a tile's loads all depend only on
  // values already in registers (one memory round trip per tile)
  const int my_i = tid & (TS - 1);
  int4 pn0 = make_int4(0, 0, 0, 0), pn1 = make_int4(0, 0, 0, 0);
  auto fetch = [&](int t) {
    if (t >= ntiles) return;
    const TcLat& L = lats[lattice_of(lats, nlat, t)];
    const TileRef tr = tile_ref(L, t - L.tile_begin);
    const int cb = tr.cb0 + my_i;
    if (cb < L.g.Vh) {
      const int4* p = reinterpret_cast<const int4*>(L.nbr + ((size_t)tr.par * L.g.Vh + cb) * 8);
      pn0 = __ldg(p);
      pn1 = __ldg(p + 1);
    }
  };
  fetch(blockIdx.x);
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it % NST;
    if (it >= NST) bar_sync(BAR_EMPTY + s, NT);
    Stage& S = sm.st[s];
    const TcLat& L = lats[lattice_of(lats, nlat, t)];
    const TileRef tr = tile_ref(L, t - L.tile_begin);
    const Geom& g = L.g;
    const int Vh = g.Vh;
    const int4 nb0 = pn0, nb1 = pn1;
    fetch(t + gridDim.x);
    // ---- links (threads 0..63) and stored clover (64..127) of the tile: loads first
    RawLink<R> lq;
    int lhop = 0, lsite = -1;
    uint4 cq = make_uint4(0, 0, 0, 0), cq8 = make_uint4(0, 0, 0, 0);
    int cq_site = -1, cq_c = 0;
    if (tid < TS * 8) {
      const int hop = tid / TS;
      const int mu = hop >> 1, dir = hop & 1;
      const int cb = tr.cb0 + my_i;
      if (cb < Vh) {
        const int ycb = nbr_of(nb0, nb1, hop) & 0x7fffffff;
        load_raw_link<R>(L.gauge, Vh, mu, dir == 0 ? tr.par : 1 - tr.par, dir == 0 ? cb : ycb, lq);
        lhop = hop;
        lsite = my_i;
      }
    } else {
      // 64 threads, 8 per site: stored clover chunk c (thread c = 0 also chunk 8)
      const int k = tid - TS * 8;
      const int i = k >> 3, c = k & 7;
      const int cb = tr.cb0 + i;
      if (i < TS && cb < Vh) {
        if (L.clover) {
          const char* b = L.clover + (size_t)tr.par * CloverIO<P16>::parity_bytes(Vh);
          cq = __ldg(reinterpret_cast<const uint4*>(b + ((size_t)c * Vh + cb) * 16));
          if (c == 0) cq8 = __ldg(reinterpret_cast<const uint4*>(b + ((size_t)8 * Vh + cb) * 16));
        }
        cq_site = i;
        cq_c = c;
      }
    }
    // the link and clover chunks are stored once they arrive
    if (lsite >= 0) store_link<R>(lq, lhop & 1, reinterpret_cast<uint4*>(&S.link[lsite][lhop * 12]));
    if (cq_site >= 0) {
      uint4* dst = reinterpret_cast<uint4*>(&S.craw[cq_site][0]);
      if (!L.clover) {
        // Ahat = 1: the 6 diagonal reals of each block are 1, everything else 0
        const __half one = __float2half_rn(1.0f), zero = __float2half_rn(0.0f);
        __half v[8], v8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          v[j] = (cq_c * 8 + j) % 36 < 6 ? one : zero;
          v8[j] = (64 + j) % 36 < 6 ? one : zero;
        }
        cq = *reinterpret_cast<const uint4*>(v);
        cq8 = *reinterpret_cast<const uint4*>(v8);
      }
      dst[cq_c] = cq;
      if (cq_c == 0) dst[8] = cq8;
    }
    // items: a warp takes 8 sites x 4 right-hand sides of one hop half (hh uniform in the
    // warp, so the projection code does not diverge)
    const int nitems = TS * ((tr.nrows + 3) & ~3) * 2;
    for (int q = tid; q < nitems; q += NPT) {
      const int c = q >> 5;
      const int i = q & (TS - 1), hh = c & 1, rloc = 4 * (c >> 1) + ((q >> 3) & 3);
      const int cb = tr.cb0 + i;
      if (cb >= Vh || rloc >= tr.nrows) continue;
      const size_t hb = (size_t)52 * Vh;
      const char* fld = L.in + (size_t)(tr.rg * ROWS + rloc) * L.field_bytes;
      const char* src = fld + (size_t)(1 - tr.par) * hb;   // neighbours: other parity
      const char* self = fld + (size_t)tr.par * hb;
      const int nb[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};  // site i == my_i
      const int4 nbs = hh ? nb1 : nb0;  // this half's 4 hops
      const int nh[4] = {nbs.x, nbs.y, nbs.z, nbs.w};
      // loads first: all 8 norms, own norm, this half's 4 neighbour spinors
      float n[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        n[j] = __ldg(reinterpret_cast<const float*>(src + (size_t)48 * Vh) + (nb[j] & 0x7fffffff));
      const float nself = __ldg(reinterpret_cast<const float*>(self + (size_t)48 * Vh) + cb);
      const float ncl = L.clover ? __ldg(reinterpret_cast<const float*>(
                                           L.clover + (size_t)tr.par * CloverIO<P16>::parity_bytes(Vh) +
                                           (size_t)144 * Vh) + cb)
                                 : 1.0f;
      uint4 q4[4][3];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int y = nh[jj] & 0x7fffffff;
#pragma unroll
        for (int k = 0; k < 3; ++k) q4[jj][k] = __ldg(reinterpret_cast<const uint4*>(src + ((size_t)k * Vh + y) * 16));
      }
      uint4 qs[3];
      if (hh == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) qs[k] = __ldg(reinterpret_cast<const uint4*>(self + ((size_t)k * Vh + cb) * 16));
      }
      // row scale S = max(kappa n_j, n_self n_cl)
      const float kap = L.kappa;
      float m = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) m = fmaxf(m, n[j]);
      const float sc = nself * ncl;
      const float Sr = fmaxf(m * fabsf(kap), sc);
      const float inv = Sr > 0.f ? 1.0f / Sr : 0.f;
      const int sw = (rloc ^ i) & 7;
      uint32_t h[2][12];  // [s'][4 hops x 3 colours]
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float nj = hh ? n[4 + jj] : n[jj];
        const float rj = ((nh[jj] < 0) ? kap : -kap) * nj * inv;  // -kappa * bc * n / S
        const __half2 rr = __float2half2_rn(rj);
        const uint32_t* w = reinterpret_cast<const uint32_t*>(q4[jj]);
        const int dir = jj & 1;
        if (hh == 0) {
          if (jj < 2) project<0>(w, dir, rr, &h[0][3 * jj], &h[1][3 * jj]);
          else project<1>(w, dir, rr, &h[0][3 * jj], &h[1][3 * jj]);
        } else {
          if (jj < 2) project<2>(w, dir, rr, &h[0][3 * jj], &h[1][3 * jj]);
          else project<3>(w, dir, rr, &h[0][3 * jj], &h[1][3 * jj]);
        }
      }
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        uint4* row = S.A[i][sp][rloc];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          row[(3 * hh + c) ^ sw] = make_uint4(h[sp][4 * c], h[sp][4 * c + 1], h[sp][4 * c + 2], h[sp][4 * c + 3]);
      }
      if (hh == 0) {
        // own spinor for the clover rows: chirality chi = spins 2 chi, 2 chi + 1
        S.S[i][rloc] = Sr;
        const uint32_t* w = reinterpret_cast<const uint32_t*>(qs);
        const __half2 rs = __float2half2_rn(sc * inv);
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
          uint32_t cv[8];
#pragma unroll
          for (int jp = 0; jp < 2; ++jp) {
#pragma unroll
            for (int c = 0; c < 3; ++c) cv[4 * jp + c] = h2u(__hmul2(u2h(w[3 * (2 * chi + jp) + c]), rs));
            cv[4 * jp + 3] = 0u;
          }
          uint4* row = S.A[i][chi][rloc];
          row[6 ^ sw] = make_uint4(cv[0], cv[1], cv[2], cv[3]);
          row[7 ^ sw] = make_uint4(cv[4], cv[5], cv[6], cv[7]);
        }
      }
    }
    bar_arrive(BAR_FULL + s, NT);
  }
  // the consumers' arrivals for the last NST tiles
  for (int k = it - NST < 0 ? 0 : it - NST; k < it; ++k) bar_sync(BAR_EMPTY + k % NST, NT);
}

// ---------------------------------------------------------------- consumers
// Per-lane constants of the B operands (lattice independent).
struct LaneTab {
  uint32_t selU;             // upper spins: F_reim
  uint32_t selL[2][6];       // lower spin 2 + s', position slot p = 2 kt + half
  int lbase;                 // word offset in link[]
  int cw[4];                 // clover: word offset of entry (jn, j') in block 0
  uint32_t csel[4], cmask[4];
};

__device__ __forceinline__ LaneTab lane_tables(int lane) {
  const int gq = lane >> 2, tq = lane & 3;
  const int reim = gq & 1, a = gq >> 1;  // column n = gq: colour a (3: padding), re / im
  LaneTab T;
  T.selU = kSel[(4 - reim) & 3];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int P = 8 * (p >> 1) + 4 * (p & 1) + tq;
    const int hop = P / 3, mu = hop >> 1, dir = hop & 1;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) T.selL[sp][p] = kSel[(kLowK[dir][sp][mu] - reim + 4) & 3];
  }
  T.lbase = tq * 4 + a;
  // clover entry Ahat[3 jn + a][3 j' + tq] of a packed Hermitian block (6 real diagonal
  // entries, then the 15 complex entries below the diagonal, row-major)
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int jn = e >> 1, jp = e & 1;
    int w = 0;
    uint32_t sel = 0x4444u, mask = 0u;  // zero entry (padding row or column)
    if (a < 3 && tq < 3) {
      const int i = 3 * jn + a, k = 3 * jp + tq;
      if (i == k) {
        const int rho = i;
        w = rho >> 1;
        const uint32_t d0 = (rho & 1) ? 2u : 0u;
        sel = reim == 0 ? (d0 | (d0 + 1) << 4 | 4u << 8 | 5u << 12) : (4u | 5u << 4 | d0 << 8 | (d0 + 1) << 12);
      } else if (i > k) {
        w = (6 + 2 * (i * (i - 1) / 2 + k)) >> 1;
        sel = reim == 0 ? 0x7610u : 0x1032u;
        mask = 0xffffffffu;
      } else {
        w = (6 + 2 * (k * (k - 1) / 2 + i)) >> 1;
        sel = reim == 0 ? 0x3210u : 0x1076u;  // conjugate of the stored entry
        mask = 0xffffffffu;
      }
    }
    T.cw[e] = w;
    T.csel[e] = sel;
    T.cmask[e] = mask;
  }
  return T;
}

// one site on one warp: 16 MMAs and the FP16 re-encoding of its outputs into the
// site's A area (row r at 64 bytes: 12 binary16 pairs, then the FP32 norm)
__device__ __forceinline__ void site_mma(Stage& S, int i, const LaneTab& T, int nrows) {
  const int lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  // ldmatrix row of this lane and its k half
  const int row = (lane & 7) + 8 * ((lane >> 3) & 1);
  const int hi = lane >> 4;
  const int swz = (row ^ i) & 7;
  float d[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int k = 0; k < 4; ++k) d[s][k] = 0.f;
  // k-tile kt: positions 8 kt .. 8 kt + 7 of both spin rows. Upper output spins 0, 1 take
  // the projected components as they are; lower spins 2 + s' take, for chunks 0..2 (x, y
  // hops), the other component and for chunks 3..5 (z, t) the same one, with the phases
  // in the link operand variants bl0 / bl1.
#pragma unroll
  for (int kt = 0; kt < 3; ++kt) {
    uint32_t a0[4], a1[4];
    ldsm_x4(a0, &S.A[i][0][row][(2 * kt + hi) ^ swz]);
    ldsm_x4(a1, &S.A[i][1][row][(2 * kt + hi) ^ swz]);
    uint32_t bu[2], bl0[2], bl1[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = 2 * kt + h;  // slot: position P = 8 kt + 4 h + tq
      const uint32_t w = S.link[i][16 * p + T.lbase];
      const uint32_t wn = w ^ 0x80008000u;
      bu[h] = prmt(w, wn, T.selU);
      bl0[h] = prmt(w, wn, T.selL[0][p]);
      bl1[h] = prmt(w, wn, T.selL[1][p]);
    }
    mma16816(d[0], a0, bu[0], bu[1]);
    mma16816(d[1], a1, bu[0], bu[1]);
    if (kt == 0) {
      mma16816(d[2], a1, bl0[0], bl0[1]);
      mma16816(d[3], a0, bl1[0], bl1[1]);
    } else if (kt == 1) {
      const uint32_t l0[4] = {a1[0], a1[1], a0[2], a0[3]};
      const uint32_t l1[4] = {a0[0], a0[1], a1[2], a1[3]};
      mma16816(d[2], l0, bl0[0], bl0[1]);
      mma16816(d[3], l1, bl1[0], bl1[1]);
    } else {
      mma16816(d[2], a0, bl0[0], bl0[1]);
      mma16816(d[3], a1, bl1[0], bl1[1]);
    }
  }
  // clover: chirality chi (block chi at word offset 18 chi), output spin 2 chi + jn
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    uint32_t ac[4];
    ldsm_x4(ac, &S.A[i][chi][row][(6 + hi) ^ swz]);
#pragma unroll
    for (int jn = 0; jn < 2; ++jn) {
      uint32_t b[2];
#pragma unroll
      for (int jp = 0; jp < 2; ++jp) {
        const int e = 2 * jn + jp;
        const uint32_t w = S.craw[i][18 * chi + T.cw[e]];
        b[jp] = prmt(w, (w ^ 0x80008000u) & T.cmask[e], T.csel[e]);
      }
      mma16816(d[2 * chi + jn], ac, b[0], b[1]);
    }
  }
  // outputs: lane holds, for rows gq and gq + 8, spin s colour tq (tq < 3): (re, im) =
  // (d[s][0], d[s][1]) and (d[s][2], d[s][3]); value = S_row * d
  float m0 = 0.f, m1 = 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    m0 = fmaxf(m0, fmaxf(fabsf(d[s][0]), fabsf(d[s][1])));
    m1 = fmaxf(m1, fmaxf(fabsf(d[s][2]), fabsf(d[s][3])));
  }
  m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
  m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
  m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
  m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
  const float i0 = m0 > 0.f ? 1.0f / m0 : 0.f;
  const float i1 = m1 > 0.f ? 1.0f / m1 : 0.f;
  __syncwarp();
  uint32_t* out = reinterpret_cast<uint32_t*>(&S.A[i][0][0][0]) + 4 * i;
  if (tq < 3) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (gq < nrows) out[gq * OUT_ROW_W + 3 * s + tq] = h2u(__floats2half2_rn(d[s][0] * i0, d[s][1] * i0));
      if (gq + 8 < nrows)
        out[(gq + 8) * OUT_ROW_W + 3 * s + tq] = h2u(__floats2half2_rn(d[s][2] * i1, d[s][3] * i1));
    }
  }
  if (tq == 0) {
    if (gq < nrows) reinterpret_cast<float*>(out)[gq * OUT_ROW_W + 12] = S.S[i][gq] * m0;
    if (gq + 8 < nrows) reinterpret_cast<float*>(out)[(gq + 8) * OUT_ROW_W + 12] = S.S[i][gq + 8] * m1;
  }
}

__device__ void consumer(Smem& sm, const TcLat* __restrict__ lats, int nlat, int ntiles) {
  const int lane = threadIdx.x & 31, cw = (threadIdx.x >> 5) - NPT / 32;  // consumer warp 0..3
  const int ctid = threadIdx.x - NPT;
  const LaneTab T = lane_tables(lane);
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it % NST;
    bar_sync(BAR_FULL + s, NT);
    Stage& S = sm.st[s];
    const TcLat& L = lats[lattice_of(lats, nlat, t)];
    const TileRef tr = tile_ref(L, t - L.tile_begin);
    const int Vh = L.g.Vh;
    for (int i = cw; i < TS; i += NCW)
      if (tr.cb0 + i < Vh) site_mma(S, i, T, tr.nrows);
    bar_sync(BAR_CONS, NT - NPT);
    // store: one thread per (site, rhs), consecutive sites in consecutive threads
    const size_t hb = (size_t)52 * Vh;
    for (int q = ctid; q < TS * tr.nrows; q += NT - NPT) {
      const int i = q & (TS - 1), r = q / TS;
      const int cb = tr.cb0 + i;
      if (cb >= Vh) continue;
      const uint4* o = reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(&S.A[i][0][0][0]) + 4 * i +
                                                      r * OUT_ROW_W);
      char* dst = L.out + (size_t)(tr.rg * ROWS + r) * L.field_bytes + (size_t)tr.par * hb;
#pragma unroll
      for (int k = 0; k < 3; ++k) *reinterpret_cast<uint4*>(dst + ((size_t)k * Vh + cb) * 16) = o[k];
      reinterpret_cast<float*>(dst + (size_t)48 * Vh)[cb] = reinterpret_cast<const float*>(o)[12];
    }
    bar_arrive(BAR_EMPTY + s, NT);
  }
}

template <int R>
__global__ void __launch_bounds__(NT, 2) mrhs_tc_kernel(const TcLat* __restrict__ lats, int nlat, int ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  if (threadIdx.x < NPT) producer<R>(sm, lats, nlat, ntiles);
  else consumer(sm, lats, nlat, ntiles);
}

}  // namespace tc

namespace tc {
// neighbour table: entry (par, hop, cb) = cb of the hop's target, bit 31 for the
// antiperiodic sign (fermion hops across the t edge)
__global__ void nbr_kernel(const Geom g, int* table) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * 8 * g.Vh) return;
  const int hop = k & 7, pc = k >> 3, cb = pc % g.Vh, par = pc / g.Vh;
  const int mu = hop >> 1, dir = hop & 1;
  int x[4];
  cb_coords(g, cb, par, x);
  bool neg = false;
  if (dir == 0) {
    if (++x[mu] == g.L[mu]) { x[mu] = 0; neg = (mu == 3 && g.apbc); }
  } else {
    if (x[mu]-- == 0) { x[mu] = g.L[mu] - 1; neg = (mu == 3 && g.apbc); }
  }
  table[k] = cb_index(g, x) | (neg ? (int)0x80000000 : 0);
}
}  // namespace tc

int tc_build_nbr(const Geom& g, int** table, cudaStream_t st) {
  *table = nullptr;
  const size_t n = (size_t)16 * g.Vh;
  if (cudaMalloc(table, n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return DIRAC_ERR_OOM;
  }
  tc::nbr_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, *table);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}

int tc_ctiles(int Vh) { return (Vh + tc::TS - 1) / tc::TS; }
int tc_tiles(const TcLat& L) { return 2 * tc_ctiles(L.g.Vh) * ((L.nrhs + tc::ROWS - 1) / tc::ROWS); }

static int tc_prepare(int recon) {
  static bool done[2] = {false, false};
  const int k = recon == 18 ? 1 : 0;
  if (!done[k]) {
    const int bytes = (int)sizeof(tc::Smem);
    cudaError_t e = recon == 18 ? cudaFuncSetAttribute(tc::mrhs_tc_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                                : cudaFuncSetAttribute(tc::mrhs_tc_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return -1;
    done[k] = true;
  }
  return 0;
}

int tc_ctas_per_sm(int recon) {
  if (tc_prepare(recon)) return 1;
  int n = 0;
  const size_t bytes = sizeof(tc::Smem);
  if (recon == 18) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tc::mrhs_tc_kernel<18>, tc::NT, bytes);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tc::mrhs_tc_kernel<12>, tc::NT, bytes);
  return n > 0 ? n : 1;
}

void launch_mrhs_tc(int recon, const TcLat* d_lats, int nlat, int ntiles, int grid, cudaStream_t st) {
  if (tc_prepare(recon)) return;
  const size_t bytes = sizeof(tc::Smem);
  if (recon == 18) tc::mrhs_tc_kernel<18><<<grid, tc::NT, bytes, st>>>(d_lats, nlat, ntiles);
  else tc::mrhs_tc_kernel<12><<<grid, tc::NT, bytes, st>>>(d_lats, nlat, ntiles);
}

}  // namespace dirac
