// Non-overlapping additive Schwarz preconditioner (Sec. 3.2, Sec. 8.1): on every
// block B of the lattice the Wilson-clover operator restricted to B, with Dirichlet
// (zero) block boundaries, is solved approximately by n steps of minimal residual
// from x = 0:
//     p = M_B r;  alpha = (p, r) / (p, p);  x += alpha r;  r -= alpha p,
// with block-local inner products ("the reductions ... are restricted to that
// domain only", Sec. 8.1). Blocks are independent (block Jacobi), so one CTA owns
// one block: thread t owns site t of the block (x fastest). A hop is kept iff its
// wrapped target lies in the same block; a block spanning a whole lattice extent
// keeps that extent's periodic / antiperiodic wrap.
//
// FP32/FP16 storage: the block's forward links and clover are copied into shared
// memory in their storage format (raw chunks: binary16 stays binary16, so an FP16
// block needs 87 KB and two CTAs fit on an SM) and decoded on use; the clover's FP16
// per-site norm scales the 6-component input instead of the 36 entries. The hopping
// sum is accumulated unscaled and multiplied by -kappa once, only a wrapping t hop
// with antiperiodic time taking its sign. The residual r lives in shared memory in
// FP32, x in registers; reductions are warp shuffles plus one shared-memory stage.
// FP64 storage: r in shared memory, links and clover read through the read-only cache.
#include "internal.h"
#include "wilson.cuh"

namespace dirac {

static constexpr int kMaxBlockSites = 256;

struct SchwarzArg {
  char* out;
  const char* in;
  const char* gauge;
  const char* clover;
  Geom g;
  int b[4];        // block extents
  int nb[4];       // blocks per dimension
  int steps;
  double kappa;
};

template <int PREC, int R>
struct SchwarzLayout {
  using T = typename Real<PREC>::T;
  static constexpr bool kStage = PREC != P64;
  static constexpr int kLinkSite = kStage ? 4 * LinkIO<PREC, R>::kChunks * LinkIO<PREC, R>::kChunkBytes : 0;
  static constexpr int kClovSite = kStage ? (PREC == P32 ? 288 : 148) : 0;
  static constexpr int kRSite = 24 * (int)sizeof(T);
  static constexpr int kSite = kRSite + kLinkSite + kClovSite;  // bytes of smem per block site
  static constexpr int kMinBlocks = PREC == P16 ? 2 : 1;
};

template <typename T>
__device__ __forceinline__ void block_sum3(T v[3], T (*sh)[3], int nwarp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) sh[warp][k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T s = 0;
    for (int w = 0; w < nwarp; ++w) s += sh[w][k];
    v[k] = s;
  }
}

template <int CB>
__device__ __forceinline__ void copy_chunk(char* dst, const char* src) {
  if constexpr (CB == 16) *reinterpret_cast<int4*>(dst) = __ldg(reinterpret_cast<const int4*>(src));
  else if constexpr (CB == 8) *reinterpret_cast<int2*>(dst) = __ldg(reinterpret_cast<const int2*>(src));
  else *reinterpret_cast<int*>(dst) = __ldg(reinterpret_cast<const int*>(src));
}

// The 36 stored reals of chirality block `blk` of site i, without the FP16 per-site
// norm, which is returned instead (1 for FP32 / FP64): A_blk = n * v.
template <int PREC, bool NC, typename T>
__device__ __forceinline__ T clover_block_raw(const char* b, int stride, int i, int blk, T v[36]) {
  if constexpr (PREC == P16) {
    const float n = ld_chunk<float, NC>(b + (size_t)144 * stride + (size_t)i * 4);
    // the block's 36 halves are half2 words 2 blk .. 2 blk + 17 of chunks 4 blk .. 4 blk + 4
    // (block 1 starts 4 halves into chunk 4): only those 18 words are converted
    uint32_t w[20];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int4 q = ld_chunk<int4, NC>(b + ((size_t)(4 * blk + k) * stride + i) * 16);
      w[4 * k] = (uint32_t)q.x; w[4 * k + 1] = (uint32_t)q.y; w[4 * k + 2] = (uint32_t)q.z; w[4 * k + 3] = (uint32_t)q.w;
    }
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const uint32_t word = blk ? w[k + 2] : w[k];
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&word));
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
    return n;
  } else {
    clover_block<PREC, NC, T>(b, stride, i, blk, v);
    return (T)1;
  }
}

// The 12 reals of chirality half `blk` (spins 2 blk, 2 blk + 1) of site i of the
// residual in shared memory.
template <int RP, typename T>
__device__ __forceinline__ void r_chirality_half(const char* r_s, int nbs, int i, int blk, T v[12]) {
  if constexpr (RP == P64) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double2 q = *reinterpret_cast<const double2*>(r_s + ((size_t)(6 * blk + k) * nbs + i) * 16);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 q = *reinterpret_cast<const float4*>(r_s + ((size_t)(3 * blk + k) * nbs + i) * 16);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  }
}

// y += A x for one Hermitian 6x6 block (d[6], then 15 complex L_ij, i>j)
template <typename T>
__device__ __forceinline__ void herm6_mac(const T* blk, const C<T> x[6], C<T> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    y[i].r = fma(blk[i], x[i].r, y[i].r);
    y[i].i = fma(blk[i], x[i].i, y[i].i);
  }
  int o = 6;
#pragma unroll
  for (int i = 1; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) {
      C<T> l = {blk[o], blk[o + 1]};
      o += 2;
      cmac(y[i], l, x[j]);   // y_i += L_ij x_j
      cmacc(y[j], l, x[i]);  // y_j += conj(L_ij) x_i
    }
  }
}

template <int PREC, int R>
__global__ void __launch_bounds__(kMaxBlockSites, (SchwarzLayout<PREC, R>::kMinBlocks))
    schwarz_kernel(const SchwarzArg a) {
  using L = SchwarzLayout<PREC, R>;
  using T = typename L::T;
  using LIO = LinkIO<PREC, R>;
  constexpr int RP = PREC == P64 ? P64 : P32;  // precision of the residual in smem
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nbs = a.b[0] * a.b[1] * a.b[2] * a.b[3];
  char* r_s = reinterpret_cast<char*>(smem_raw);
  char* l_s = r_s + (size_t)L::kRSite * nbs;
  char* c_s = l_s + (size_t)L::kLinkSite * nbs;
  __shared__ T red[kMaxBlockSites / 32][3];
  const int nwarp = (nbs + 31) / 32;
  const Geom& g = a.g;
  const int Vh = g.Vh;

  // block origin and this thread's site
  int bi = blockIdx.x, bo[4];
  for (int mu = 0; mu < 4; ++mu) {
    bo[mu] = (bi % a.nb[mu]) * a.b[mu];
    bi /= a.nb[mu];
  }
  const int t = threadIdx.x;
  const bool active = t < nbs;
  int l[4] = {0, 0, 0, 0}, x[4];
  {
    int r = active ? t : 0;
    for (int mu = 0; mu < 4; ++mu) {
      l[mu] = r % a.b[mu];
      r /= a.b[mu];
      x[mu] = bo[mu] + l[mu];
    }
  }
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(g, x);
  const size_t hb = SpinorIO<PREC, 24>::half_bytes(Vh);
  const char* clov_g = a.clover + par * CloverIO<PREC>::parity_bytes(Vh);

  // neighbour local indices, -1 where the hop leaves the block, and the sign of the
  // two t hops (-1 for a wrapping hop with antiperiodic time)
  int nbr[8];
  T tsign[2] = {(T)1, (T)1};
  {
    int stride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
      for (int dir = 0; dir < 2; ++dir) {
        int ln = l[mu] + (dir == 0 ? 1 : -1);
        bool ok = true;
        if (ln == a.b[mu] || ln < 0) {
          if (a.b[mu] != g.L[mu]) ok = false;
          ln = dir == 0 ? 0 : a.b[mu] - 1;
          if (mu == 3 && g.apbc) tsign[dir] = (T)-1;
        }
        nbr[2 * mu + dir] = ok ? t + (ln - l[mu]) * stride : -1;
      }
      stride *= a.b[mu];
    }
  }

  // stage r = b, and (FP32/FP16) the forward links and clover in storage format
  T xs[24];
  if (active) {
    T v[24];
    SpinorIO<PREC, 24>::load(a.in + par * hb, Vh, cb, v);
    SpinorIO<RP, 24>::store(r_s, nbs, t, v);
#pragma unroll
    for (int k = 0; k < 24; ++k) xs[k] = 0;
    if constexpr (L::kStage) {
      constexpr int CB = LIO::kChunkBytes, NCH = LIO::kChunks;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const char* gp = a.gauge + (size_t)(mu * 2 + par) * link_plane_bytes(R, LIO::W, Vh);
        char* sp = l_s + (size_t)mu * NCH * CB * nbs;
#pragma unroll
        for (int k = 0; k < NCH; ++k)
          copy_chunk<CB>(sp + ((size_t)k * nbs + t) * CB, gp + ((size_t)k * Vh + cb) * CB);
      }
      constexpr int CCH = PREC == P32 ? 18 : 9;
#pragma unroll
      for (int k = 0; k < CCH; ++k)
        copy_chunk<16>(c_s + ((size_t)k * nbs + t) * 16, clov_g + ((size_t)k * Vh + cb) * 16);
      if constexpr (PREC == P16)
        reinterpret_cast<float*>(c_s + (size_t)144 * nbs)[t] =
            __ldg(reinterpret_cast<const float*>(clov_g + (size_t)144 * Vh) + cb);
    }
  }
  __syncthreads();

  const T mk = (T)(-a.kappa);
  for (int step = 0; step < a.steps; ++step) {
    T p[24];
    T red3[3] = {0, 0, 0};
    if (active) {
      // p = Ahat r - kappa D_B r on this site: the hopping sum first, unscaled
      C<T> acc[4][3];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = C<T>{0, 0};
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
          const int lt = nbr[2 * mu + dir];
          if (lt < 0) continue;  // Dirichlet: the hop leaves the block
          T psi[24];
          SpinorIO<RP, 24>::template load<false>(r_s, nbs, lt, psi);
          Link<T> U;
          const int ls = dir == 0 ? t : lt;  // forward: own link; backward: the neighbour's
          if constexpr (L::kStage) {
            LIO::template load_plane<false>(l_s + (size_t)mu * LIO::kChunks * LIO::kChunkBytes * nbs, nbs, ls, U);
          } else {
            if (dir == 0) {
              LIO::load(a.gauge, Vh, mu, par, cb, U);
            } else {
              int y[4] = {x[0], x[1], x[2], x[3]};
              int lb = l[mu] - 1;
              y[mu] = bo[mu] + (lb < 0 ? a.b[mu] - 1 : lb);
              LIO::load(a.gauge, Vh, mu, 1 - par, cb_index(g, y), U);
            }
          }
          const T s = dir == 0 ? (T)-1 : (T)1;
          if (mu == 0) wilson_hop<0>(acc, psi, U, dir == 1, s, (T)1);
          if (mu == 1) wilson_hop<1>(acc, psi, U, dir == 1, s, (T)1);
          if (mu == 2) wilson_hop<2>(acc, psi, U, dir == 1, s, (T)1);
          if (mu == 3) wilson_hop<3>(acc, psi, U, dir == 1, s, tsign[dir]);
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = C<T>{mk * acc[s][c].r, mk * acc[s][c].i};
      // + Ahat r, chirality block by block; the FP16 norm scales the 6-component input
#pragma unroll
      for (int blk = 0; blk < 2; ++blk) {
        T cl[36], rv[12];
        T n;
        if constexpr (L::kStage) n = clover_block_raw<PREC, false, T>((const char*)c_s, nbs, t, blk, cl);
        else n = clover_block_raw<PREC, true, T>(clov_g, Vh, cb, blk, cl);
        r_chirality_half<RP>(r_s, nbs, t, blk, rv);
        C<T> in6[6], out6[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          in6[k] = C<T>{n * rv[2 * k], n * rv[2 * k + 1]};
          out6[k] = acc[2 * blk + k / 3][k % 3];
        }
        herm6_mac<T>(cl, in6, out6);
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[2 * blk + k / 3][k % 3] = out6[k];
      }
      T rv[24];
      SpinorIO<RP, 24>::template load<false>(r_s, nbs, t, rv);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          p[6 * s + 2 * c] = acc[s][c].r;
          p[6 * s + 2 * c + 1] = acc[s][c].i;
        }
      // (p, r) and (p, p)
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        T pr = p[2 * k], pi = p[2 * k + 1], rr = rv[2 * k], ri = rv[2 * k + 1];
        red3[0] = fma(pr, rr, red3[0]); red3[0] = fma(pi, ri, red3[0]);
        red3[1] = fma(pr, ri, red3[1]); red3[1] = fma(-pi, rr, red3[1]);
        red3[2] = fma(pr, pr, red3[2]); red3[2] = fma(pi, pi, red3[2]);
      }
    }
    block_sum3<T>(red3, red, nwarp);  // also the barrier before r is overwritten
    T ar = 0, ai = 0;
    if (red3[2] > 0) {
      ar = red3[0] / red3[2];
      ai = red3[1] / red3[2];
    }
    if (active) {
      T rv[24];
      SpinorIO<RP, 24>::template load<false>(r_s, nbs, t, rv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        T rr = rv[2 * k], ri = rv[2 * k + 1];
        xs[2 * k] += ar * rr - ai * ri;
        xs[2 * k + 1] += ar * ri + ai * rr;
        rv[2 * k] = rr - (ar * p[2 * k] - ai * p[2 * k + 1]);
        rv[2 * k + 1] = ri - (ar * p[2 * k + 1] + ai * p[2 * k]);
      }
      SpinorIO<RP, 24>::store(r_s, nbs, t, rv);
    }
    __syncthreads();
  }
  if (active) SpinorIO<PREC, 24>::store(a.out + par * hb, Vh, cb, xs);
}

template <int PREC, int R>
static int schwarz_launch(const SchwarzArg& a, int nblocks, int nbs, cudaStream_t st) {
  using L = SchwarzLayout<PREC, R>;
  const size_t smem = (size_t)L::kSite * nbs;
  const int threads = ((nbs + 31) / 32) * 32;
  auto kern = schwarz_kernel<PREC, R>;
  static bool configured = false;  // the attribute is per kernel, set once
  if (!configured) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)L::kSite * kMaxBlockSites)) != cudaSuccess)
      return DIRAC_ERR_CUDA;
    configured = true;
  }
  kern<<<nblocks, threads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}

template <int PREC>
static int schwarz_prec(int recon, const SchwarzArg& a, int nblocks, int nbs, cudaStream_t st) {
  if (recon == 18) return schwarz_launch<PREC, 18>(a, nblocks, nbs, st);
  if (recon == 12) return schwarz_launch<PREC, 12>(a, nblocks, nbs, st);
  return schwarz_launch<PREC, 8>(a, nblocks, nbs, st);
}

int launch_schwarz(int prec, int recon, char* out, const char* in, const char* gauge,
                   const char* clover, const Geom& g, const int block[4], int mr_steps,
                   double kappa, cudaStream_t st) {
  SchwarzArg a;
  a.out = out; a.in = in; a.gauge = gauge; a.clover = clover; a.g = g;
  a.steps = mr_steps; a.kappa = kappa;
  int nblocks = 1, nbs = 1;
  for (int mu = 0; mu < 4; ++mu) {
    a.b[mu] = block[mu];
    a.nb[mu] = g.L[mu] / block[mu];
    nblocks *= a.nb[mu];
    nbs *= block[mu];
  }
  if (nbs > kMaxBlockSites) return DIRAC_ERR_ARG;
  if (prec == P64) return schwarz_prec<P64>(recon, a, nblocks, nbs, st);
  if (prec == P32) return schwarz_prec<P32>(recon, a, nblocks, nbs, st);
  return schwarz_prec<P16>(recon, a, nblocks, nbs, st);
}

}  // namespace dirac
