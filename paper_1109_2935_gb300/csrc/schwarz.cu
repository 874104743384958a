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
// FP32/FP16 storage: the block's residual r, its 4*|B| forward links (decoded to
// 18 FP32 reals) and its clover blocks are staged in shared memory; x and p live in
// registers; reductions are warp shuffles plus one shared-memory stage.
// FP64 storage: r is staged in shared memory, links and clover are read through
// the read-only cache.
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

// Shared-memory layout (floats, FP32 compute): r[24][nbs] | links[4][18][nbs] | clov[72][nbs]
template <int PREC, int R>
__global__ void __launch_bounds__(kMaxBlockSites) schwarz_kernel(const SchwarzArg a) {
  using T = typename Real<PREC>::T;
  constexpr bool STAGE = PREC != P64;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* r_s = reinterpret_cast<T*>(smem_raw);
  const int nbs = a.b[0] * a.b[1] * a.b[2] * a.b[3];
  float* l_s = reinterpret_cast<float*>(smem_raw + sizeof(T) * 24 * nbs);
  float* c_s = l_s + 4 * 18 * nbs;
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

  // stage r = b, the forward links and the clover
  T xs[24];
  if (active) {
    T v[24];
    SpinorIO<PREC, 24>::load(a.in + par * hb, Vh, cb, v);
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      r_s[k * nbs + t] = v[k];
      xs[k] = 0;
    }
    if constexpr (STAGE) {
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        Link<T> U;
        LinkIO<PREC, R>::load(a.gauge, Vh, mu, par, cb, U);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            l_s[(mu * 18 + 6 * i + 2 * j) * nbs + t] = U.m[i][j].r;
            l_s[(mu * 18 + 6 * i + 2 * j + 1) * nbs + t] = U.m[i][j].i;
          }
      }
      float cv[72];
      CloverIO<PREC>::load(a.clover + par * CloverIO<PREC>::parity_bytes(Vh), Vh, cb, cv);
#pragma unroll
      for (int k = 0; k < 72; ++k) c_s[k * nbs + t] = cv[k];
    }
  }
  __syncthreads();

  const T mk = -(T)a.kappa;
  for (int step = 0; step < a.steps; ++step) {
    T p[24];
    T red3[3] = {0, 0, 0};
    if (active) {
      // p = Ahat r - kappa D_B r on this site
      C<T> acc[4][3];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[s][c] = C<T>{0, 0};
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
          int ln = l[mu] + (dir == 0 ? 1 : -1);
          T bc = 1;
          if (ln == a.b[mu] || ln < 0) {
            if (a.b[mu] != g.L[mu]) continue;  // Dirichlet: hop leaves the block
            ln = dir == 0 ? 0 : a.b[mu] - 1;
            if (mu == 3 && g.apbc) bc = -1;
          }
          int lt = t;
          {  // local index of the neighbour
            int stride = 1;
            for (int nu = 0; nu < mu; ++nu) stride *= a.b[nu];
            lt = t + (ln - l[mu]) * stride;
          }
          T psi[24];
#pragma unroll
          for (int k = 0; k < 24; ++k) psi[k] = r_s[k * nbs + lt];
          Link<T> U;
          const int ls = dir == 0 ? t : lt;  // forward: own link; backward: neighbour's
          if constexpr (STAGE) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int j = 0; j < 3; ++j)
                U.m[i][j] = C<T>{l_s[(mu * 18 + 6 * i + 2 * j) * nbs + ls],
                                 l_s[(mu * 18 + 6 * i + 2 * j + 1) * nbs + ls]};
          } else {
            int y[4] = {x[0], x[1], x[2], x[3]};
            y[mu] = bo[mu] + ln;
            if (dir == 0) LinkIO<PREC, R>::load(a.gauge, Vh, mu, par, cb, U);
            else LinkIO<PREC, R>::load(a.gauge, Vh, mu, 1 - par, cb_index(g, y), U);
          }
          const T s = dir == 0 ? (T)-1 : (T)1;
          const bool dag = dir == 1;
          if (mu == 0) wilson_hop<0>(acc, psi, U, dag, s, bc);
          if (mu == 1) wilson_hop<1>(acc, psi, U, dag, s, bc);
          if (mu == 2) wilson_hop<2>(acc, psi, U, dag, s, bc);
          if (mu == 3) wilson_hop<3>(acc, psi, U, dag, s, bc);
        }
      }
      C<T> rv[12], av[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) rv[k] = C<T>{r_s[(2 * k) * nbs + t], r_s[(2 * k + 1) * nbs + t]};
      if constexpr (STAGE) {
        T cl[72];
#pragma unroll
        for (int k = 0; k < 72; ++k) cl[k] = c_s[k * nbs + t];
        herm6_mv<T>(cl, rv, av);
        herm6_mv<T>(cl + 36, rv + 6, av + 6);
      } else {
        apply_clover_site<PREC, T>(a.clover + par * CloverIO<PREC>::parity_bytes(Vh), Vh, cb, rv, av);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          p[6 * s + 2 * c] = fma(mk, acc[s][c].r, av[3 * s + c].r);
          p[6 * s + 2 * c + 1] = fma(mk, acc[s][c].i, av[3 * s + c].i);
        }
      // (p, r) and (p, p)
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        T pr = p[2 * k], pi = p[2 * k + 1];
        red3[0] = fma(pr, rv[k].r, red3[0]); red3[0] = fma(pi, rv[k].i, red3[0]);
        red3[1] = fma(pr, rv[k].i, red3[1]); red3[1] = fma(-pi, rv[k].r, red3[1]);
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
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        T rr = r_s[(2 * k) * nbs + t], ri = r_s[(2 * k + 1) * nbs + t];
        xs[2 * k] += ar * rr - ai * ri;
        xs[2 * k + 1] += ar * ri + ai * rr;
        r_s[(2 * k) * nbs + t] = rr - (ar * p[2 * k] - ai * p[2 * k + 1]);
        r_s[(2 * k + 1) * nbs + t] = ri - (ar * p[2 * k + 1] + ai * p[2 * k]);
      }
    }
    __syncthreads();
  }
  if (active) SpinorIO<PREC, 24>::store(a.out + par * hb, Vh, cb, xs);
}

template <int PREC>
static int schwarz_prec(int recon, const SchwarzArg& a, int nblocks, int nbs, cudaStream_t st) {
  size_t smem = sizeof(typename Real<PREC>::T) * 24 * nbs;
  if (PREC != P64) smem += sizeof(float) * (4 * 18 + 72) * nbs;
  int threads = ((nbs + 31) / 32) * 32;
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<nblocks, threads, smem, st>>>(a);
  };
  if (recon == 18) launch(schwarz_kernel<PREC, 18>);
  else if (recon == 12) launch(schwarz_kernel<PREC, 12>);
  else launch(schwarz_kernel<PREC, 8>);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
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
