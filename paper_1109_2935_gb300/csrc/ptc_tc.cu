// Tensor-core (tcgen05) form of a PTC layer for inference: BF16 operands, FP32
// accumulation in tensor memory.
//
// The spin mixing of a layer, out_c(x)[s][a] = sum_p sum_c' sum_t W[p][c][c'][s][t]
// (T_p in_c')(x)[t][a], is a dense contraction whose weights are the same at every site.
// For a tile of 128 sites and one colour a it is the real GEMM
//   D[m][n] = sum_p sum_k X_p[m][k] B_p[k][n],  m = site, per path p:
//   X_p[m] = [Re (T_p in)(x_m)[c'][t][a] | Im ...]                       K = 2 KH
//   B_p    = [[Re W, Im W], [-Im W, Re W]] over (c', t) x (c, s)          N = 2 NH
// with KH = max(8, 4 c_in), NH = max(8, 4 c_out) (zero padding). One CTA of 128 threads
// owns a tile: one thread per site and input channel computes the 8 parallel transports
// of that spinor (FP32 CUDA cores), writes its columns of X_p (three colours) into shared memory in the canonical K-major
// layout without swizzle (8x8 core matrices of 128 B; LBO 128 B along K, SBO 16 KC B
// along the rows); a fifth warp issues tcgen05.mma for the three colours (accumulators
// in 3 x N TMEM columns) as soon as a stage is full. Producers and the MMA warp meet
// only at mbarriers (a ring of X_p stages, double-buffered accumulators), so the loads
// and transports of later paths overlap the MMAs of earlier ones. After the 9 paths each
// producer warp reads its 32 lanes (= sites) back with tcgen05.ld. B for all paths is
// copied to shared memory once per CTA by a bulk asynchronous copy (cp.async.bulk).
// Every wait has a time budget (the global timer); on expiry the kernel records an error
// in a host-mapped flag, stops issuing, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace dirac {
namespace {

constexpr int NPATH_TC = 9;
constexpr int TC_M = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (row) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M = 128.
template <int N>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity));
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// true when the phase completed, false when the wait gave up after limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <>
__device__ __forceinline__ void tmem_ld<4>(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

template <int CIN, int COUT>
struct TcShape {
  static constexpr int KH = CIN * 4 < 8 ? 8 : CIN * 4;
  static constexpr int KC = 2 * KH;                   // K per path (16 or 32)
  static constexpr int NH = COUT * 4 < 8 ? 8 : COUT * 4;
  static constexpr int N = 2 * NH;                    // 16 or 32
  static constexpr int A_BYTES = TC_M * KC * 2;       // one colour, one path
  static constexpr int B_BYTES = N * KC * 2;          // one path
};

// byte offset of element (row, k) in a K-major no-swizzle tile with KC columns
__host__ __device__ __forceinline__ int canon_off(int row, int k, int kc) {
  return (row >> 3) * (kc * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Weight image: B_p for all paths in the shared-memory layout, from FP32 weights
// w[p][c][c'][s][t] (complex).
template <int CIN, int COUT>
__global__ void ptc_tc_pack_weights(const float2* w, __nv_bfloat16* img) {
  using S = TcShape<CIN, COUT>;
  const int total = NPATH_TC * S::N * S::KC;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int k = i % S::KC, n = (i / S::KC) % S::N, p = i / (S::KC * S::N);
  const bool kim = k >= S::KH, nim = n >= S::NH;
  const int j = kim ? k - S::KH : k, o = nim ? n - S::NH : n;
  float v = 0.f;
  if (j < 4 * CIN && o < 4 * COUT) {
    const int ci = j >> 2, t = j & 3, co = o >> 2, s = o & 3;
    const float2 q = w[((p * COUT + co) * CIN + ci) * 16 + 4 * s + t];
    v = !nim ? (!kim ? q.x : -q.y) : (!kim ? q.y : q.x);
  }
  img[(size_t)p * (S::B_BYTES / 2) + canon_off(n, k, S::KC) / 2] = __float2bfloat16_rn(v);
}

struct TcArg {
  uint64_t wait_ns;    // budget of every wait (a pipeline step takes microseconds)
  int stall;           // failure tests only: the MMA warp stops after loading the weights
  const char* in[4];   // input channels (FP32 full fields)
  char* out[4];        // output channels
  const char* gauge;   // FP32 links
  const __nv_bfloat16* wimg;
  Geom g;
  int ntiles;
  int* err;            // host-mapped error flag
};

// Neighbour of path p >= 1 with selects only (a runtime index into a local array or
// the geometry would go through local memory): checkerboard index of the neighbour,
// the link, whether it is applied as U^dagger, and the boundary sign.
template <int R>
__device__ __forceinline__ void tc_path_site(const Geom& g, const char* gauge, int p, const int x[4], int par,
                                             int cb, int& ycb, Link<float>& U, bool& dag, float& sgn) {
  const int mu = (p - 1) >> 1;
  dag = ((p - 1) & 1) != 0;
  const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
  const int xm = mu == 0 ? x[0] : mu == 1 ? x[1] : mu == 2 ? x[2] : x[3];
  int ym;
  bool wrap;
  if (!dag) {
    wrap = xm + 1 == L;
    ym = wrap ? 0 : xm + 1;
  } else {
    wrap = xm == 0;
    ym = wrap ? L - 1 : xm - 1;
  }
  sgn = (wrap && mu == 3 && g.apbc) ? -1.f : 1.f;
  const int y[4] = {mu == 0 ? ym : x[0], mu == 1 ? ym : x[1], mu == 2 ? ym : x[2], mu == 3 ? ym : x[3]};
  ycb = cb_index(g, y);
  if (!dag) LinkIO<P32, R>::load(gauge, g.Vh, mu, par, cb, U);
  else LinkIO<P32, R>::load(gauge, g.Vh, mu, 1 - par, ycb, U);
}

// Where path p >= 1 reads: the neighbour's checkerboard index and parity, the link's
// plane and index in it, U or U^dagger, and the boundary sign (selects only).
template <int R>
__device__ __forceinline__ void tc_path_geom(const Geom& g, const char* gauge, int p, const int x[4], int par, int cb,
                                             int& ycb, const char*& lplane, int& lidx, bool& dag, float& sgn) {
  const int mu = (p - 1) >> 1;
  dag = ((p - 1) & 1) != 0;
  const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
  const int xm = mu == 0 ? x[0] : mu == 1 ? x[1] : mu == 2 ? x[2] : x[3];
  const bool wrap = dag ? xm == 0 : xm + 1 == L;
  const int ym = dag ? (wrap ? L - 1 : xm - 1) : (wrap ? 0 : xm + 1);
  sgn = (wrap && mu == 3 && g.apbc) ? -1.f : 1.f;
  const int y[4] = {mu == 0 ? ym : x[0], mu == 1 ? ym : x[1], mu == 2 ? ym : x[2], mu == 3 ? ym : x[3]};
  ycb = cb_index(g, y);
  const int lpar = dag ? 1 - par : par;
  lplane = gauge + (size_t)(mu * 2 + lpar) * link_plane_bytes(R, 4, g.Vh);
  lidx = dag ? ycb : cb;
}

template <int B>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src) {
  if constexpr (B == 16) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
  else if constexpr (B == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src));
}

// Per-path prefetch buffer: every producer thread's neighbour spinor ([chunk][thread],
// 16 B chunks), then the link of each site ([chunk][site], fetched by the site's first
// thread); two of them alternate between paths.
template <int CIN, int R>
struct TcPrefetch {
  using LIO = LinkIO<P32, R>;
  static constexpr int SP_BYTES = CIN * 6 * TC_M * 16;
  static constexpr int BUF = SP_BYTES + LIO::kChunks * TC_M * LIO::kChunkBytes;
  static constexpr int BYTES = 2 * BUF;
};

template <int CIN, int R>
__device__ __forceinline__ void tc_prefetch(uint8_t* buf, const char* const* in, size_t hb, int Vh, int ycb, int ypar,
                                            const char* lplane, int lidx, bool link, int q, int m) {
  using PF = TcPrefetch<CIN, R>;
  constexpr int TPS = CIN == 4 ? 4 : 1, CPT = CIN / TPS, NT = TC_M * TPS;
  const uint32_t b = smem_u32(buf);
#pragma unroll
  for (int cc = 0; cc < CPT; ++cc) {
    const char* src = in[cc] + (size_t)ypar * hb;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      cp_async<16>(b + ((cc * 6 + k) * NT + q) * 16, src + ((size_t)k * Vh + ycb) * 16);
  }
  if (link) {
#pragma unroll
    for (int k = 0; k < PF::LIO::kChunks; ++k)
      cp_async<PF::LIO::kChunkBytes>(b + PF::SP_BYTES + (k * TC_M + m) * PF::LIO::kChunkBytes,
                                     lplane + ((size_t)k * Vh + lidx) * PF::LIO::kChunkBytes);
  }
}

// Warp-specialised pipeline: producer warps (TPS threads per site, each transporting CPT
// input channels and writing their X_p columns), then one warp that issues the MMAs.
// A ring of STAGES X_p buffers: full[s] completes when every producer warp wrote stage s,
// empty[s] when the MMAs that read it finished (tcgen05.commit). The tile's accumulators
// are double buffered in tensor memory: accf[b] completes when the MMAs of a tile
// finished, acce[b] when every producer warp read its results out.
template <int CIN>
struct TcWarps {
  // threads per site: one per input channel for c_in = 4 (measured faster); otherwise one
  // thread does all channels of its site (the link and geometry work is per thread)
  static constexpr int TPS = CIN == 4 ? 4 : 1;
  static constexpr int CPT = CIN / TPS;  // channels per thread
  static constexpr int PROD = 4 * TPS;
  static constexpr int THREADS = 32 * (PROD + 1);
};
constexpr int TC_STAGES = 3;

template <int CIN, int COUT>
struct TcPipe {
  using S = TcShape<CIN, COUT>;
  static constexpr int STAGE_BYTES = 3 * S::A_BYTES;
  static constexpr int SMEM = NPATH_TC * S::B_BYTES + TC_STAGES * STAGE_BYTES;
  static constexpr int ACC_COLS = 3 * S::N;                          // one tile, three colours
  static constexpr int TMEM = 2 * ACC_COLS <= 128 ? 128 : 256;       // two accumulator buffers
};

template <int CIN, int COUT, int R>
__global__ void __launch_bounds__(TcWarps<CIN>::THREADS, 1) ptc_tc_layer_kernel(const TcArg a) {
  using S = TcShape<CIN, COUT>;
  using PP = TcPipe<CIN, COUT>;
  using PF = TcPrefetch<CIN, R>;
  constexpr int PROD = TcWarps<CIN>::PROD, THREADS = TcWarps<CIN>::THREADS;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], accf[2], acce[2], wbar, dbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  uint8_t* Bs = smem;
  uint8_t* As = smem + NPATH_TC * S::B_BYTES;
  uint8_t* Ps = As + TC_STAGES * PP::STAGE_BYTES;  // two per-path prefetch buffers
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const size_t hb = (size_t)96 * Vh;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(PP::TMEM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_s = 0;
    for (int i = 0; i < TC_STAGES; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(PROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&accf[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[i])), "r"(PROD));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&wbar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&dbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // zero the X buffers once: padding columns (c_in = 1) are never written again and
  // must be finite (they meet zero rows of B)
  for (int i = tid; i < TC_STAGES * PP::STAGE_BYTES / 16; i += THREADS)
    reinterpret_cast<uint4*>(As)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_s;

  if (warp < PROD) {
    // ---------------------------------------------------------------- producers
    constexpr int TPS = TcWarps<CIN>::TPS, CPT = TcWarps<CIN>::CPT;
    const int q = tid, m = q / TPS, cg = q % TPS;  // site row of the tile, channel group
    const char* inp[CPT];  // this thread's input channels cg * CPT + cc
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      inp[cc] = a.in[cc];
#pragma unroll
      for (int c = 1; c < TPS; ++c)
        if (cg == c) inp[cc] = a.in[c * CPT + cc];
    }
    uint32_t it = 0, tcount = 0;
    // abort decisions are warp-uniform (votes): the warp-wide tcgen05.ld and __syncwarp
    // below need every lane
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++tcount) {
      if (__any_sync(0xffffffffu, abort_s != 0)) break;
      const int idx = tile * TC_M + m;
      const bool active = idx < 2 * Vh;
      const int par = active && idx >= Vh ? 1 : 0, cb = active ? idx - par * Vh : 0;
      int x[4] = {0, 0, 0, 0};
      if (active) cb_coords(g, cb, par, x);
      // path 0 (the site itself) goes to prefetch buffer 0; path p + 1 is requested
      // while path p is computed
      if (active) tc_prefetch<CIN, R>(Ps, inp, hb, Vh, cb, par, nullptr, 0, false, q, m);
      asm volatile("cp.async.commit_group;");
      bool dag_c = false, dag_n = false;
      float sgn_c = 1.f, sgn_n = 1.f;
#pragma unroll 1
      for (int p = 0; p < NPATH_TC; ++p, ++it) {
        if (p + 1 < NPATH_TC) {
          if (active) {
            int ycb;
            const char* lplane;
            int lidx;
            tc_path_geom<R>(g, a.gauge, p + 1, x, par, cb, ycb, lplane, lidx, dag_n, sgn_n);
            tc_prefetch<CIN, R>(Ps + ((p + 1) & 1) * PF::BUF, inp, hb, Vh, ycb, 1 - par, lplane, lidx, cg == 0, q, m);
          }
          asm volatile("cp.async.commit_group;");
          asm volatile("cp.async.wait_group 1;");
        } else {
          asm volatile("cp.async.wait_group 0;");
        }
        __syncwarp();  // the site's link, fetched by its first thread, is visible to the others
        const uint32_t st = it % TC_STAGES, ph = (it / TC_STAGES) & 1u;
        const bool late = !mbar_wait(&empty[st], ph ^ 1u, a.wait_ns);
        if (__any_sync(0xffffffffu, late || abort_s != 0)) {
          abort_s = 1;
          asm volatile("cp.async.wait_group 0;");
          break;
        }
        C<float> t[CPT][12];
        if (active) {
          const char* buf = reinterpret_cast<const char*>(Ps + (p & 1) * PF::BUF);
          Link<float> U;
          if (p > 0) LinkIO<P32, R>::template load_plane<false>(buf + PF::SP_BYTES, TC_M, m, U);
#pragma unroll
          for (int cc = 0; cc < CPT; ++cc) {
            float v[24];
            SpinorIO<P32, 24>::template load<false>(buf + cc * 6 * TC_M * TPS * 16, TC_M * TPS, q, v);
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) {
              C<float> f[3];
              f[0] = C<float>{v[6 * s2], v[6 * s2 + 1]};
              f[1] = C<float>{v[6 * s2 + 2], v[6 * s2 + 3]};
              f[2] = C<float>{v[6 * s2 + 4], v[6 * s2 + 5]};
              if (p > 0) {
                C<float> w3[3];
                if (dag_c) su3_mv_dag(U, f, w3);
                else su3_mv(U, f, w3);
#pragma unroll
                for (int c = 0; c < 3; ++c) t[cc][3 * s2 + c] = sgn_c * w3[c];
              } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) t[cc][3 * s2 + c] = f[c];
              }
            }
          }
        } else {
#pragma unroll
          for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
            for (int k = 0; k < 12; ++k) t[cc][k] = C<float>{0.f, 0.f};
        }
        dag_c = dag_n;
        sgn_c = sgn_n;
        // this thread's columns of row m of X_p (three colours): the 4 spins of each of
        // its channels ci, real part at K = 4 ci, imaginary part at KH + 4 ci
        uint8_t* stage = As + (size_t)st * PP::STAGE_BYTES;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          uint8_t* A = stage + (size_t)c * S::A_BYTES;
#pragma unroll
          for (int cc = 0; cc < CPT; ++cc) {
            const int ci = cg * CPT + cc;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float qv[4];
#pragma unroll
              for (int t4 = 0; t4 < 4; ++t4) qv[t4] = h ? t[cc][3 * t4 + c].i : t[cc][3 * t4 + c].r;
              const __nv_bfloat162 lo = __floats2bfloat162_rn(qv[0], qv[1]);
              const __nv_bfloat162 hi = __floats2bfloat162_rn(qv[2], qv[3]);
              *reinterpret_cast<uint2*>(A + canon_off(m, h * S::KH + 4 * ci, S::KC)) =
                  make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[st])));
      }
      if (__any_sync(0xffffffffu, abort_s != 0)) break;
      // the tile's results: warp w reads lane quarter w % 4 (sites 32 (w % 4) + lane) and
      // stores the output channels co = w / 4 (mod TPS)
      const uint32_t b = tcount & 1u, pb = (tcount >> 1) & 1u;
      const bool late = !mbar_wait(&accf[b], pb, a.wait_ns);
      if (__any_sync(0xffffffffu, late || abort_s != 0)) {
        abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int quarter = warp & 3, grp = warp >> 2;
      const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + b * PP::ACC_COLS;
      const int oidx = tile * TC_M + quarter * 32 + lane;
      const bool oact = oidx < 2 * Vh;
      const int opar = oact && oidx >= Vh ? 1 : 0, ocb = oact ? oidx - opar * Vh : 0;
      if constexpr (S::N == 16) {
        // all 16 columns of each colour at once (48 registers)
        float d[3][16];
#pragma unroll
        for (int c = 0; c < 3; ++c) tmem_ld<16>(base + c * S::N, d[c]);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        // the accumulator is free as soon as it is in registers
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])));
        if (oact) {
#pragma unroll
          for (int co = 0; co < COUT; ++co) {
            if (co % TPS != grp) continue;
            float o[24];
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                o[6 * s2 + 2 * c] = d[c][co * 4 + s2];
                o[6 * s2 + 2 * c + 1] = d[c][S::NH + co * 4 + s2];
              }
            SpinorIO<P32, 24>::store(a.out[co] + opar * hb, Vh, ocb, o);
          }
        }
      } else {
        // per output channel: 4 real and 4 imaginary columns of each colour
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
          if (co % TPS != grp) continue;  // warp-uniform
          float re[3][4], im[3][4];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            tmem_ld<4>(base + c * S::N + co * 4, re[c]);
            tmem_ld<4>(base + c * S::N + S::NH + co * 4, im[c]);
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          if (oact) {
            float o[24];
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                o[6 * s2 + 2 * c] = re[c][s2];
                o[6 * s2 + 2 * c + 1] = im[c][s2];
              }
            SpinorIO<P32, 24>::store(a.out[co] + opar * hb, Vh, ocb, o);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[b])));
      }
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    {
      const uint32_t bytes = NPATH_TC * S::B_BYTES;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&wbar)), "r"(bytes));
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(Bs)),
                   "l"(a.wimg), "r"(bytes), "r"(smem_u32(&wbar)));
      if (!mbar_wait(&wbar, 0, a.wait_ns)) abort_s = 1;
    }
    constexpr uint32_t IDESC = instr_desc<S::N>();
    uint32_t it = 0, tcount = 0;
    // a.stall: this warp issues nothing, as if it had died; the producers' waits run out
    for (int tile = blockIdx.x; tile < a.ntiles && !abort_s && !a.stall; tile += gridDim.x, ++tcount) {
      const uint32_t b = tcount & 1u, pb = (tcount >> 1) & 1u;
      if (!mbar_wait(&acce[b], pb ^ 1u, a.wait_ns)) { abort_s = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t dcol = tmem + b * PP::ACC_COLS;
      for (int p = 0; p < NPATH_TC; ++p, ++it) {
        const uint32_t st = it % TC_STAGES, ph = (it / TC_STAGES) & 1u;
        if (!mbar_wait(&full[st], ph, a.wait_ns)) { abort_s = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sbase = smem_u32(As + (size_t)st * PP::STAGE_BYTES);
        const uint32_t bbase = smem_u32(Bs + (size_t)p * S::B_BYTES);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int ks = 0; ks < S::KC / 16; ++ks) {
            const uint64_t da = smem_desc(sbase + c * S::A_BYTES + ks * 256, 128, S::KC * 16);
            const uint64_t db = smem_desc(bbase + ks * 256, 128, S::KC * 16);
            mma_bf16(dcol + c * S::N, da, db, IDESC, (p > 0 || ks > 0) ? 1u : 0u);
          }
        mma_commit(&empty[st]);
      }
      if (abort_s) break;
      mma_commit(&accf[b]);
    }
    // every MMA issued here has finished before the tensor memory is freed
    mma_commit(&dbar);
    if (!mbar_wait(&dbar, 0, a.wait_ns)) abort_s = 1;
  }
  if (abort_s && tid == 0) *(volatile int*)a.err = 1;
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PP::TMEM));
}

template <int CIN, int COUT, int R>
int launch_tc(const TcArg& a, cudaStream_t st) {
  using PP = TcPipe<CIN, COUT>;
  constexpr int SMEM = PP::SMEM + TcPrefetch<CIN, R>::BYTES;
  // once per instantiation: the shared-memory opt-in and the persistent grid (resident
  // CTAs per SM, capped so that every CTA gets its tensor memory)
  static int resident = 0;
  if (!resident) {
    if (cudaFuncSetAttribute(ptc_tc_layer_kernel<CIN, COUT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM) != cudaSuccess)
      return DIRAC_ERR_CUDA;
    int dev = 0, sms = 0, smem_sm = 0;
    cudaFuncAttributes fa{};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaFuncGetAttributes(&fa, ptc_tc_layer_kernel<CIN, COUT, R>);
    // resident CTAs per SM from tensor memory (512 columns), shared memory (1 KB reserved
    // per CTA) and registers (allocated per warp in units of 256)
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int per_sm = 512 / PP::TMEM;
    per_sm = std::min(per_sm, smem_sm / (int)(SMEM + fa.sharedSizeBytes + 1024));
    per_sm = std::min(per_sm, 65536 / (regs_warp * (TcWarps<CIN>::THREADS / 32)));
    resident = sms * std::max(per_sm, 1);
  }
  int grid = resident;
  if (grid > a.ntiles) grid = a.ntiles;
  ptc_tc_layer_kernel<CIN, COUT, R><<<grid, TcWarps<CIN>::THREADS, SMEM, st>>>(a);
  return DIRAC_OK;
}

template <int CIN, int COUT>
int tc_r(int recon, const TcArg& a, cudaStream_t st) {
  if (recon == 18) return launch_tc<CIN, COUT, 18>(a, st);
  if (recon == 12) return launch_tc<CIN, COUT, 12>(a, st);
  return launch_tc<CIN, COUT, 8>(a, st);
}

template <int CIN>
int tc_co(int cout, int recon, const TcArg& a, cudaStream_t st) {
  if (cout == 1) return tc_r<CIN, 1>(recon, a, st);
  if (cout == 2) return tc_r<CIN, 2>(recon, a, st);
  return tc_r<CIN, 4>(recon, a, st);
}

template <int CIN, int COUT>
void pack_w(const float2* w, __nv_bfloat16* img, cudaStream_t st) {
  using S = TcShape<CIN, COUT>;
  const int total = NPATH_TC * S::N * S::KC;
  ptc_tc_pack_weights<CIN, COUT><<<(total + 255) / 256, 256, 0, st>>>(w, img);
}

template <int CIN>
void pack_co(int cout, const float2* w, __nv_bfloat16* img, cudaStream_t st) {
  if (cout == 1) pack_w<CIN, 1>(w, img, st);
  else if (cout == 2) pack_w<CIN, 2>(w, img, st);
  else pack_w<CIN, 4>(w, img, st);
}

}  // namespace

size_t ptc_tc_image_bytes(int cin, int cout) {
  const int kh = cin * 4 < 8 ? 8 : cin * 4, nh = cout * 4 < 8 ? 8 : cout * 4;
  return (size_t)NPATH_TC * (2 * nh) * (2 * kh) * 2;
}

void ptc_tc_pack(int cin, int cout, const float2* w, void* img, cudaStream_t st) {
  __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(img);
  if (cin == 1) pack_co<1>(cout, w, p, st);
  else if (cin == 2) pack_co<2>(cout, w, p, st);
  else pack_co<4>(cout, w, p, st);
}

int ptc_tc_layer(int cin, int cout, int recon, const char* const* in, char* const* out, const char* gauge,
                 const void* img, const Geom& g, int* err, uint64_t wait_ns, int stall, cudaStream_t st) {
  TcArg a{};
  a.wait_ns = wait_ns;
  a.stall = stall;
  for (int c = 0; c < cin; ++c) a.in[c] = in[c];
  for (int c = 0; c < cout; ++c) a.out[c] = out[c];
  a.gauge = gauge;
  a.wimg = reinterpret_cast<const __nv_bfloat16*>(img);
  a.g = g;
  a.ntiles = (2 * g.Vh + TC_M - 1) / TC_M;
  a.err = err;
  if (cin == 1) return tc_co<1>(cout, recon, a, st);
  if (cin == 2) return tc_co<2>(cout, recon, a, st);
  return tc_co<4>(cout, recon, a, st);
}

}  // namespace dirac
