// Batched mixed-precision BiCGstab: many right-hand sides of several lattices (of any
// sizes) solved together, one Krylov iteration for all of them at a time.
//
// Each right-hand side runs its own BiCGstab (Sec. 3.1) with reliable updates (Sec. 8.2:
// the Krylov space and the operator in a sloppy precision, the solution and the true
// residual r = b - M x in FP64). What is shared is the work of one iteration: the two
// operator applications go to batched operator plans (dirac_batch_*, the CUDA-core
// kernel: it skips the systems that are no longer active), the BLAS
// updates and reductions of all right-hand sides are single launches over a segment
// table, and the scalar algebra is one thread per right-hand side. Scalars stay on the
// GPU; every iteration is replayed from a CUDA graph (two graphs: the iteration's
// launches depend only on the mirror slot). The host reads the per-right-hand-side
// residual norms one iteration behind from mapped memory (skipping, for a right-hand side
// just updated, the value of the iteration before its update) and decides reliable updates
// (taken together, in one set of launches, for the right-hand sides that ask; the others
// are masked out and keep iterating) and convergence; a converged right-hand side is
// frozen (masked out of the operator and BLAS launches, so x, the correction and the
// residual stay as they are) while the others continue. Nothing of one right-hand side's
// arithmetic depends on the others, so each returns the bytes, iterations and reliable
// updates of solve_batched on it alone.
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace dirac {
namespace bs {

constexpr int NT = 256;       // threads per BLAS block
constexpr int MAXBPR = 256;   // blocks per right-hand side
constexpr int MAXRHS = 256;   // right-hand sides per batched solve
constexpr int NSC = 32;       // doubles of scalar state per right-hand side
enum : int {
  SC_RHO = 0, SC_RHOOLD = 2, SC_ALPHA = 4, SC_OMEGA = 6, SC_SIGMA = 8, SC_TS = 10, SC_RN = 13,
  SC_BETA = 16, SC_NBW = 18, SC_NALPHA = 20, SC_NOMEGA = 22, SC_ACTIVE = 24, SC_FLAG = 25,
  SC_TMP = 26, SC_RR = 29, SC_BB = 30
};
enum : int { FL_OK = 0, FL_BREAKDOWN = 1, FL_NONFINITE = 2 };

// vectors of a segment (one lattice): nrhs consecutive full fields each
enum : int { VX = 0, VB, VR, VRS, VR0, VP, VV, VT, VXS, NVEC };

struct Seg {
  int Vh, nrhs, rhs0, blk0, bpr;
  char* f[NVEC];
  size_t fb[NVEC];   // bytes of one full field of the vector
};

// site s (0 .. 2 Vh - 1) of right-hand side r of vector v: half-field base and cb
__device__ __forceinline__ const char* site_base(const Seg& g, int v, int r, int s, int& cb) {
  const int q = s >= g.Vh ? 1 : 0;
  cb = s - q * g.Vh;
  return g.f[v] + (size_t)r * g.fb[v] + (size_t)q * (g.fb[v] / 2);
}
template <int PREC, typename T>
__device__ __forceinline__ void load_v(const Seg& g, int v, int r, int s, T out[24]) {
  int cb;
  const char* b = site_base(g, v, r, s, cb);
  typename Real<PREC>::T t[24];
  SpinorIO<PREC, 24>::template load<false>(b, g.Vh, cb, t);
#pragma unroll
  for (int k = 0; k < 24; ++k) out[k] = (T)t[k];
}
template <int PREC, typename T>
__device__ __forceinline__ void store_v(const Seg& g, int v, int r, int s, const T in[24]) {
  int cb;
  char* b = const_cast<char*>(site_base(g, v, r, s, cb));
  typename Real<PREC>::T t[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) t[k] = (typename Real<PREC>::T)in[k];
  SpinorIO<PREC, 24>::store(b, g.Vh, cb, t);
}

// ---------------------------------------------------------------- operations
// op(g, r, s, sc, acc): site s of local right-hand side r; sc = its scalar state
template <int SP> struct OpPUpd {  // p = rs + beta p + nbw v
  static constexpr int NRED = 0, OUT = 0;
  using T = typename Real<SP>::T;
  __device__ void operator()(const Seg& g, int r, int s, const double* sc, double*) const {
    const T br = (T)sc[SC_BETA], bi = (T)sc[SC_BETA + 1], cr = (T)sc[SC_NBW], ci = (T)sc[SC_NBW + 1];
    T u[24], v[24], p[24];
    load_v<SP>(g, VRS, r, s, u);
    load_v<SP>(g, VV, r, s, v);
    load_v<SP>(g, VP, r, s, p);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const T pr = p[2 * k], pi = p[2 * k + 1], vr = v[2 * k], vi = v[2 * k + 1];
      p[2 * k] = u[2 * k] + br * pr - bi * pi + cr * vr - ci * vi;
      p[2 * k + 1] = u[2 * k + 1] + br * pi + bi * pr + cr * vi + ci * vr;
    }
    store_v<SP>(g, VP, r, s, p);
  }
};
template <int SP, int VA, int VBB, int OUTSLOT> struct OpCdot {  // (a, b) = sum conj(a) b
  static constexpr int NRED = 2, OUT = OUTSLOT;
  using T = typename Real<SP>::T;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double* acc) const {
    T a[24], b[24];
    load_v<SP>(g, VA, r, s, a);
    load_v<SP>(g, VBB, r, s, b);
    T re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re += a[2 * k] * b[2 * k] + a[2 * k + 1] * b[2 * k + 1];
      im += a[2 * k] * b[2 * k + 1] - a[2 * k + 1] * b[2 * k];
    }
    acc[0] += re;
    acc[1] += im;
  }
};
template <int SP> struct OpSUpd {  // rs += nalpha v
  static constexpr int NRED = 0, OUT = 0;
  using T = typename Real<SP>::T;
  __device__ void operator()(const Seg& g, int r, int s, const double* sc, double*) const {
    const T ar = (T)sc[SC_NALPHA], ai = (T)sc[SC_NALPHA + 1];
    T u[24], v[24];
    load_v<SP>(g, VRS, r, s, u);
    load_v<SP>(g, VV, r, s, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      u[2 * k] += ar * v[2 * k] - ai * v[2 * k + 1];
      u[2 * k + 1] += ar * v[2 * k + 1] + ai * v[2 * k];
    }
    store_v<SP>(g, VRS, r, s, u);
  }
};
template <int SP> struct OpTS {  // (t, s) and ||t||^2
  static constexpr int NRED = 3, OUT = SC_TS;
  using T = typename Real<SP>::T;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double* acc) const {
    T t[24], u[24];
    load_v<SP>(g, VT, r, s, t);
    load_v<SP>(g, VRS, r, s, u);
    T re = 0, im = 0, tt = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re += t[2 * k] * u[2 * k] + t[2 * k + 1] * u[2 * k + 1];
      im += t[2 * k] * u[2 * k + 1] - t[2 * k + 1] * u[2 * k];
      tt += t[2 * k] * t[2 * k] + t[2 * k + 1] * t[2 * k + 1];
    }
    acc[0] += re;
    acc[1] += im;
    acc[2] += tt;
  }
};
// xs += alpha p + omega rs; rs += nomega t; then ||rs||^2 and (r0, rs)
template <int SP, int AP> struct OpXR {
  static constexpr int NRED = 3, OUT = SC_RN;
  using T = typename Real<AP>::T;
  __device__ void operator()(const Seg& g, int r, int s, const double* sc, double* acc) const {
    const T ar = (T)sc[SC_ALPHA], ai = (T)sc[SC_ALPHA + 1];
    const T wr = (T)sc[SC_OMEGA], wi = (T)sc[SC_OMEGA + 1];
    const T nr = (T)sc[SC_NOMEGA], ni = (T)sc[SC_NOMEGA + 1];
    T p[24], u[24], t[24], x[24], z[24];
    load_v<SP>(g, VP, r, s, p);
    load_v<SP>(g, VRS, r, s, u);
    load_v<SP>(g, VT, r, s, t);
    load_v<AP>(g, VXS, r, s, x);
    load_v<SP>(g, VR0, r, s, z);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      x[2 * k] += ar * p[2 * k] - ai * p[2 * k + 1] + wr * u[2 * k] - wi * u[2 * k + 1];
      x[2 * k + 1] += ar * p[2 * k + 1] + ai * p[2 * k] + wr * u[2 * k + 1] + wi * u[2 * k];
      u[2 * k] += nr * t[2 * k] - ni * t[2 * k + 1];
      u[2 * k + 1] += nr * t[2 * k + 1] + ni * t[2 * k];
    }
    store_v<AP>(g, VXS, r, s, x);
    store_v<SP>(g, VRS, r, s, u);
    load_v<SP>(g, VRS, r, s, u);  // the residual as stored
    T rr = 0, re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rr += u[2 * k] * u[2 * k] + u[2 * k + 1] * u[2 * k + 1];
      re += z[2 * k] * u[2 * k] + z[2 * k + 1] * u[2 * k + 1];
      im += z[2 * k] * u[2 * k + 1] - z[2 * k + 1] * u[2 * k];
    }
    acc[0] += rr;
    acc[1] += re;
    acc[2] += im;
  }
};
template <int AP> struct OpXUpd {  // x += xs; xs = 0
  static constexpr int NRED = 0, OUT = 0;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double*) const {
    double x[24], c[24];
    load_v<P64>(g, VX, r, s, x);
    load_v<AP>(g, VXS, r, s, c);
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      x[k] += c[k];
      c[k] = 0;
    }
    store_v<P64>(g, VX, r, s, x);
    store_v<AP>(g, VXS, r, s, c);
  }
};
struct OpXmy {  // r = b - r; ||r||^2
  static constexpr int NRED = 1, OUT = SC_RR;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double* acc) const {
    double b[24], y[24];
    load_v<P64>(g, VB, r, s, b);
    load_v<P64>(g, VR, r, s, y);
    double n = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      y[k] = b[k] - y[k];
      n += y[k] * y[k];
    }
    store_v<P64>(g, VR, r, s, y);
    acc[0] += n;
  }
};
struct OpNormB {  // ||b||^2
  static constexpr int NRED = 1, OUT = SC_BB;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double* acc) const {
    double b[24];
    load_v<P64>(g, VB, r, s, b);
    double n = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) n += b[k] * b[k];
    acc[0] += n;
  }
};
// start: X0 = 0: x = 0 and r = b; X0 = 1: x kept (r is computed from it). Both: the
// sloppy residual and shadow residual from b (replaced after an initial guess), p = v =
// 0, the sloppy correction xs = 0
template <int SP, int AP, bool X0> struct OpInit {
  static constexpr int NRED = 0, OUT = 0;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double*) const {
    double b[24], z[24];
    load_v<P64>(g, VB, r, s, b);
#pragma unroll
    for (int k = 0; k < 24; ++k) z[k] = 0;
    if (!X0) {
      store_v<P64>(g, VX, r, s, z);
      store_v<P64>(g, VR, r, s, b);
    }
    store_v<SP>(g, VRS, r, s, b);
    store_v<SP>(g, VR0, r, s, b);
    store_v<SP>(g, VP, r, s, z);
    store_v<SP>(g, VV, r, s, z);
    store_v<AP>(g, VXS, r, s, z);
  }
};
template <int SP> struct OpShadow {  // r0 = rs
  static constexpr int NRED = 0, OUT = 0;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double*) const {
    typename Real<SP>::T u[24];
    load_v<SP>(g, VRS, r, s, u);
    store_v<SP>(g, VR0, r, s, u);
  }
};
template <int SP, int AP> struct OpRestart {  // rs = r (sloppy); xs = 0
  static constexpr int NRED = 0, OUT = 0;
  __device__ void operator()(const Seg& g, int r, int s, const double*, double*) const {
    double y[24], z[24];
    load_v<P64>(g, VR, r, s, y);
    store_v<SP>(g, VRS, r, s, y);
#pragma unroll
    for (int k = 0; k < 24; ++k) z[k] = 0;
    store_v<AP>(g, VXS, r, s, z);
  }
};

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ void block_sum(double v[3], int n) {
  __shared__ double sh[NT / 32][3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[w][k] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < n; ++k) {
      double x = 0;
      for (int j = 0; j < NT / 32; ++j) x += sh[j][k];
      v[k] = x;
    }
  __syncthreads();
}

// One launch over every right-hand side of every segment: block b -> (segment,
// right-hand side, block within it). Reductions: per right-hand side, each block writes
// its partial sums; the last block of that right-hand side adds them in block order
// (deterministic) into its scalar slots.
// A right-hand side whose mask entry (mask[rhs * mstride], when mask is given) is 0 is
// skipped by all its blocks: no site work, no partial sums, its ticket untouched.
template <class Op>
__global__ void __launch_bounds__(NT) mb_kernel(const Seg* __restrict__ segs, int nseg, Op op, double* scal,
                                                double* part, unsigned* tick, const double* mask, int mstride) {
  int l = 0;
  while (l + 1 < nseg && (int)blockIdx.x >= segs[l + 1].blk0) ++l;
  const Seg& g = segs[l];
  const int k = blockIdx.x - g.blk0;
  const int r = k / g.bpr, bx = k - r * g.bpr;
  const int rhs = g.rhs0 + r;
  if (mask && mask[(size_t)rhs * mstride] == 0.0) return;  // uniform over the block
  double* sc = scal + (size_t)rhs * NSC;
  double acc[3] = {0, 0, 0};
  const int n = 2 * g.Vh;
  for (int s = bx * NT + threadIdx.x; s < n; s += g.bpr * NT) op(g, r, s, sc, acc);
  if constexpr (Op::NRED > 0) {
    __shared__ bool last;
    block_sum(acc, Op::NRED);
    if (threadIdx.x == 0) {
      double* pp = part + ((size_t)rhs * MAXBPR + bx) * 3;
      for (int j = 0; j < Op::NRED; ++j) pp[j] = acc[j];
      __threadfence();
      last = atomicAdd(tick + rhs, 1u) == (unsigned)g.bpr - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
      double s3[3] = {0, 0, 0};
      for (int b = 0; b < g.bpr; ++b)
        for (int j = 0; j < Op::NRED; ++j) s3[j] += __ldcg(part + ((size_t)rhs * MAXBPR + b) * 3 + j);
      for (int j = 0; j < Op::NRED; ++j) sc[Op::OUT + j] = s3[j];
      tick[rhs] = 0;
    }
  }
}

// scalar algebra, one thread per right-hand side
__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& qr, double& qi) {
  const double d = br * br + bi * bi;
  qr = (ar * br + ai * bi) / d;
  qi = (ai * br - ar * bi) / d;
}
__device__ __forceinline__ void fail(double* S, int f) {
  if (S[SC_FLAG] == FL_OK) S[SC_FLAG] = f;
  S[SC_ACTIVE] = 0;
}
// beta = (rho / rho_old)(alpha / omega); nbw = -beta omega
__global__ void k_b1(double* scal, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double* S = scal + (size_t)j * NSC;
  double br = 0, bi = 0, cr = 0, ci = 0;
  if (S[SC_ACTIVE] != 0) {
    if ((S[SC_RHOOLD] == 0 && S[SC_RHOOLD + 1] == 0) || (S[SC_OMEGA] == 0 && S[SC_OMEGA + 1] == 0)) {
      fail(S, FL_BREAKDOWN);
    } else {
      double q1r, q1i, q2r, q2i;
      cdiv(S[SC_RHO], S[SC_RHO + 1], S[SC_RHOOLD], S[SC_RHOOLD + 1], q1r, q1i);
      cdiv(S[SC_ALPHA], S[SC_ALPHA + 1], S[SC_OMEGA], S[SC_OMEGA + 1], q2r, q2i);
      br = q1r * q2r - q1i * q2i;
      bi = q1r * q2i + q1i * q2r;
      const double wr = S[SC_OMEGA], wi = S[SC_OMEGA + 1];
      cr = -(br * wr - bi * wi);
      ci = -(br * wi + bi * wr);
    }
  }
  S[SC_BETA] = br; S[SC_BETA + 1] = bi;
  S[SC_NBW] = cr; S[SC_NBW + 1] = ci;
}
// alpha = rho / (r0, v)
__global__ void k_b2(double* scal, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double* S = scal + (size_t)j * NSC;
  double ar = 0, ai = 0;
  if (S[SC_ACTIVE] != 0) {
    const double sr = S[SC_SIGMA], si = S[SC_SIGMA + 1];
    if (bad(sr) || bad(si)) fail(S, FL_NONFINITE);
    else if (sr == 0 && si == 0) fail(S, FL_BREAKDOWN);
    else cdiv(S[SC_RHO], S[SC_RHO + 1], sr, si, ar, ai);
  }
  S[SC_ALPHA] = ar; S[SC_ALPHA + 1] = ai;
  S[SC_NALPHA] = -ar; S[SC_NALPHA + 1] = -ai;
}
// omega = (t, s) / (t, t)
__global__ void k_b3(double* scal, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double* S = scal + (size_t)j * NSC;
  double wr = 0, wi = 0;
  if (S[SC_ACTIVE] != 0) {
    const double tt = S[SC_TS + 2];
    if (bad(tt) || bad(S[SC_TS]) || bad(S[SC_TS + 1])) fail(S, FL_NONFINITE);
    else if (tt == 0) fail(S, FL_BREAKDOWN);
    else { wr = S[SC_TS] / tt; wi = S[SC_TS + 1] / tt; }
  }
  if (S[SC_ACTIVE] == 0) {
    // frozen (converged, or failed in this iteration): no update of x, xs or r
    S[SC_ALPHA] = S[SC_ALPHA + 1] = 0;
    wr = wi = 0;
  }
  S[SC_OMEGA] = wr; S[SC_OMEGA + 1] = wi;
  S[SC_NOMEGA] = -wr; S[SC_NOMEGA + 1] = -wi;
}
// rho_old = rho; rho = (r0, r); mirror ||r||^2 and the flag for the host
__global__ void k_b4(double* scal, int n, double* mirror) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double* S = scal + (size_t)j * NSC;
  if (S[SC_ACTIVE] != 0) {
    if (bad(S[SC_RN])) fail(S, FL_NONFINITE);
    S[SC_RHOOLD] = S[SC_RHO]; S[SC_RHOOLD + 1] = S[SC_RHO + 1];
    S[SC_RHO] = S[SC_RN + 1]; S[SC_RHO + 1] = S[SC_RN + 2];
  }
  mirror[2 * j] = S[SC_RN];
  mirror[2 * j + 1] = S[SC_FLAG];
}
// start / after a reliable update of the right-hand sides with upd[j] != 0: rho = (r0, rs)
// (in SC_TMP); active flags from the host
__global__ void k_restart(double* scal, int n, const double* active, const double* upd, int first) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || upd[j] == 0.0) return;
  double* S = scal + (size_t)j * NSC;
  if (first) {
    S[SC_RHOOLD] = 1; S[SC_RHOOLD + 1] = 0;
    S[SC_ALPHA] = 1; S[SC_ALPHA + 1] = 0;
    S[SC_OMEGA] = 1; S[SC_OMEGA + 1] = 0;
    S[SC_FLAG] = FL_OK;
  }
  S[SC_ACTIVE] = active[j];
  S[SC_RHO] = S[SC_TMP]; S[SC_RHO + 1] = S[SC_TMP + 1];
}
// per-right-hand-side value of a scalar slot into host-visible memory
__global__ void k_gather(const double* scal, int n, int slot, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = scal[(size_t)j * NSC + slot];
}

}  // namespace bs
}  // namespace dirac

using namespace dirac;
using namespace dirac::bs;

namespace {

struct Run {
  std::vector<dirac_ctx*> ctx;
  std::vector<Seg> segs;
  Seg* d_segs = nullptr;
  int nseg = 0, nrhs = 0, nblk = 0;
  double* scal = nullptr;
  double* part = nullptr;
  unsigned* tick = nullptr;
  double* host = nullptr;      // mapped: [2][nrhs][2] mirror, [nrhs] gathered values, [nrhs] active,
                               // [nrhs] reliable-update mask
  double* dhost = nullptr;
  std::vector<void*> bufs;
  dirac_batch* plan_pv = nullptr;
  dirac_batch* plan_st = nullptr;
  dirac_batch* plan_x = nullptr;
  dirac_batch* plan_xds = nullptr;   // r = M x in double-single arithmetic
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  ~Run() {
    if (own_stream && st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (plan_pv) dirac_batch_destroy(plan_pv);
    if (plan_st) dirac_batch_destroy(plan_st);
    if (plan_x) dirac_batch_destroy(plan_x);
    if (plan_xds) dirac_batch_destroy(plan_xds);
    for (void* p : bufs) cudaFree(p);
    if (d_segs) cudaFree(d_segs);
    if (scal) cudaFree(scal);
    if (part) cudaFree(part);
    if (tick) cudaFree(tick);
    if (host) cudaFreeHost(host);
  }
  double* mirror(int slot) { return dhost + 2 * nrhs * slot; }
  volatile double* hmirror(int slot) { return host + 2 * nrhs * slot; }
  double* gathered() { return dhost + 4 * nrhs; }
  volatile double* hgathered() { return host + 4 * nrhs; }
  double* active_d() { return dhost + 5 * nrhs; }
  double* active_h() { return host + 5 * nrhs; }
  double* upd_d() { return dhost + 6 * nrhs; }
  double* upd_h() { return host + 6 * nrhs; }
};

// which right-hand sides a batched BLAS launch covers
enum : int { ALL = 0, ACTIVE = 1, UPDATING = 2 };

template <class Op>
int launch(Run& R, const Op& op, int which = ALL) {
  const double* mask = which == ACTIVE ? R.scal + SC_ACTIVE : (which == UPDATING ? R.upd_d() : nullptr);
  const int stride = which == ACTIVE ? NSC : 1;
  mb_kernel<Op><<<R.nblk, NT, 0, R.st>>>(R.d_segs, R.nseg, op, R.scal, R.part, R.tick, mask, stride);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}
int scalar(Run& R, int which, int slot = 0) {
  const int g = (R.nrhs + 63) / 64;
  switch (which) {
    case 1: k_b1<<<g, 64, 0, R.st>>>(R.scal, R.nrhs); break;
    case 2: k_b2<<<g, 64, 0, R.st>>>(R.scal, R.nrhs); break;
    case 3: k_b3<<<g, 64, 0, R.st>>>(R.scal, R.nrhs); break;
    case 4: k_b4<<<g, 64, 0, R.st>>>(R.scal, R.nrhs, R.mirror(slot)); break;
  }
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}

#define RT(...)                  \
  do {                           \
    int _rc = (__VA_ARGS__);     \
    if (_rc) return _rc;         \
  } while (0)

// one BiCGstab iteration of every right-hand side (launches depend only on `slot`)
template <int SP, int AP>
int iteration(Run& R, int slot) {
  // right-hand sides that are not active (converged or failed) are skipped throughout
  RT(scalar(R, 1));
  RT(launch(R, OpPUpd<SP>{}, ACTIVE));
  RT(dirac_batch_apply(R.plan_pv, R.st));  // v = M p
  RT(launch(R, OpCdot<SP, VR0, VV, SC_SIGMA>{}, ACTIVE));
  RT(scalar(R, 2));
  RT(launch(R, OpSUpd<SP>{}, ACTIVE));     // s = r - alpha v
  RT(dirac_batch_apply(R.plan_st, R.st));  // t = M s
  RT(launch(R, OpTS<SP>{}, ACTIVE));
  RT(scalar(R, 3));
  RT(launch(R, OpXR<SP, AP>{}, ACTIVE));
  RT(scalar(R, 4, slot));
  return DIRAC_OK;
}

// r = b - M x (FP64 fields) with the given plan; the per-rhs ||r||^2 is left in the host
// array gathered()
// (the right-hand sides with upd[j] != 0 only)
int residual(Run& R, dirac_batch* plan) {
  RT(dirac_batch_apply(plan, R.st));   // r = M x
  RT(launch(R, OpXmy{}, UPDATING));
  k_gather<<<(R.nrhs + 63) / 64, 64, 0, R.st>>>(R.scal, R.nrhs, SC_RR, R.gathered());
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(R.st) != cudaSuccess) return DIRAC_ERR_CUDA;
  return DIRAC_OK;
}
// reliable update of every right-hand side: x += xs, then the true residual, in
// double-single arithmetic when the plan for it exists (exact = false) else in FP64
template <int SP, int AP>
int reliable(Run& R, bool exact) {
  RT(launch(R, OpXUpd<AP>{}, UPDATING));
  return residual(R, (exact || !R.plan_xds) ? R.plan_x : R.plan_xds);
}
template <int SP, int AP>
int restart(Run& R, int first) {
  RT(launch(R, OpRestart<SP, AP>{}, UPDATING));
  RT(launch(R, OpCdot<SP, VR0, VRS, SC_TMP>{}, UPDATING));
  // the host's active flags (pinned, mapped) for the scalar state
  k_restart<<<(R.nrhs + 63) / 64, 64, 0, R.st>>>(R.scal, R.nrhs, R.active_d(), R.upd_d(), first);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}

template <int SP>
int solve_batched_impl(Run& R, const dirac_solver_params& P, dirac_solver_stats* stats,
                       std::vector<double>& bb) {
  constexpr int AP = SP == P16 ? P32 : SP;  // sloppy corrections accumulated in >= FP32
  const int n = R.nrhs;
  // ||b||^2, r = b, x = 0 (or r = b - M x from the initial guess)
  RT(launch(R, OpNormB{}));
  k_gather<<<(n + 63) / 64, 64, 0, R.st>>>(R.scal, n, SC_BB, R.gathered());
  if (cudaStreamSynchronize(R.st) != cudaSuccess) return DIRAC_ERR_CUDA;
  std::vector<double> target(n), rmax(n), rr(n);
  std::vector<int> active(n, 1), relup(n, 0), stale(n, 0);
  for (int j = 0; j < n; ++j) R.upd_h()[j] = 1;  // the start covers every right-hand side
  for (int j = 0; j < n; ++j) {
    bb[j] = R.hgathered()[j];
    if (!std::isfinite(bb[j])) {
      R.err = "non-finite source";
      return DIRAC_ERR_NONFINITE;
    }
    target[j] = P.tol * P.tol * bb[j];
  }
  if (P.use_x0) {
    // r = b - M x from the caller's x; the sloppy and shadow residuals from it
    RT(launch(R, OpInit<SP, AP, true>{}));
    RT(dirac_batch_apply(R.plan_x, R.st));
    RT(launch(R, OpXmy{}));
    RT(launch(R, OpRestart<SP, AP>{}));
    RT(launch(R, OpShadow<SP>{}));
    k_gather<<<(n + 63) / 64, 64, 0, R.st>>>(R.scal, n, SC_RR, R.gathered());
    if (cudaStreamSynchronize(R.st) != cudaSuccess) return DIRAC_ERR_CUDA;
    for (int j = 0; j < n; ++j) rr[j] = R.hgathered()[j];
  } else {
    RT(launch(R, OpInit<SP, AP, false>{}));
    rr = bb;
  }
  for (int j = 0; j < n; ++j) {
    rmax[j] = rr[j];
    active[j] = rr[j] >= target[j] && bb[j] > 0;
    R.active_h()[j] = active[j];
  }
  RT(restart<SP, AP>(R, 1));
  const double d2 = P.delta * P.delta;
  cudaEvent_t ev[2];
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int gstate[2] = {0, 0};
  int rc = DIRAC_OK;
  int it = 0, total = 0;
  auto any_active = [&] {
    for (int j = 0; j < n; ++j)
      if (active[j]) return true;
    return false;
  };
  while (rc == DIRAC_OK && any_active() && total < P.max_iter) {
    const int slot = it & 1;
    // iteration, replayed from its graph after the first two
    if (gstate[slot] == 0) {
      rc = iteration<SP, AP>(R, slot);
      gstate[slot] = 1;
    } else if (gstate[slot] == 1) {
      cudaGraph_t gr = nullptr;
      if (cudaStreamBeginCapture(R.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = DIRAC_ERR_CUDA; break; }
      const int rc2 = iteration<SP, AP>(R, slot);
      const cudaError_t ec = cudaStreamEndCapture(R.st, &gr);
      if (rc2 || ec != cudaSuccess || cudaGraphInstantiate(&graph[slot], gr, 0) != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        rc = rc2 ? rc2 : DIRAC_ERR_CUDA;
        break;
      }
      cudaGraphDestroy(gr);
      gstate[slot] = 2;
      rc = cudaGraphLaunch(graph[slot], R.st) == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
    } else {
      rc = cudaGraphLaunch(graph[slot], R.st) == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
    }
    if (rc) break;
    cudaEventRecord(ev[slot], R.st);
    ++total;
    for (int j = 0; j < n; ++j)
      if (active[j]) stats[j].iters++;
    if (it > 0) {
      // the previous iteration's residuals decide reliable updates and convergence
      const int ps = (it - 1) & 1;
      if (cudaEventSynchronize(ev[ps]) != cudaSuccess) { rc = DIRAC_ERR_CUDA; break; }
      volatile double* m = R.hmirror(ps);
      bool upd = false;
      for (int j = 0; j < n; ++j) {
        R.upd_h()[j] = 0;
        if (!active[j]) continue;
        if (stale[j]) {  // its previous iteration ran before its reliable update
          stale[j] = 0;
          continue;
        }
        const int fl = (int)m[2 * j + 1];
        if (fl != FL_OK) {
          active[j] = 0;
          stats[j].precond_kind = -fl;  // recorded below as the status of this rhs
          continue;
        }
        const double rp = m[2 * j];
        if ((d2 > 0 && rp < d2 * rmax[j]) || rp < target[j]) {
          upd = true;
          R.upd_h()[j] = 1;  // only the right-hand sides that ask are updated
        }
      }
      if (upd) {
        nvtxRangePushA("batched reliable update (FP64)");
        rc = reliable<SP, AP>(R, false);
        // a right-hand side that the double-single residual finds converged is decided
        // by the FP64 operator
        bool fresh = false;
        for (int j = 0; rc == DIRAC_OK && j < n; ++j)
          fresh = fresh || (R.upd_h()[j] != 0 && R.hgathered()[j] < target[j]);
        if (rc == DIRAC_OK && fresh && R.plan_xds) rc = residual(R, R.plan_x);
        if (rc == DIRAC_OK) {
          for (int j = 0; j < n; ++j) {
            R.active_h()[j] = active[j];
            if (R.upd_h()[j] == 0) continue;
            rr[j] = R.hgathered()[j];
            relup[j]++;
            stale[j] = 1;
            if (rr[j] < target[j]) active[j] = 0;
            rmax[j] = rr[j];
            R.active_h()[j] = active[j];
          }
          rc = restart<SP, AP>(R, 0);
          // the restart kernels read the mapped update and active flags, which the host
          // rewrites at the next check: they must have run first
          if (rc == DIRAC_OK && cudaStreamSynchronize(R.st) != cudaSuccess) rc = DIRAC_ERR_CUDA;
        }
        nvtxRangePop();
      }
    }
    ++it;
  }
  if (rc == DIRAC_OK) {
    // fold in what is left of the sloppy corrections and take the final FP64 residuals
    // of every right-hand side
    if (cudaStreamSynchronize(R.st) != cudaSuccess) {
      rc = DIRAC_ERR_CUDA;
    } else {
      for (int j = 0; j < n; ++j) R.upd_h()[j] = 1;
      rc = reliable<SP, AP>(R, true);
    }
    if (rc == DIRAC_OK)
      for (int j = 0; j < n; ++j) rr[j] = R.hgathered()[j];
  }
  for (int s = 0; s < 2; ++s) {
    if (graph[s]) cudaGraphExecDestroy(graph[s]);
    cudaEventDestroy(ev[s]);
  }
  for (int j = 0; j < n; ++j) {
    stats[j].reliable_updates = relup[j];
    stats[j].true_rel_resid = bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0;
    stats[j].dslash_calls = 2 * stats[j].iters + relup[j] + 1;
  }
  return rc;
}

}  // namespace

extern "C" int solve_batched(dirac_ctx* const* ctxs, int nlat, void* const* x, const void* const* b,
                             const int* nrhs, const dirac_solver_params* params, dirac_solver_stats* stats,
                             void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctxs || !x || !b || !nrhs || !params || !stats || nlat < 1 || nlat > 16) return DIRAC_ERR_ARG;
  const dirac_solver_params& P = *params;
  if (P.alg != DIRAC_SOLVER_BICGSTAB) return set_err(ctxs[0], DIRAC_ERR_UNSUPPORTED, "solve_batched: BiCGstab only");
  const int sp = P.prec_sloppy;
  if (sp < P64 || sp > P16) return set_err(ctxs[0], DIRAC_ERR_ARG, "solve_batched: bad sloppy precision");
  Run R;
  int tot = 0;
  for (int l = 0; l < nlat; ++l) {
    dirac_ctx* c = ctxs[l];
    if (!c || !x[l] || !b[l] || nrhs[l] < 1) return DIRAC_ERR_ARG;
    if (c->p.kind != DIRAC_WILSON_CLOVER) return set_err(c, DIRAC_ERR_UNSUPPORTED, "solve_batched: Wilson-clover only");
    int rc = check_op(c, P64, false);
    if (!rc) rc = check_op(c, sp, false);
    if (rc) return rc;
    tot += nrhs[l];
  }
  if (tot > MAXRHS) return set_err(ctxs[0], DIRAC_ERR_ARG, "solve_batched: more than 256 right-hand sides");
  for (int j = 0; j < tot; ++j) stats[j] = dirac_solver_stats{};
  // a private stream (graph capture needs one) ordered after the caller's stream
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t order = nullptr;
  if (cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&order, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctxs[0], DIRAC_ERR_CUDA, "solve_batched: stream");
  }
  R.own_stream = true;
  cudaEventRecord(order, caller);
  cudaStreamWaitEvent(R.st, order, 0);
  cudaEventDestroy(order);
  R.nrhs = tot;
  const int ap = sp == P16 ? P32 : sp;
  const int prec_of[NVEC] = {P64, P64, P64, sp, sp, sp, sp, sp, ap};
  // segments: caller's x and b, workspace for the others
  int blk = 0, rhs0 = 0;
  for (int l = 0; l < nlat; ++l) {
    dirac_ctx* c = ctxs[l];
    Seg g;
    g.Vh = (int)c->Vh;
    g.nrhs = nrhs[l];
    g.rhs0 = rhs0;
    g.blk0 = blk;
    long bpr = (2 * c->Vh + NT * 16 - 1) / (NT * 16);
    g.bpr = (int)(bpr < 1 ? 1 : (bpr > MAXBPR ? MAXBPR : bpr));
    for (int v = 0; v < NVEC; ++v) {
      g.fb[v] = 2 * spinor_half_bytes(prec_of[v], 24, c->Vh);
      if (v == VX) g.f[v] = (char*)x[l];
      else if (v == VB) g.f[v] = (char*)b[l];
      else {
        void* p = nullptr;
        if (cudaMalloc(&p, g.fb[v] * nrhs[l]) != cudaSuccess) {
          cudaGetLastError();
          return set_err(c, DIRAC_ERR_OOM, "solve_batched: workspace");
        }
        R.bufs.push_back(p);
        g.f[v] = (char*)p;
      }
    }
    R.segs.push_back(g);
    R.ctx.push_back(c);
    blk += g.bpr * g.nrhs;
    rhs0 += g.nrhs;
  }
  R.nseg = nlat;
  R.nblk = blk;
  if (cudaMalloc(&R.d_segs, sizeof(Seg) * nlat) != cudaSuccess ||
      cudaMalloc(&R.scal, sizeof(double) * NSC * tot) != cudaSuccess ||
      cudaMalloc(&R.part, sizeof(double) * 3 * MAXBPR * tot) != cudaSuccess ||
      cudaMalloc(&R.tick, sizeof(unsigned) * tot) != cudaSuccess ||
      cudaHostAlloc(&R.host, sizeof(double) * 7 * tot, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&R.dhost, R.host, 0) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctxs[0], DIRAC_ERR_OOM, "solve_batched: scalar state");
  }
  for (int j = 0; j < 7 * tot; ++j) R.host[j] = 0;
  cudaMemsetAsync(R.scal, 0, sizeof(double) * NSC * tot, R.st);
  cudaMemsetAsync(R.tick, 0, sizeof(unsigned) * tot, R.st);
  cudaMemcpyAsync(R.d_segs, R.segs.data(), sizeof(Seg) * nlat, cudaMemcpyHostToDevice, R.st);
  // operator plans: v = M p and t = M s in the sloppy precision, r = M x in FP64
  {
    std::vector<void*> pin(nlat), pout(nlat), sin(nlat), sout(nlat), xin(nlat), rout(nlat);
    for (int l = 0; l < nlat; ++l) {
      pin[l] = R.segs[l].f[VP];
      pout[l] = R.segs[l].f[VV];
      sin[l] = R.segs[l].f[VRS];
      sout[l] = R.segs[l].f[VT];
      xin[l] = R.segs[l].f[VX];
      rout[l] = R.segs[l].f[VR];
    }
    // the sloppy plans run the default CUDA-core shape (their masks skip converged systems,
    // which the tensor-core kernel cannot); none of the plans is timed (the FP64 plan's
    // launches are seconds of FP64 arithmetic)
    int rc = batch_create(ctxs, nlat, pout.data(), (const void* const*)pin.data(), nrhs, sp, R.st, &R.plan_pv, -1);
    if (!rc) rc = batch_create(ctxs, nlat, sout.data(), (const void* const*)sin.data(), nrhs, sp, R.st, &R.plan_st, -1);
    if (!rc) rc = batch_create(ctxs, nlat, rout.data(), (const void* const*)xin.data(), nrhs, P64, R.st, &R.plan_x, 0);
    // the reliable updates' residuals in double-single arithmetic where every lattice
    // allows it (FP64 18-real links) and every context has it switched on
    bool ds = true;
    for (int l = 0; l < nlat; ++l) ds = ds && ctxs[l]->ds_residual && ds_available(ctxs[l]);
    if (!rc && ds)
      rc = batch_create(ctxs, nlat, rout.data(), (const void* const*)xin.data(), nrhs, P64, R.st, &R.plan_xds, 0, true);
    // the sloppy plans skip right-hand sides that are no longer active, the FP64 plans
    // those that are not being updated
    if (!rc) rc = batch_set_mask(R.plan_pv, R.scal + SC_ACTIVE, NSC, R.st);
    if (!rc) rc = batch_set_mask(R.plan_st, R.scal + SC_ACTIVE, NSC, R.st);
    if (!rc) rc = batch_set_mask(R.plan_x, R.upd_d(), 1, R.st);
    if (!rc && R.plan_xds) rc = batch_set_mask(R.plan_xds, R.upd_d(), 1, R.st);
    if (rc) return set_err(ctxs[0], rc, "solve_batched: operator plans");
  }
  std::vector<double> bb(tot, 0.0);
  nvtxRangePushA("solve_batched");
  int rc;
  if (sp == P16) rc = solve_batched_impl<P16>(R, P, stats, bb);
  else if (sp == P32) rc = solve_batched_impl<P32>(R, P, stats, bb);
  else rc = solve_batched_impl<P64>(R, P, stats, bb);
  nvtxRangePop();
  const cudaError_t e = cudaStreamSynchronize(R.st);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = DIRAC_OK;
  for (int j = 0; j < tot; ++j) {
    stats[j].seconds = secs;
    const int fl = stats[j].precond_kind;
    stats[j].precond_kind = 0;
    int st = DIRAC_OK;
    if (fl == -FL_BREAKDOWN) st = DIRAC_ERR_BREAKDOWN;
    else if (fl == -FL_NONFINITE) st = DIRAC_ERR_NONFINITE;
    else if (!(stats[j].true_rel_resid <= P.tol)) st = DIRAC_ERR_NOT_CONVERGED;
    if (st != DIRAC_OK && worst == DIRAC_OK) worst = st;
  }
  if (rc == DIRAC_OK && e != cudaSuccess) rc = DIRAC_ERR_CUDA;
  if (rc) return set_err(ctxs[0], rc, "solve_batched: " + (R.err.empty() ? std::string("CUDA error") : R.err));
  if (worst != DIRAC_OK) return set_err(ctxs[0], worst, "solve_batched: some right-hand sides did not converge");
  return DIRAC_OK;
}
