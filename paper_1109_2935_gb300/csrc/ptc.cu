// Gauge-equivariant parallel-transport convolution (PTC) network: a learned, linear
// preconditioner K for the flexible GCR of Algorithm 1 (not part of the paper).
//
// Layer l: out_c(x) = sum_c' sum_p W_l[p][c][c'] (T_p in_c')(x) over the 9 paths
// p = 0, +x, -x, +y, -y, +z, -z, +t, -t, with (T_+mu f)(x) = U_mu(x) f(x + mu) and
// (T_-mu f)(x) = U_mu(x - mu)^dagger f(x - mu) (fermion sign across an antiperiodic t
// edge) and W a complex 4x4 spin matrix. Spin mixing and colour transport commute, so
// each path transports min(c_in, c_out) spinors: the inputs (c_in <= c_out), or the
// spin-mixed combinations (c_in > c_out).
//
// Kernels (FP32 fields in the context's chunk-major layout, FP32 weights):
//   ptc_layer_kernel  one thread per site, weights in shared memory, blockIdx.y = pair
//   ptc_wgrad_kernel  dL/dconj(W_l[p][c][c']) = sum_x sum_colour g_c(x) (T_p in_c'(x))^dagger,
//                     a lattice-wide 4x4 contraction per (p, c, c'): per-thread FP32 sums,
//                     warp-shuffle + shared-memory block sums, a fixed-order FP64 pass
//   ptc_loss_kernel   d = K r - v, dL/dconj(K r) = d / (B ||v||^2), the batch loss
//   ptc_adam_kernel   Adam on the real and imaginary parts (gradient 2 dL/dconj(W))
// The input gradient of a layer is the layer with adjoint weights: T_p^dagger = T_{-p}, so
// dL/dconj(in_c') = sum_p sum_c T_{-p} W[p][c][c']^dagger g_c, a forward layer whose
// weights ptc_adjoint_kernel builds. The 4x4 contraction per path leaves tensor-core
// tiles mostly empty, so the gradient runs on the FP32 pipes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

#include "internal.h"

namespace dirac {
namespace {

constexpr int NPATH = 9;
constexpr int MAXB = 16;  // pairs per launch
constexpr int MAXC = 4;   // channels per layer
constexpr int TPB = 128;  // layer kernel threads per block
constexpr int GTPB = 256; // gradient / loss kernel threads per block

struct InTab { const char* p[MAXB * MAXC]; };   // [pair][channel] full fields
struct OutTab { char* p[MAXB * MAXC]; };

struct LayerArg {
  InTab in;
  OutTab out;
  const float2* w;    // [p][c_out][c_in][4][4]
  const char* gauge;  // FP32 links of the context
  Geom g;
};

struct GradArg {
  InTab x;            // layer inputs [pair][c_in]
  InTab gy;           // dL/dconj(layer output) [pair][c_out]
  float* partial;     // [pair][p * c_out + c][block][c_in * 32]
  const char* gauge;
  Geom g;
};

__device__ __forceinline__ void load_c(const float v[24], C<float> t[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) t[k] = C<float>{v[2 * k], v[2 * k + 1]};
}

// t = sgn * (U or U^dagger) f on each of the 4 spins
__device__ __forceinline__ void transport(const Link<float>& U, bool dag, float sgn, const C<float> f[12],
                                          C<float> t[12]) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    C<float> v[3];
    if (dag) su3_mv_dag(U, f + 3 * s, v);
    else su3_mv(U, f + 3 * s, v);
#pragma unroll
    for (int a = 0; a < 3; ++a) t[3 * s + a] = sgn * v[a];
  }
}

// acc[s][a] += sum_t W[s][t] f[t][a]
__device__ __forceinline__ void spin_mac(C<float> acc[12], const float2* W, const C<float> f[12]) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float2 w = W[4 * s + t];
      C<float> wc = {w.x, w.y};
#pragma unroll
      for (int a = 0; a < 3; ++a) cmac(acc[3 * s + a], wc, f[3 * t + a]);
    }
}

// Neighbour of path p >= 1: its checkerboard index (opposite parity), the link and
// whether it is applied as U^dagger, and the boundary sign.
template <int R>
__device__ __forceinline__ void path_site(const Geom& g, const char* gauge, int p, const int x[4], int par,
                                          int cb, int& ycb, Link<float>& U, bool& dag, float& sgn) {
  const int mu = (p - 1) >> 1;
  dag = ((p - 1) & 1) != 0;
  int y[4] = {x[0], x[1], x[2], x[3]};
  sgn = 1.f;
  if (!dag) {
    if (++y[mu] == g.L[mu]) {
      y[mu] = 0;
      if (mu == 3 && g.apbc) sgn = -1.f;
    }
    ycb = cb_index(g, y);
    LinkIO<P32, R>::load(gauge, g.Vh, mu, par, cb, U);
  } else {
    if (y[mu]-- == 0) {
      y[mu] = g.L[mu] - 1;
      if (mu == 3 && g.apbc) sgn = -1.f;
    }
    ycb = cb_index(g, y);
    LinkIO<P32, R>::load(gauge, g.Vh, mu, 1 - par, ycb, U);
  }
}

template <int CIN, int COUT, int R>
__global__ void __launch_bounds__(TPB) ptc_layer_kernel(const LayerArg a) {
  constexpr int NW = NPATH * COUT * CIN * 16;
  __shared__ float2 sw[NW];
  for (int i = threadIdx.x; i < NW; i += TPB) sw[i] = a.w[i];
  __syncthreads();
  const Geom& g = a.g;
  const int Vh = g.Vh, z = blockIdx.y;
  const int idx = blockIdx.x * TPB + threadIdx.x;
  if (idx >= 2 * Vh) return;
  const int par = idx >= Vh ? 1 : 0, cb = idx - par * Vh;
  const size_t hb = (size_t)96 * Vh;
  int x[4];
  cb_coords(g, cb, par, x);
  C<float> acc[COUT][12];
#pragma unroll
  for (int c = 0; c < COUT; ++c)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[c][k] = C<float>{0.f, 0.f};

#pragma unroll 1
  for (int p = 0; p < NPATH; ++p) {
    int ycb = cb, ypar = par;
    Link<float> U;
    bool dag = false;
    float sgn = 1.f;
    if (p > 0) {
      path_site<R>(g, a.gauge, p, x, par, cb, ycb, U, dag, sgn);
      ypar = 1 - par;
    }
    if constexpr (CIN <= COUT) {
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        float v[24];
        SpinorIO<P32, 24>::load(a.in.p[z * MAXC + ci] + ypar * hb, Vh, ycb, v);
        C<float> f[12], t[12];
        load_c(v, f);
        if (p > 0) transport(U, dag, sgn, f, t);
        else
#pragma unroll
          for (int k = 0; k < 12; ++k) t[k] = f[k];
#pragma unroll
        for (int co = 0; co < COUT; ++co) spin_mac(acc[co], sw + ((p * COUT + co) * CIN + ci) * 16, t);
      }
    } else {
      C<float> m[COUT][12];
#pragma unroll
      for (int co = 0; co < COUT; ++co)
#pragma unroll
        for (int k = 0; k < 12; ++k) m[co][k] = C<float>{0.f, 0.f};
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        float v[24];
        SpinorIO<P32, 24>::load(a.in.p[z * MAXC + ci] + ypar * hb, Vh, ycb, v);
        C<float> f[12];
        load_c(v, f);
#pragma unroll
        for (int co = 0; co < COUT; ++co) spin_mac(m[co], sw + ((p * COUT + co) * CIN + ci) * 16, f);
      }
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        if (p > 0) {
          C<float> t[12];
          transport(U, dag, sgn, m[co], t);
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[co][k] = acc[co][k] + t[k];
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[co][k] = acc[co][k] + m[co][k];
        }
      }
    }
  }
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    float v[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) { v[2 * k] = acc[co][k].r; v[2 * k + 1] = acc[co][k].i; }
    SpinorIO<P32, 24>::store(a.out.p[z * MAXC + co] + par * hb, Vh, cb, v);
  }
}

// blockIdx.y = p * COUT + co, blockIdx.z = pair; grid-stride over the sites.
template <int CIN, int COUT, int R>
__global__ void __launch_bounds__(GTPB) ptc_wgrad_kernel(const GradArg a) {
  const int p = blockIdx.y / COUT, co = blockIdx.y % COUT, z = blockIdx.z;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const size_t hb = (size_t)96 * Vh;
  float acc[CIN][32];
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[ci][k] = 0.f;

  for (int idx = blockIdx.x * GTPB + threadIdx.x; idx < 2 * Vh; idx += gridDim.x * GTPB) {
    const int par = idx >= Vh ? 1 : 0, cb = idx - par * Vh;
    int x[4];
    cb_coords(g, cb, par, x);
    float gv[24];
    SpinorIO<P32, 24>::load(a.gy.p[z * MAXC + co] + par * hb, Vh, cb, gv);
    C<float> gy[12];
    load_c(gv, gy);
    int ycb = cb, ypar = par;
    Link<float> U;
    bool dag = false;
    float sgn = 1.f;
    if (p > 0) {
      path_site<R>(g, a.gauge, p, x, par, cb, ycb, U, dag, sgn);
      ypar = 1 - par;
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      float v[24];
      SpinorIO<P32, 24>::load(a.x.p[z * MAXC + ci] + ypar * hb, Vh, ycb, v);
      C<float> f[12], t[12];
      load_c(v, f);
      if (p > 0) transport(U, dag, sgn, f, t);
      else
#pragma unroll
        for (int k = 0; k < 12; ++k) t[k] = f[k];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
          C<float> q = {acc[ci][2 * (4 * s + tt)], acc[ci][2 * (4 * s + tt) + 1]};
#pragma unroll
          for (int c = 0; c < 3; ++c) cmacc(q, t[3 * tt + c], gy[3 * s + c]);
          acc[ci][2 * (4 * s + tt)] = q.r;
          acc[ci][2 * (4 * s + tt) + 1] = q.i;
        }
    }
  }
  constexpr int NV = CIN * 32;
  __shared__ float red[GTPB / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      float v = acc[ci][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][ci * 32 + k] = v;
    }
  __syncthreads();
  float* dst = a.partial + (((size_t)z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * NV;
  for (int j = threadIdx.x; j < NV; j += GTPB) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < GTPB / 32; ++w) s += red[w][j];
    dst[j] = s;
  }
}

// grad[(p * COUT + co) * CIN * 32 + ci * 32 + k] = sum over pairs and blocks, FP64, fixed order
__global__ void ptc_wgrad_reduce(const float* partial, int nblk, int npair, int cout, int cin, double* grad) {
  const int n = NPATH * cout * cin * 32;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int nv = cin * 32, pco = j / nv, r = j % nv;
  double s = 0;
  for (int z = 0; z < npair; ++z)
    for (int b = 0; b < nblk; ++b)
      s += partial[(((size_t)z * NPATH * cout + pco) * nblk + b) * nv + r];
  grad[j] = s;
}

// W'[pbar][ci][co][s][t] = conj(W[p][co][ci][t][s]), pbar the reversed path
__global__ void ptc_adjoint_kernel(const float2* w, float2* wa, int cout, int cin) {
  const int n = NPATH * cout * cin * 16;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int t = j & 3, s = (j >> 2) & 3;
  int r = j >> 4;
  const int ci = r % cin;
  r /= cin;
  const int co = r % cout, p = r / cout;
  const int pb = p == 0 ? 0 : (((p - 1) & 1) ? p - 1 : p + 1);
  const float2 v = w[((p * cout + co) * cin + ci) * 16 + 4 * t + s];
  wa[((pb * cin + ci) * cout + co) * 16 + 4 * s + t] = make_float2(v.x, -v.y);
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < GTPB / 32; ++w) s += sh[w];
  return s;
}

// partial[z * gridDim.x + block] = sum |v_z|^2 over the block's float4 chunks
__global__ void __launch_bounds__(GTPB) ptc_norm_kernel(const InTab v, int64_t n4, double* partial) {
  __shared__ double sh[GTPB / 32];
  const int z = blockIdx.y;
  const float4* p = reinterpret_cast<const float4*>(v.p[z * MAXC]);
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * GTPB + threadIdx.x; i < n4; i += (int64_t)gridDim.x * GTPB) {
    float4 q = p[i];
    s = fmaf(q.x, q.x, s); s = fmaf(q.y, q.y, s); s = fmaf(q.z, q.z, s); s = fmaf(q.w, q.w, s);
  }
  double t = block_sum((double)s, sh);
  if (threadIdx.x == 0) partial[(size_t)z * gridDim.x + blockIdx.x] = t;
}

// inv[z] = 1 / (npair ||v_z||^2) (0 for a zero v)
__global__ void ptc_inv_kernel(const double* partial, int nblk, int npair, double* inv) {
  const int z = threadIdx.x;
  if (z >= npair) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)z * nblk + b];
  inv[z] = s > 0 ? 1.0 / (npair * s) : 0.0;
}

// d = k - v; gk = inv_z d; partial = inv_z |d|^2 per block
__global__ void __launch_bounds__(GTPB) ptc_loss_kernel(const InTab k, const InTab v, OutTab gk, const double* inv,
                                                        int64_t n4, double* partial) {
  __shared__ double sh[GTPB / 32];
  const int z = blockIdx.y;
  const float4* kp = reinterpret_cast<const float4*>(k.p[z * MAXC]);
  const float4* vp = reinterpret_cast<const float4*>(v.p[z * MAXC]);
  float4* gp = reinterpret_cast<float4*>(gk.p[z * MAXC]);
  const float w = (float)inv[z];
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * GTPB + threadIdx.x; i < n4; i += (int64_t)gridDim.x * GTPB) {
    float4 a = kp[i], b = vp[i];
    float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    s = fmaf(d.x, d.x, s); s = fmaf(d.y, d.y, s); s = fmaf(d.z, d.z, s); s = fmaf(d.w, d.w, s);
    gp[i] = make_float4(w * d.x, w * d.y, w * d.z, w * d.w);
  }
  double t = block_sum((double)s, sh);
  if (threadIdx.x == 0) partial[(size_t)z * gridDim.x + blockIdx.x] = t * inv[z];
}

__global__ void ptc_sum_kernel(const double* partial, int n, double* out) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += partial[i];
  *out = s;
}

// Adam (Kingma and Ba, Algorithm 1) on theta = (Re W, Im W) with gradient 2 dL/dconj(W);
// c1 = 1 - beta1^t, c2 = 1 - beta2^t
__global__ void ptc_adam_kernel(float* w, const double* g, float* m, float* v, int n, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gr = 2.0f * (float)g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gr;
  const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------- launch dispatch
template <int CIN, int COUT>
void layer_r(int recon, const LayerArg& a, int npair, cudaStream_t st) {
  dim3 grid((2 * a.g.Vh + TPB - 1) / TPB, npair);
  if (recon == 18) ptc_layer_kernel<CIN, COUT, 18><<<grid, TPB, 0, st>>>(a);
  else if (recon == 12) ptc_layer_kernel<CIN, COUT, 12><<<grid, TPB, 0, st>>>(a);
  else ptc_layer_kernel<CIN, COUT, 8><<<grid, TPB, 0, st>>>(a);
}
template <int CIN>
void layer_co(int cout, int recon, const LayerArg& a, int npair, cudaStream_t st) {
  if (cout == 1) layer_r<CIN, 1>(recon, a, npair, st);
  else if (cout == 2) layer_r<CIN, 2>(recon, a, npair, st);
  else layer_r<CIN, 4>(recon, a, npair, st);
}
void launch_layer(int cin, int cout, int recon, const LayerArg& a, int npair, cudaStream_t st) {
  if (cin == 1) layer_co<1>(cout, recon, a, npair, st);
  else if (cin == 2) layer_co<2>(cout, recon, a, npair, st);
  else layer_co<4>(cout, recon, a, npair, st);
}

template <int CIN, int COUT>
void wgrad_r(int recon, const GradArg& a, dim3 grid, cudaStream_t st) {
  if (recon == 18) ptc_wgrad_kernel<CIN, COUT, 18><<<grid, GTPB, 0, st>>>(a);
  else if (recon == 12) ptc_wgrad_kernel<CIN, COUT, 12><<<grid, GTPB, 0, st>>>(a);
  else ptc_wgrad_kernel<CIN, COUT, 8><<<grid, GTPB, 0, st>>>(a);
}
template <int CIN>
void wgrad_co(int cout, int recon, const GradArg& a, dim3 grid, cudaStream_t st) {
  if (cout == 1) wgrad_r<CIN, 1>(recon, a, grid, st);
  else if (cout == 2) wgrad_r<CIN, 2>(recon, a, grid, st);
  else wgrad_r<CIN, 4>(recon, a, grid, st);
}
void launch_wgrad(int cin, int cout, int recon, const GradArg& a, dim3 grid, cudaStream_t st) {
  if (cin == 1) wgrad_co<1>(cout, recon, a, grid, st);
  else if (cin == 2) wgrad_co<2>(cout, recon, a, grid, st);
  else wgrad_co<4>(cout, recon, a, grid, st);
}

bool valid_channels(int c) { return c == 1 || c == 2 || c == 4; }

}  // namespace
}  // namespace dirac

using namespace dirac;

struct dirac_ptc {
  dirac_ctx* c = nullptr;
  int L = 0;
  int ch[5] = {};
  size_t woff[5] = {};     // complex offset of each layer's weights; woff[L] = total
  float* w = nullptr;      // 2 * nw floats
  float* wadj = nullptr;   // one layer's adjoint weights
  double* grad = nullptr;  // 2 * nw
  float* am = nullptr;     // Adam moments
  float* av = nullptr;
  long long t = 0;         // Adam steps taken
  char* act = nullptr;     // per layer: activations and gradients of a batch
  size_t act_bytes = 0;
  float* partial = nullptr;
  size_t partial_bytes = 0;
  double* dsc = nullptr;   // [0, MAXB): inv; [MAXB]: loss; then norm / loss partials
  char* hid = nullptr;     // inference: two hidden-layer buffers of MAXC fields
  size_t fb = 0;           // bytes of one FP32 full field
  // tensor-core inference: BF16 weight images per layer, rebuilt after weight changes,
  // and a host-mapped flag the kernels set when a wait gave up
  int tc = 0;
  char* tcimg = nullptr;
  size_t tcoff[5] = {};
  bool tc_dirty = true;
  int* tc_err_h = nullptr;
  int* tc_err_d = nullptr;
  uint64_t tc_wait_ns = 2000000000ull;  // budget of each tensor-core pipeline wait
  int tc_stall = 0;                     // failure tests: the MMA warp stops issuing
};

namespace dirac {
namespace {

constexpr int DSC_PARTIAL = MAXB + 8;
constexpr int NORM_BLOCKS = 152;
constexpr size_t DSC_DOUBLES = DSC_PARTIAL + (size_t)MAXB * NORM_BLOCKS;

int net_err(dirac_ptc* n, int code, const char* msg) { return set_err(n->c, code, msg); }

int grow(dirac_ptc* n, char** p, size_t* have, size_t need) {
  if (*have >= need) return DIRAC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return net_err(n, DIRAC_ERR_OOM, "PTC workspace");
  }
  *have = need;
  return DIRAC_OK;
}

int check_net(dirac_ptc* n) {
  dirac_ctx* c = n->c;
  if (!c->gauge[P32] || !c->have_gauge) return net_err(n, DIRAC_ERR_STATE, "PTC: FP32 gauge field not loaded");
  return DIRAC_OK;
}

Geom geom(const dirac_ptc* n) { return n->c->g; }

// Layer l (1-based) on npair pairs: inputs in[z][c], outputs out[z][c].
void run_layer(dirac_ptc* n, int l, const float2* w, int cin, int cout, char* const* in, char* const* out,
               int npair, cudaStream_t st) {
  LayerArg a{};
  for (int z = 0; z < npair; ++z) {
    for (int c = 0; c < cin; ++c) a.in.p[z * MAXC + c] = in[z * MAXC + c];
    for (int c = 0; c < cout; ++c) a.out.p[z * MAXC + c] = out[z * MAXC + c];
  }
  a.w = w;
  a.gauge = n->c->gauge[P32];
  a.g = geom(n);
  launch_layer(cin, cout, n->c->p.recon[P32], a, npair, st);
  (void)l;
}

int wgrad(dirac_ptc* n, int l, char* const* x, char* const* gy, int npair, cudaStream_t st) {
  const int cin = n->ch[l - 1], cout = n->ch[l];
  const int Vh = n->c->g.Vh;
  const int maxblk = (2 * Vh + GTPB - 1) / GTPB;
  int nblk = (152 * 8 + NPATH * cout * npair - 1) / (NPATH * cout * npair);
  nblk = std::max(1, std::min(nblk, maxblk));
  size_t need = (size_t)npair * NPATH * cout * nblk * cin * 32 * sizeof(float);
  int rc = grow(n, reinterpret_cast<char**>(&n->partial), &n->partial_bytes, need);
  if (rc) return rc;
  GradArg a{};
  for (int z = 0; z < npair; ++z) {
    for (int c = 0; c < cin; ++c) a.x.p[z * MAXC + c] = x[z * MAXC + c];
    for (int c = 0; c < cout; ++c) a.gy.p[z * MAXC + c] = gy[z * MAXC + c];
  }
  a.partial = n->partial;
  a.gauge = n->c->gauge[P32];
  a.g = geom(n);
  launch_wgrad(cin, cout, n->c->p.recon[P32], a, dim3(nblk, NPATH * cout, npair), st);
  const int nv = NPATH * cout * cin * 32;
  ptc_wgrad_reduce<<<(nv + 127) / 128, 128, 0, st>>>(n->partial, nblk, npair, cout, cin,
                                                     n->grad + 2 * n->woff[l - 1]);
  return DIRAC_OK;
}

// Field pointers of the batch workspace: for layer l (1..L) activations act(l, z, c) and
// gradients gra(l, z, c), each npair x ch[l] fields.
struct Work {
  dirac_ptc* n;
  int npair;
  size_t layer_off[5];
  char* act(int l, int z, int c) const {
    return n->act + layer_off[l - 1] + ((size_t)z * n->ch[l] + c) * n->fb;
  }
  char* gra(int l, int z, int c) const {
    return n->act + layer_off[l - 1] + ((size_t)(npair + z) * n->ch[l] + c) * n->fb;
  }
};

int make_work(dirac_ptc* n, int npair, Work* w) {
  w->n = n;
  w->npair = npair;
  size_t off = 0;
  for (int l = 1; l <= n->L; ++l) {
    w->layer_off[l - 1] = off;
    off += (size_t)2 * npair * n->ch[l] * n->fb;
  }
  return grow(n, &n->act, &n->act_bytes, off);
}

// Forward over the batch (r[z] the inputs) storing every layer's output, then the loss
// against v[z] into dsc[MAXB] and, when grads is set, dL/dconj(W) of every layer.
int forward_backward(dirac_ptc* n, const Work& W, const char* const* r, const char* const* v, bool grads,
                     cudaStream_t st) {
  const int B = W.npair, L = n->L;
  const Geom g = geom(n);
  const int64_t n4 = (int64_t)12 * g.Vh;  // float4 chunks of a full FP32 field
  std::vector<char*> in(MAXB * MAXC), out(MAXB * MAXC);
  for (int l = 1; l <= L; ++l) {
    for (int z = 0; z < B; ++z) {
      for (int c = 0; c < n->ch[l - 1]; ++c)
        in[z * MAXC + c] = l == 1 ? const_cast<char*>(r[z]) : W.act(l - 1, z, c);
      for (int c = 0; c < n->ch[l]; ++c) out[z * MAXC + c] = W.act(l, z, c);
    }
    run_layer(n, l, reinterpret_cast<const float2*>(n->w) + n->woff[l - 1], n->ch[l - 1], n->ch[l], in.data(),
              out.data(), B, st);
  }
  // loss: inv_z = 1 / (B ||v_z||^2)
  InTab vt{}, kt{};
  OutTab gt{};
  for (int z = 0; z < B; ++z) {
    vt.p[z * MAXC] = v[z];
    kt.p[z * MAXC] = W.act(L, z, 0);
    gt.p[z * MAXC] = W.gra(L, z, 0);
  }
  double* part = n->dsc + DSC_PARTIAL;
  ptc_norm_kernel<<<dim3(NORM_BLOCKS, B), GTPB, 0, st>>>(vt, n4, part);
  ptc_inv_kernel<<<1, 32, 0, st>>>(part, NORM_BLOCKS, B, n->dsc);
  ptc_loss_kernel<<<dim3(NORM_BLOCKS, B), GTPB, 0, st>>>(kt, vt, gt, n->dsc, n4, part);
  ptc_sum_kernel<<<1, 1, 0, st>>>(part, NORM_BLOCKS * B, n->dsc + MAXB);
  if (!grads) return DIRAC_OK;
  for (int l = L; l >= 1; --l) {
    std::vector<char*> x(MAXB * MAXC), gy(MAXB * MAXC), gx(MAXB * MAXC);
    for (int z = 0; z < B; ++z) {
      for (int c = 0; c < n->ch[l - 1]; ++c) {
        x[z * MAXC + c] = l == 1 ? const_cast<char*>(r[z]) : W.act(l - 1, z, c);
        if (l > 1) gx[z * MAXC + c] = W.gra(l - 1, z, c);
      }
      for (int c = 0; c < n->ch[l]; ++c) gy[z * MAXC + c] = W.gra(l, z, c);
    }
    int rc = wgrad(n, l, x.data(), gy.data(), B, st);
    if (rc) return rc;
    if (l > 1) {
      const int cin = n->ch[l - 1], cout = n->ch[l];
      const int nw = NPATH * cout * cin * 16;
      ptc_adjoint_kernel<<<(nw + 127) / 128, 128, 0, st>>>(
          reinterpret_cast<const float2*>(n->w) + n->woff[l - 1], reinterpret_cast<float2*>(n->wadj), cout, cin);
      run_layer(n, l, reinterpret_cast<const float2*>(n->wadj), cout, cin, gy.data(), gx.data(), B, st);
    }
  }
  return DIRAC_OK;
}

int ptc_apply_tc(dirac_ptc* n, char* out, const char* in, cudaStream_t st) {
  if (*(volatile int*)n->tc_err_h) return net_err(n, DIRAC_ERR_TIMEOUT, "PTC tensor-core layer: a wait gave up");
  if (!n->hid && cudaMalloc(&n->hid, 2 * MAXC * n->fb) != cudaSuccess) {
    cudaGetLastError();
    n->hid = nullptr;
    return net_err(n, DIRAC_ERR_OOM, "PTC inference buffers");
  }
  if (n->tc_dirty) {
    for (int l = 1; l <= n->L; ++l)
      ptc_tc_pack(n->ch[l - 1], n->ch[l], reinterpret_cast<const float2*>(n->w) + n->woff[l - 1],
                  n->tcimg + n->tcoff[l - 1], st);
    n->tc_dirty = false;
  }
  for (int l = 1; l <= n->L; ++l) {
    const char* a[MAXC];
    char* b[MAXC];
    for (int c = 0; c < n->ch[l - 1]; ++c)
      a[c] = l == 1 ? in : n->hid + ((size_t)((l - 1) & 1) * MAXC + c) * n->fb;
    for (int c = 0; c < n->ch[l]; ++c) b[c] = l == n->L ? out : n->hid + ((size_t)(l & 1) * MAXC + c) * n->fb;
    int rc = ptc_tc_layer(n->ch[l - 1], n->ch[l], n->c->p.recon[P32], a, b, n->c->gauge[P32], n->tcimg + n->tcoff[l - 1],
                          geom(n), n->tc_err_d, n->tc_wait_ns, n->tc_stall, st);
    if (rc) return net_err(n, rc, "PTC tensor-core layer launch");
  }
  return cuda_check(n->c, "PTC apply (tensor cores)");
}

double layer_flops(int cin, int cout) {
  // 8 transports of min(cin, cout) spinors (4 SU(3) matvecs, 66 flops each) and
  // 9 x cin x cout spin mixes (16 x 3 complex multiply-adds, 8 flops each)
  return 8.0 * std::min(cin, cout) * 264.0 + 9.0 * cin * cout * 384.0;
}

}  // namespace

// ---------------------------------------------------------------- used by solvers.cu
int ptc_apply_internal(dirac_ptc* n, char* out, const char* in, cudaStream_t st) {
  if (!n) return DIRAC_ERR_STATE;
  int rc = check_net(n);
  if (rc) return rc;
  if (n->tc) return ptc_apply_tc(n, out, in, st);
  if (!n->hid) {
    if (cudaMalloc(&n->hid, 2 * MAXC * n->fb) != cudaSuccess) {
      cudaGetLastError();
      n->hid = nullptr;
      return net_err(n, DIRAC_ERR_OOM, "PTC inference buffers");
    }
  }
  std::vector<char*> a(MAXB * MAXC), b(MAXB * MAXC);
  for (int l = 1; l <= n->L; ++l) {
    for (int c = 0; c < n->ch[l - 1]; ++c)
      a[c] = l == 1 ? const_cast<char*>(in) : n->hid + ((size_t)((l - 1) & 1) * MAXC + c) * n->fb;
    for (int c = 0; c < n->ch[l]; ++c) b[c] = l == n->L ? out : n->hid + ((size_t)(l & 1) * MAXC + c) * n->fb;
    run_layer(n, l, reinterpret_cast<const float2*>(n->w) + n->woff[l - 1], n->ch[l - 1], n->ch[l], a.data(),
              b.data(), 1, st);
  }
  return cuda_check(n->c, "PTC apply");
}

double ptc_flops_per_apply(const dirac_ptc* n) {
  double f = 0;
  for (int l = 1; l <= n->L; ++l) f += layer_flops(n->ch[l - 1], n->ch[l]);
  return f * (double)n->c->V;
}

dirac_ctx* ptc_ctx(const dirac_ptc* n) { return n->c; }

void ptc_release(dirac_ptc* n) {
  if (!n) return;
  cudaFree(n->w);
  cudaFree(n->wadj);
  cudaFree(n->grad);
  cudaFree(n->am);
  cudaFree(n->av);
  cudaFree(n->act);
  cudaFree(n->partial);
  cudaFree(n->dsc);
  cudaFree(n->hid);
  cudaFree(n->tcimg);
  if (n->tc_err_h) cudaFreeHost(n->tc_err_h);
  delete n;
}

}  // namespace dirac

// ---------------------------------------------------------------- C ABI
extern "C" int dirac_ptc_create(dirac_ctx* c, const dirac_ptc_params* p, dirac_ptc** out) {
  if (!c || !p || !out) return set_err(c, DIRAC_ERR_ARG, "bad PTC arguments");
  *out = nullptr;
  if (c->p.kind != DIRAC_WILSON_CLOVER) return set_err(c, DIRAC_ERR_UNSUPPORTED, "PTC needs a Wilson-clover context");
  if (!(c->mask & (1u << P32))) return set_err(c, DIRAC_ERR_UNSUPPORTED, "PTC needs FP32 (prec_mask bit 1)");
  if (p->layers < 1 || p->layers > 4) return set_err(c, DIRAC_ERR_ARG, "PTC layers must be 1..4");
  if (p->channels[0] != 1 || p->channels[p->layers] != 1)
    return set_err(c, DIRAC_ERR_ARG, "PTC: first and last channel counts must be 1");
  for (int l = 0; l <= p->layers; ++l)
    if (!valid_channels(p->channels[l])) return set_err(c, DIRAC_ERR_ARG, "PTC channels must be 1, 2 or 4");
  dirac_ptc* n = new dirac_ptc();
  n->c = c;
  n->L = p->layers;
  size_t off = 0, maxl = 0;
  for (int l = 0; l <= n->L; ++l) n->ch[l] = p->channels[l];
  for (int l = 1; l <= n->L; ++l) {
    n->woff[l - 1] = off;
    size_t k = (size_t)NPATH * n->ch[l] * n->ch[l - 1] * 16;
    off += k;
    maxl = std::max(maxl, k);
  }
  n->woff[n->L] = off;
  n->fb = (size_t)192 * c->Vh;
  const size_t nw = off;
  bool ok = cudaMalloc(&n->w, nw * 8) == cudaSuccess && cudaMalloc(&n->wadj, maxl * 8) == cudaSuccess &&
            cudaMalloc(&n->grad, nw * 16) == cudaSuccess && cudaMalloc(&n->am, nw * 8) == cudaSuccess &&
            cudaMalloc(&n->av, nw * 8) == cudaSuccess &&
            cudaMalloc(&n->dsc, DSC_DOUBLES * sizeof(double)) == cudaSuccess;
  if (ok) {
    // K = 1: every layer passes channel 0 through on the local path
    std::vector<float> w0(2 * nw, 0.f);
    for (int l = 1; l <= n->L; ++l)
      for (int s = 0; s < 4; ++s) w0[2 * (n->woff[l - 1] + 5 * s)] = 1.f;
    ok = cudaMemcpy(n->w, w0.data(), nw * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(n->am, 0, nw * 8) == cudaSuccess && cudaMemset(n->av, 0, nw * 8) == cudaSuccess &&
         cudaMemset(n->grad, 0, nw * 16) == cudaSuccess;
  }
  size_t img = 0;
  for (int l = 1; l <= n->L; ++l) {
    n->tcoff[l - 1] = img;
    img += ptc_tc_image_bytes(n->ch[l - 1], n->ch[l]);
  }
  if (ok)
    ok = cudaMalloc(&n->tcimg, img) == cudaSuccess &&
         cudaHostAlloc(&n->tc_err_h, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostGetDevicePointer(&n->tc_err_d, n->tc_err_h, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ptc_release(n);
    return set_err(c, DIRAC_ERR_OOM, "PTC weights");
  }
  *n->tc_err_h = 0;
  c->ptcs.push_back(n);
  *out = n;
  return DIRAC_OK;
}

extern "C" long long dirac_ptc_num_weights(const dirac_ptc* n) { return n ? (long long)n->woff[n->L] : 0; }

extern "C" int dirac_ptc_set_weights(dirac_ptc* n, const double* w, long long cnt) {
  if (!n || !w) return DIRAC_ERR_ARG;
  if (cnt != (long long)n->woff[n->L]) return net_err(n, DIRAC_ERR_ARG, "PTC: wrong number of weights");
  std::vector<float> f(2 * cnt);
  for (long long i = 0; i < 2 * cnt; ++i) f[i] = (float)w[i];
  if (cudaMemcpy(n->w, f.data(), f.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_check(n->c, "PTC set weights");
  n->tc_dirty = true;
  // new weights start a new optimisation
  cudaMemset(n->am, 0, f.size() * 4);
  cudaMemset(n->av, 0, f.size() * 4);
  n->t = 0;
  return cuda_check(n->c, "PTC set weights");
}

extern "C" int dirac_ptc_get_weights(const dirac_ptc* n, double* w, long long cnt) {
  if (!n || !w) return DIRAC_ERR_ARG;
  dirac_ptc* m = const_cast<dirac_ptc*>(n);
  if (cnt != (long long)n->woff[n->L]) return net_err(m, DIRAC_ERR_ARG, "PTC: wrong number of weights");
  std::vector<float> f(2 * cnt);
  if (cudaMemcpy(f.data(), n->w, f.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check(m->c, "PTC get weights");
  for (long long i = 0; i < 2 * cnt; ++i) w[i] = f[i];
  return DIRAC_OK;
}

extern "C" int dirac_ptc_apply(dirac_ptc* n, void* out, const void* in, void* stream) {
  if (!n || !out || !in || out == in) return n ? net_err(n, DIRAC_ERR_ARG, "bad PTC apply arguments") : DIRAC_ERR_ARG;
  return ptc_apply_internal(n, (char*)out, (const char*)in, (cudaStream_t)stream);
}

extern "C" int dirac_ptc_gradient(dirac_ptc* n, const void* r, const void* v, double* loss, double* grad,
                                  void* stream) {
  if (!n || !r || !v) return n ? net_err(n, DIRAC_ERR_ARG, "bad PTC gradient arguments") : DIRAC_ERR_ARG;
  int rc = check_net(n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Work W;
  if ((rc = make_work(n, 1, &W))) return rc;
  const char* rr[1] = {(const char*)r};
  const char* vv[1] = {(const char*)v};
  if ((rc = forward_backward(n, W, rr, vv, grad != nullptr, st))) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(n->c, "PTC gradient");
  if (loss && cudaMemcpy(loss, n->dsc + MAXB, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check(n->c, "PTC gradient");
  if (grad && cudaMemcpy(grad, n->grad, 16 * n->woff[n->L], cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check(n->c, "PTC gradient");
  return cuda_check(n->c, "PTC gradient");
}

extern "C" int dirac_ptc_train(dirac_ptc* n, const void* const* r, const void* const* v, int npairs,
                               const dirac_ptc_train_params* P, double* loss, void* stream) {
  if (!n || !v || !P || npairs < 1) return n ? net_err(n, DIRAC_ERR_ARG, "bad PTC train arguments") : DIRAC_ERR_ARG;
  if (P->batch < 1 || P->batch > MAXB || P->steps < 0 || !(P->lr > 0) || !(P->beta1 >= 0 && P->beta1 < 1) ||
      !(P->beta2 >= 0 && P->beta2 < 1) || !(P->eps > 0))
    return net_err(n, DIRAC_ERR_ARG, "PTC: bad training parameters");
  int rc = check_net(n);
  if (rc) return rc;
  dirac_ctx* c = n->c;
  cudaStream_t st = (cudaStream_t)stream;
  const int B = std::min(P->batch, npairs);
  // r_i = M v_i (FP32) when the caller gives only v
  char* rbuf = nullptr;
  std::vector<const char*> rs(npairs);
  if (!r) {
    if (cudaMalloc(&rbuf, (size_t)npairs * n->fb) != cudaSuccess) {
      cudaGetLastError();
      return net_err(n, DIRAC_ERR_OOM, "PTC training pairs");
    }
    for (int i = 0; i < npairs; ++i) {
      if ((rc = apply_op(c, rbuf + (size_t)i * n->fb, (const char*)v[i], -1, P32, 0, st))) {
        cudaFree(rbuf);
        return rc;
      }
      rs[i] = rbuf + (size_t)i * n->fb;
    }
  } else {
    for (int i = 0; i < npairs; ++i) rs[i] = (const char*)r[i];
  }
  double* dloss = nullptr;
  if (P->steps > 0 && cudaMalloc(&dloss, P->steps * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(rbuf);
    return net_err(n, DIRAC_ERR_OOM, "PTC loss history");
  }
  Work W;
  if ((rc = make_work(n, B, &W))) {
    cudaFree(rbuf);
    cudaFree(dloss);
    return rc;
  }
  // visiting order: Fisher-Yates shuffles of the pairs, one per epoch
  std::mt19937 gen(P->seed);
  std::vector<int> order(npairs);
  for (int i = 0; i < npairs; ++i) order[i] = i;
  int pos = npairs;
  const int nw2 = (int)(2 * n->woff[n->L]);
  for (int s = 0; s < P->steps && rc == DIRAC_OK; ++s) {
    const char* rb[MAXB];
    const char* vb[MAXB];
    for (int z = 0; z < B; ++z) {
      if (pos == npairs) {
        for (int i = npairs - 1; i > 0; --i) std::swap(order[i], order[gen() % (unsigned)(i + 1)]);
        pos = 0;
      }
      const int i = order[pos++];
      rb[z] = rs[i];
      vb[z] = (const char*)v[i];
    }
    if ((rc = forward_backward(n, W, rb, vb, true, st))) break;
    n->tc_dirty = true;
    cudaMemcpyAsync(dloss + s, n->dsc + MAXB, sizeof(double), cudaMemcpyDeviceToDevice, st);
    n->t++;
    const double c1 = 1.0 - std::pow(P->beta1, (double)n->t), c2 = 1.0 - std::pow(P->beta2, (double)n->t);
    ptc_adam_kernel<<<(nw2 + 255) / 256, 256, 0, st>>>(n->w, n->grad, n->am, n->av, nw2, (float)P->lr,
                                                       (float)P->beta1, (float)P->beta2, (float)P->eps,
                                                       (float)c1, (float)c2);
  }
  if (rc == DIRAC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = cuda_check(c, "PTC train");
  if (rc == DIRAC_OK && loss && P->steps > 0 &&
      cudaMemcpy(loss, dloss, P->steps * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = cuda_check(c, "PTC train");
  cudaStreamSynchronize(st);
  cudaFree(dloss);
  cudaFree(rbuf);
  if (rc == DIRAC_OK) rc = cuda_check(c, "PTC train");
  return rc;
}

extern "C" int dirac_ptc_set_tensor_cores(dirac_ptc* n, int on) {
  if (!n || (on != 0 && on != 1)) return n ? net_err(n, DIRAC_ERR_ARG, "PTC: tensor cores on must be 0 or 1") : DIRAC_ERR_ARG;
  n->tc = on;
  *n->tc_err_h = 0;  // a new start after a wait that gave up
  return DIRAC_OK;
}

extern "C" int dirac_ptc_test_stall(dirac_ptc* n, int stall, double wait_seconds) {
  if (!n || (stall != 0 && stall != 1) || !(wait_seconds > 0) || wait_seconds > 60)
    return n ? net_err(n, DIRAC_ERR_ARG, "PTC test stall: bad arguments") : DIRAC_ERR_ARG;
  n->tc_stall = stall;
  n->tc_wait_ns = (uint64_t)(wait_seconds * 1e9);
  return DIRAC_OK;
}

extern "C" int dirac_ptc_attach(dirac_ctx* c, dirac_ptc* n, int force) {
  if (!c) return DIRAC_ERR_ARG;
  if (n && n->c != c) return set_err(c, DIRAC_ERR_ARG, "PTC network belongs to another context");
  if (force != 0 && force != 1) return set_err(c, DIRAC_ERR_ARG, "PTC attach: force must be 0 or 1");
  c->ptc_attached = n;
  c->ptc_force = force;
  return DIRAC_OK;
}

extern "C" int dirac_ptc_destroy(dirac_ptc* n) {
  if (!n) return DIRAC_OK;
  dirac_ctx* c = n->c;
  if (c->ptc_attached == n) c->ptc_attached = nullptr;
  c->ptcs.erase(std::remove(c->ptcs.begin(), c->ptcs.end(), n), c->ptcs.end());
  ptc_release(n);
  return cuda_check(c, "PTC destroy");
}
