// Domain decomposition of the Wilson-clover operator (Sec. 6), emulated on one GPU.
//
// The lattice is cut along t into P virtual ranks of LT/P time-slices (even, >= 2). Each
// rank owns its local links, clover and spinors in the library's chunk-major layout of
// its local volume, plus two ghost zones of one time-slice each:
//   ghost_fwd  the forward neighbour's first slice, spin-projected for the forward
//              t-hop: h = psi_up + s_f psi_low (B_t = 1), 12 reals per face site
//   ghost_bwd  the backward neighbour's last slice projected for the backward t-hop, and
//              (copied once at set-up, as the paper exchanges gauge ghosts once per solve)
//              the backward links U_t(x - t) of those face sites in the stored format.
// One application: every rank packs its two faces (its own stream), each face is copied
// into the neighbour's ghost zone (cudaMemcpyAsync device to device, after an event from
// the packing rank), and the stencil runs as two kernels per rank: the interior slices
// (no ghost needed, overlapping the exchange) and the two boundary slices once both
// ghosts have arrived. A site is computed entirely by one kernel, in the same operation
// order as the single-domain stencil (wilson_hop is reused; a projected ghost spinor
// enters as [h; 0], whose projection returns h exactly), so the result is bit-identical
// to dirac_apply on the whole lattice in FP64 and FP32. (With FP16 storage the compiler
// fuses the decode product, half x site norm, into different multiply-adds in the two
// kernels: the results then agree to FP32 rounding, one FP16 unit after re-encoding.)
// The fermion sign of hops across the global t edge is applied by the receiving rank
// (last rank forward, first rank backward). FP16 faces travel as FP32 projected values
// (the single-domain kernel projects in FP32).
#include <algorithm>
#include <vector>

#include "internal.h"
#include "wilson.cuh"

namespace dirac {
namespace {

constexpr int DD_THREADS = 128;

// Per-site layout of one plane: n arrays of e bytes per site, plus an optional array of
// 4-byte per-site scales (FP16 spinors and clover); planes k * 2 + parity, k < nk.
struct SiteLayout {
  int n, e, tail, nk;
  __host__ __device__ size_t plane_bytes(int Vh) const { return ((size_t)n * e + tail) * Vh; }
};

SiteLayout spinor_layout(int prec) {
  if (prec == P64) return {12, 16, 0, 1};
  if (prec == P32) return {6, 16, 0, 1};
  return {3, 16, 4, 1};
}
SiteLayout clover_layout(int prec) {
  if (prec == P64) return {36, 16, 0, 1};
  if (prec == P32) return {18, 16, 0, 1};
  return {9, 16, 4, 1};
}
SiteLayout link_layout(int prec, int recon) {
  int w = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
  int cb = prec == P64 ? 16 : prec == P32 ? (recon == 18 ? 8 : 16) : (recon == 18 ? 4 : (recon == 12 ? 8 : 16));
  return {recon * w / cb, cb, 0, 4};
}

__device__ __forceinline__ void copy_bytes(char* d, const char* s, int e) {
  if (e == 16) *reinterpret_cast<int4*>(d) = *reinterpret_cast<const int4*>(s);
  else if (e == 8) *reinterpret_cast<int2*>(d) = *reinterpret_cast<const int2*>(s);
  else *reinterpret_cast<int*>(d) = *reinterpret_cast<const int*>(s);
}

// Copy one field between the global layout and rank r's local layout (to_local: global
// -> local). One thread per local site.
__global__ void dd_copy_kernel(char* loc, const Geom gl, char* glob, const Geom gg, SiteLayout lay, int t0,
                               int to_local) {
  const int V = 2 * gl.Vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  int x[4];
  int r = i;
  x[0] = r % gl.L[0]; r /= gl.L[0];
  x[1] = r % gl.L[1]; r /= gl.L[1];
  x[2] = r % gl.L[2];
  x[3] = r / gl.L[2];
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;  // LT_loc even: local parity = global parity
  const int lcb = cb_index(gl, x);
  int y[4] = {x[0], x[1], x[2], x[3] + t0};
  const int gcb = cb_index(gg, y);
  const size_t lpb = lay.plane_bytes(gl.Vh), gpb = lay.plane_bytes(gg.Vh);
  for (int k = 0; k < lay.nk; ++k) {
    char* lp = loc + (size_t)(k * 2 + par) * lpb;
    char* gp = glob + (size_t)(k * 2 + par) * gpb;
    for (int j = 0; j < lay.n; ++j) {
      char* l = lp + ((size_t)j * gl.Vh + lcb) * lay.e;
      char* g = gp + ((size_t)j * gg.Vh + gcb) * lay.e;
      if (to_local) copy_bytes(l, g, lay.e);
      else copy_bytes(g, l, lay.e);
    }
    if (lay.tail) {
      char* l = lp + (size_t)lay.n * lay.e * gl.Vh + (size_t)lcb * 4;
      char* g = gp + (size_t)lay.n * lay.e * gg.Vh + (size_t)gcb * 4;
      if (to_local) copy_bytes(l, g, 4);
      else copy_bytes(g, l, 4);
    }
  }
}

// Face index of a site on a t-slice: (z * LY + y) * LX + x.
__device__ __forceinline__ int face_index(const Geom& g, const int x[4]) {
  return (x[2] * g.L[1] + x[1]) * g.L[0] + x[0];
}

// The t-links U_t of the last local slice into a face plane (chunk stride = face volume),
// read by the next rank for its backward t-hops.
__global__ void dd_pack_links_kernel(char* face, const char* links, const Geom gl, SiteLayout lay) {
  const int F = gl.L[0] * gl.L[1] * gl.L[2];
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= F) return;
  int x[4] = {fi % gl.L[0], (fi / gl.L[0]) % gl.L[1], fi / (gl.L[0] * gl.L[1]), gl.L[3] - 1};
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(gl, x);
  const char* plane = links + (size_t)(3 * 2 + par) * lay.plane_bytes(gl.Vh);
  for (int j = 0; j < lay.n; ++j)
    copy_bytes(face + ((size_t)j * F + fi) * lay.e, plane + ((size_t)j * gl.Vh + cb) * lay.e, lay.e);
}

template <int PREC>
struct Face {
  using T = typename Real<PREC>::T;
  // 12 reals per face site: h0 (3 complex), h1 (3 complex)
  static constexpr size_t site_bytes = 12 * sizeof(T);
};

// Pack both faces of a rank: slice 0 projected for the previous rank's forward hop
// (send_bwd) and slice LT_loc - 1 projected for the next rank's backward hop (send_fwd).
template <int PREC>
__global__ void dd_pack_kernel(char* send_bwd, char* send_fwd, const char* in, const Geom gl, int dagger) {
  using T = typename Real<PREC>::T;
  const int F = gl.L[0] * gl.L[1] * gl.L[2];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * F) return;
  const int side = i >= F, fi = i - side * F;  // side 0: slice 0, side 1: last slice
  int x[4] = {fi % gl.L[0], (fi / gl.L[0]) % gl.L[1], fi / (gl.L[0] * gl.L[1]), side ? gl.L[3] - 1 : 0};
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(gl, x);
  T psi[24];
  SpinorIO<PREC, 24>::load(in + (size_t)par * SpinorIO<PREC, 24>::half_bytes(gl.Vh), gl.Vh, cb, psi);
  const T sf = dagger ? (T)1 : (T)-1;
  const T s = side ? -sf : sf;  // slice 0 feeds a forward hop, the last slice a backward hop
  T* h = reinterpret_cast<T*>((side ? send_fwd : send_bwd) + (size_t)fi * Face<PREC>::site_bytes);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C<T> u0 = {psi[2 * c], psi[2 * c + 1]}, u1 = {psi[6 + 2 * c], psi[6 + 2 * c + 1]};
    C<T> l0 = {psi[12 + 2 * c], psi[12 + 2 * c + 1]}, l1 = {psi[18 + 2 * c], psi[18 + 2 * c + 1]};
    C<T> h0 = u0 + s * l0, h1 = u1 + s * l1;  // the t-projection of wilson_hop<3> (B_t = 1)
    h[2 * c] = h0.r; h[2 * c + 1] = h0.i;
    h[6 + 2 * c] = h1.r; h[6 + 2 * c + 1] = h1.i;
  }
}

struct DDArg {
  char* out;             // local full field
  const char* in;
  const char* gauge;     // local links
  const char* clover;    // local Ahat (null: 1)
  const char* ghost_fwd; // projected spinors of the next rank's slice 0
  const char* ghost_bwd; // projected spinors of the previous rank's last slice
  const char* ghost_links;  // U_t of the previous rank's last slice (face plane)
  Geom g;                // local geometry
  double kappa;
  int dagger;
  int first, last;       // this rank holds the global t = 0 / t = LT - 1 slice
  int apbc;
  int slice0, nslices;   // time-slices this launch computes
};

// M (or M^dagger) at one local site, the operation order of wilson_site<PREC,R,true>.
template <int PREC, int R>
__global__ void __launch_bounds__(WilsonShape<PREC>::threads, WilsonShape<PREC>::minb) dd_wilson_kernel(const DDArg a) {
  using T = typename Real<PREC>::T;
  const Geom& g = a.g;
  const int Vh = g.Vh, F = g.L[0] * g.L[1] * g.L[2];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.nslices * F) return;
  int x[4] = {i % g.L[0], (i / g.L[0]) % g.L[1], (i / (g.L[0] * g.L[1])) % g.L[2], a.slice0 + i / F};
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(g, x);
  const size_t hb = SpinorIO<PREC, 24>::half_bytes(Vh);
  const char* src = a.in + (size_t)(1 - par) * hb;
  const T sf = a.dagger ? (T)1 : (T)-1;
  const T sb = -sf;
  C<T> acc[4][3];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[s][c] = C<T>{0, 0};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    {  // forward neighbour
      T psi[24];
      T bc = 1;
      Link<T> U;
      LinkIO<PREC, R>::load(a.gauge, Vh, mu, par, cb, U);
      if (mu == 3 && x[3] == g.L[3] - 1) {
        const T* h = reinterpret_cast<const T*>(a.ghost_fwd + (size_t)face_index(g, x) * Face<PREC>::site_bytes);
#pragma unroll
        for (int k = 0; k < 12; ++k) { psi[k] = h[k]; psi[12 + k] = 0; }
        if (a.last && a.apbc) bc = -1;
        // [h; 0] projects to h + s 0 = h exactly
      } else {
        int y[4] = {x[0], x[1], x[2], x[3]};
        if (++y[mu] == g.L[mu]) y[mu] = 0;  // x, y, z are whole: periodic, no sign
        SpinorIO<PREC, 24>::load(src, Vh, cb_index(g, y), psi);
      }
      if (mu == 0) wilson_hop<0>(acc, psi, U, false, sf, bc);
      if (mu == 1) wilson_hop<1>(acc, psi, U, false, sf, bc);
      if (mu == 2) wilson_hop<2>(acc, psi, U, false, sf, bc);
      if (mu == 3) wilson_hop<3>(acc, psi, U, false, sf, bc);
    }
    {  // backward neighbour
      T psi[24];
      T bc = 1;
      Link<T> U;
      if (mu == 3 && x[3] == 0) {
        const int fi = face_index(g, x);
        const T* h = reinterpret_cast<const T*>(a.ghost_bwd + (size_t)fi * Face<PREC>::site_bytes);
#pragma unroll
        for (int k = 0; k < 12; ++k) { psi[k] = h[k]; psi[12 + k] = 0; }
        LinkIO<PREC, R>::template load_plane<true>(a.ghost_links, F, fi, U);
        if (a.first && a.apbc) bc = -1;
      } else {
        int y[4] = {x[0], x[1], x[2], x[3]};
        if (y[mu]-- == 0) y[mu] = g.L[mu] - 1;
        const int ycb = cb_index(g, y);
        SpinorIO<PREC, 24>::load(src, Vh, ycb, psi);
        LinkIO<PREC, R>::load(a.gauge, Vh, mu, 1 - par, ycb, U);
      }
      if (mu == 0) wilson_hop<0>(acc, psi, U, true, sb, bc);
      if (mu == 1) wilson_hop<1>(acc, psi, U, true, sb, bc);
      if (mu == 2) wilson_hop<2>(acc, psi, U, true, sb, bc);
      if (mu == 3) wilson_hop<3>(acc, psi, U, true, sb, bc);
    }
  }
  T self[24], out[24];
  SpinorIO<PREC, 24>::load(a.in + (size_t)par * hb, Vh, cb, self);
  C<T> sv[12], av[12];
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
  SpinorIO<PREC, 24>::store(a.out + (size_t)par * hb, Vh, cb, out);
}

template <int PREC>
void launch_dd(int recon, const DDArg& a, cudaStream_t st) {
  const int F = a.g.L[0] * a.g.L[1] * a.g.L[2];
  const int n = a.nslices * F;
  if (n <= 0) return;
  constexpr int T = WilsonShape<PREC>::threads;  // the single-domain kernel's launch shape
  dim3 grid((n + T - 1) / T);
  if (recon == 18) dd_wilson_kernel<PREC, 18><<<grid, T, 0, st>>>(a);
  else if (recon == 12) dd_wilson_kernel<PREC, 12><<<grid, T, 0, st>>>(a);
  else dd_wilson_kernel<PREC, 8><<<grid, T, 0, st>>>(a);
}

void launch_dd_any(int prec, int recon, const DDArg& a, cudaStream_t st) {
  if (prec == P64) launch_dd<P64>(recon, a, st);
  else if (prec == P32) launch_dd<P32>(recon, a, st);
  else launch_dd<P16>(recon, a, st);
}

void launch_pack_any(int prec, char* sb, char* sf, const char* in, const Geom& gl, int dagger, cudaStream_t st) {
  const int F = gl.L[0] * gl.L[1] * gl.L[2];
  dim3 grid((2 * F + DD_THREADS - 1) / DD_THREADS);
  if (prec == P64) dd_pack_kernel<P64><<<grid, DD_THREADS, 0, st>>>(sb, sf, in, gl, dagger);
  else if (prec == P32) dd_pack_kernel<P32><<<grid, DD_THREADS, 0, st>>>(sb, sf, in, gl, dagger);
  else dd_pack_kernel<P16><<<grid, DD_THREADS, 0, st>>>(sb, sf, in, gl, dagger);
}

size_t face_site_bytes(int prec) { return prec == P64 ? 96 : 48; }

}  // namespace
}  // namespace dirac

using namespace dirac;

struct dirac_dd {
  dirac_ctx* c = nullptr;
  int P = 0, prec = 0, recon = 0;
  Geom gl{};             // local geometry (identical on every rank)
  int F = 0;             // face sites
  struct Rank {
    char *gauge = nullptr, *clover = nullptr, *in = nullptr, *out = nullptr;
    char *send_fwd = nullptr, *send_bwd = nullptr, *ghost_fwd = nullptr, *ghost_bwd = nullptr;
    char* ghost_links = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t packed = nullptr, done = nullptr;
  };
  std::vector<Rank> r;
  cudaEvent_t start = nullptr;
};

namespace {

void dd_free(dirac_dd* d) {
  for (auto& k : d->r) {
    for (char* p : {k.gauge, k.clover, k.in, k.out, k.send_fwd, k.send_bwd, k.ghost_fwd, k.ghost_bwd, k.ghost_links})
      if (p) cudaFree(p);
    if (k.st) cudaStreamDestroy(k.st);
    if (k.packed) cudaEventDestroy(k.packed);
    if (k.done) cudaEventDestroy(k.done);
  }
  if (d->start) cudaEventDestroy(d->start);
  delete d;
}

int dd_copy(dirac_dd* d, int rank, char* loc, char* glob, SiteLayout lay, int to_local, cudaStream_t st) {
  const int V = 2 * d->gl.Vh;
  dd_copy_kernel<<<(V + DD_THREADS - 1) / DD_THREADS, DD_THREADS, 0, st>>>(loc, d->gl, glob, d->c->g, lay,
                                                                          rank * d->gl.L[3], to_local);
  return DIRAC_OK;
}

}  // namespace

extern "C" int dirac_dd_create(dirac_ctx* c, int nranks, dirac_prec prec, dirac_dd** out) {
  if (!c || !out) return set_err(c, DIRAC_ERR_ARG, "bad dd arguments");
  *out = nullptr;
  if (c->p.kind != DIRAC_WILSON_CLOVER) return set_err(c, DIRAC_ERR_UNSUPPORTED, "dd: Wilson-clover only");
  int rc = check_op(c, prec, false);
  if (rc) return rc;
  const int LT = c->p.dims[3];
  if (nranks < 1 || LT % nranks || (LT / nranks) % 2 || LT / nranks < 2)
    return set_err(c, DIRAC_ERR_ARG, "dd: LT / nranks must be an even integer >= 2");
  dirac_dd* d = new dirac_dd();
  d->c = c;
  d->P = nranks;
  d->prec = prec;
  d->recon = c->p.recon[prec];
  d->gl = c->g;
  d->gl.L[3] = LT / nranks;
  d->gl.Vh = c->g.Vh / nranks;
  d->F = c->p.dims[0] * c->p.dims[1] * c->p.dims[2];
  d->r.resize(nranks);
  const SiteLayout ls = spinor_layout(prec), lc = clover_layout(prec), ll = link_layout(prec, d->recon);
  const size_t sb = 2 * ls.plane_bytes(d->gl.Vh), cbytes = 2 * lc.plane_bytes(d->gl.Vh);
  const size_t lbytes = 8 * ll.plane_bytes(d->gl.Vh), fb = (size_t)d->F * face_site_bytes(prec);
  const size_t flb = (size_t)d->F * ll.n * ll.e;
  bool ok = cudaEventCreateWithFlags(&d->start, cudaEventDisableTiming) == cudaSuccess;
  const bool clov = c->clover[prec] != nullptr;
  for (auto& k : d->r) {
    ok = ok && cudaMalloc(&k.gauge, lbytes) == cudaSuccess && cudaMalloc(&k.in, sb) == cudaSuccess &&
         cudaMalloc(&k.out, sb) == cudaSuccess && cudaMalloc(&k.send_fwd, fb) == cudaSuccess &&
         cudaMalloc(&k.send_bwd, fb) == cudaSuccess && cudaMalloc(&k.ghost_fwd, fb) == cudaSuccess &&
         cudaMalloc(&k.ghost_bwd, fb) == cudaSuccess && cudaMalloc(&k.ghost_links, flb) == cudaSuccess &&
         (!clov || cudaMalloc(&k.clover, cbytes) == cudaSuccess) &&
         cudaStreamCreateWithFlags(&k.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&k.packed, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    dd_free(d);
    return set_err(c, DIRAC_ERR_OOM, "dd: rank storage");
  }
  // local links and clover from the context's storage; then the gauge ghosts: each rank
  // packs the t-links of its last slice and the next rank copies them in (once)
  for (int q = 0; q < nranks; ++q) {
    dd_copy(d, q, d->r[q].gauge, c->gauge[prec], ll, 1, nullptr);
    if (clov) dd_copy(d, q, d->r[q].clover, c->clover[prec], lc, 1, nullptr);
  }
  char* lface = nullptr;
  if (cudaMalloc(&lface, flb) != cudaSuccess) {
    cudaGetLastError();
    dd_free(d);
    return set_err(c, DIRAC_ERR_OOM, "dd: link face");
  }
  for (int q = 0; q < nranks; ++q) {
    const int nx = (q + 1) % nranks;
    dd_pack_links_kernel<<<(d->F + DD_THREADS - 1) / DD_THREADS, DD_THREADS>>>(lface, d->r[q].gauge, d->gl, ll);
    cudaMemcpy(d->r[nx].ghost_links, lface, flb, cudaMemcpyDeviceToDevice);
  }
  const bool synced = cudaDeviceSynchronize() == cudaSuccess;
  cudaFree(lface);
  if (!synced) {
    dd_free(d);
    return cuda_check(c, "dd create");
  }
  *out = d;
  return DIRAC_OK;
}

extern "C" int dirac_dd_scatter(dirac_dd* d, const void* in, void* stream) {
  if (!d || !in) return DIRAC_ERR_ARG;
  const SiteLayout ls = spinor_layout(d->prec);
  for (int q = 0; q < d->P; ++q)
    dd_copy(d, q, d->r[q].in, (char*)in, ls, 1, (cudaStream_t)stream);
  return cuda_check(d->c, "dd scatter");
}

extern "C" int dirac_dd_gather(dirac_dd* d, void* out, void* stream) {
  if (!d || !out) return DIRAC_ERR_ARG;
  const SiteLayout ls = spinor_layout(d->prec);
  for (int q = 0; q < d->P; ++q)
    dd_copy(d, q, d->r[q].out, (char*)out, ls, 0, (cudaStream_t)stream);
  return cuda_check(d->c, "dd gather");
}

extern "C" int dirac_dd_apply(dirac_dd* d, int dagger, void* stream) {
  if (!d || (dagger != 0 && dagger != 1)) return DIRAC_ERR_ARG;
  dirac_ctx* c = d->c;
  cudaStream_t caller = (cudaStream_t)stream;
  const int P = d->P;
  const size_t fb = (size_t)d->F * face_site_bytes(d->prec);
  cudaEventRecord(d->start, caller);
  // 1. pack (every rank, its own stream)
  for (int q = 0; q < P; ++q) {
    auto& k = d->r[q];
    cudaStreamWaitEvent(k.st, d->start, 0);
    launch_pack_any(d->prec, k.send_bwd, k.send_fwd, k.in, d->gl, dagger, k.st);
    cudaEventRecord(k.packed, k.st);
  }
  for (int q = 0; q < P; ++q) {
    auto& k = d->r[q];
    DDArg a{};
    a.out = k.out;
    a.in = k.in;
    a.gauge = k.gauge;
    a.clover = k.clover;
    a.ghost_fwd = k.ghost_fwd;
    a.ghost_bwd = k.ghost_bwd;
    a.ghost_links = k.ghost_links;
    a.g = d->gl;
    a.kappa = c->p.kappa;
    a.dagger = dagger;
    a.first = q == 0;
    a.last = q == P - 1;
    a.apbc = c->g.apbc;
    // 2. interior slices: no ghost needed, overlaps the exchange
    a.slice0 = 1;
    a.nslices = d->gl.L[3] - 2;
    launch_dd_any(d->prec, d->recon, a, k.st);
    // 3. exchange: the next rank's slice 0 and the previous rank's last slice
    const int nx = (q + 1) % P, pv = (q + P - 1) % P;
    cudaStreamWaitEvent(k.st, d->r[nx].packed, 0);
    cudaStreamWaitEvent(k.st, d->r[pv].packed, 0);
    cudaMemcpyAsync(k.ghost_fwd, d->r[nx].send_bwd, fb, cudaMemcpyDeviceToDevice, k.st);
    cudaMemcpyAsync(k.ghost_bwd, d->r[pv].send_fwd, fb, cudaMemcpyDeviceToDevice, k.st);
    // 4. the two boundary slices
    a.slice0 = 0;
    a.nslices = 1;
    launch_dd_any(d->prec, d->recon, a, k.st);
    a.slice0 = d->gl.L[3] - 1;
    launch_dd_any(d->prec, d->recon, a, k.st);
    cudaEventRecord(k.done, k.st);
  }
  // the send buffers may be repacked only after every neighbour copied them: the next
  // apply starts with the caller stream waiting for every rank
  for (int q = 0; q < P; ++q) cudaStreamWaitEvent(caller, d->r[q].done, 0);
  return cuda_check(c, "dd apply");
}

extern "C" int dirac_dd_info(const dirac_dd* d, int* local_dims, long long* face_bytes) {
  if (!d) return DIRAC_ERR_ARG;
  if (local_dims)
    for (int m = 0; m < 4; ++m) local_dims[m] = d->gl.L[m];
  if (face_bytes) *face_bytes = (long long)d->F * (long long)face_site_bytes(d->prec);
  return DIRAC_OK;
}

extern "C" int dirac_dd_destroy(dirac_dd* d) {
  if (!d) return DIRAC_OK;
  dirac_ctx* c = d->c;
  cudaDeviceSynchronize();
  dd_free(d);
  return cuda_check(c, "dd destroy");
}
