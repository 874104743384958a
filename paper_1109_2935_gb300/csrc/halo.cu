// Domain decomposition of the Wilson-clover operator (Sec. 6), emulated on one GPU.
//
// The lattice is cut by a 4-D grid of P = P_x P_y P_z P_t virtual ranks (Sec. 6.1-6.3:
// any subset of the four dimensions may be partitioned); every cut dimension keeps an
// even local extent >= 2. Each rank owns its local links, clover and spinors in the
// library's chunk-major layout of its local volume, and, for every cut dimension mu,
// two ghost zones of one slice each:
//   ghost_fwd[mu]  the forward neighbour's first mu-slice, spin-projected for the forward
//                  mu-hop: h = psi_up + s_f B_mu psi_low, 12 reals per face site
//   ghost_bwd[mu]  the backward neighbour's last mu-slice projected for the backward hop,
//                  and (copied once at set-up, as the paper exchanges gauge ghosts once per
//                  solve) the backward links U_mu(x - mu) of those face sites.
// One application: every rank packs its faces (its own stream), each face is copied into
// the neighbour's ghost zone (cudaMemcpyAsync device to device, after an event from the
// packing rank), and the stencil runs as one kernel over the interior box (no ghost
// needed, overlapping the exchange) and, once the ghosts have arrived, one kernel per
// cut dimension over the boundary sites whose first edge coordinate is in that
// dimension (disjoint boxes). A site is computed entirely by one kernel, in the same
// operation order as the single-domain stencil (wilson_hop is reused, and faces are
// projected by the stencil's own wilson_project; a projected ghost spinor enters as
// [h; 0], whose projection returns h exactly), so the result is bit-identical to
// dirac_apply on the whole lattice in FP64 and FP32. (With FP16 storage the
// single-domain kernel folds the neighbours' norms into the accumulation, this one
// decodes them first: the FP32 arithmetic differs by rounding and the re-encoded outputs
// agree to one FP16 unit in the last place per site.) Dimensions that are not cut wrap
// locally; the fermion sign of hops across the global t edge is applied by the rank that
// holds that edge. FP16 faces travel as FP32 projected values.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "wilson.cuh"

namespace dirac {
namespace {

constexpr int DD_THREADS = 128;
constexpr int DD_MAX_RANKS = 256;

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

// Copy one field between the global layout and a rank's local layout (to_local: global
// -> local); the rank's sub-lattice starts at global coordinates o. One thread per local
// site. The local extents are even, so a site's local parity is its global parity.
__global__ void dd_copy_kernel(char* loc, const Geom gl, char* glob, const Geom gg, SiteLayout lay, int4 o,
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
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int lcb = cb_index(gl, x);
  int y[4] = {x[0] + o.x, x[1] + o.y, x[2] + o.z, x[3] + o.w};
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

// Faces of dimension mu: the sites of one mu-slice, indexed lexicographically by the
// other three coordinates (lowest dimension fastest).
__host__ __device__ __forceinline__ int face_volume(const Geom& g, int mu) { return 2 * g.Vh / g.L[mu]; }
__device__ __forceinline__ int face_index(const Geom& g, const int x[4], int mu) {
  int idx = 0, stride = 1;
#pragma unroll
  for (int nu = 0; nu < 4; ++nu)
    if (nu != mu) {
      idx += x[nu] * stride;
      stride *= g.L[nu];
    }
  return idx;
}
__device__ __forceinline__ void face_coords(const Geom& g, int fi, int mu, int slice, int x[4]) {
#pragma unroll
  for (int nu = 0; nu < 4; ++nu)
    if (nu != mu) {
      x[nu] = fi % g.L[nu];
      fi /= g.L[nu];
    }
  x[mu] = slice;
}

// The mu-links of the last local mu-slice into a face plane (chunk stride = face
// volume), read by the next rank in mu for its backward mu-hops.
__global__ void dd_pack_links_kernel(char* face, const char* links, const Geom gl, SiteLayout lay, int mu) {
  const int F = face_volume(gl, mu);
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= F) return;
  int x[4];
  face_coords(gl, fi, mu, gl.L[mu] - 1, x);
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(gl, x);
  const char* plane = links + (size_t)(mu * 2 + par) * lay.plane_bytes(gl.Vh);
  for (int j = 0; j < lay.n; ++j)
    copy_bytes(face + ((size_t)j * F + fi) * lay.e, plane + ((size_t)j * gl.Vh + cb) * lay.e, lay.e);
}

template <int PREC>
struct Face {
  using T = typename Real<PREC>::T;
  // 12 reals per face site: h0 (3 complex), h1 (3 complex)
  static constexpr size_t site_bytes = 12 * sizeof(T);
};

// Pack both mu-faces of a rank: slice 0 projected for the previous rank's forward hop
// (send_bwd) and slice L_mu - 1 projected for the next rank's backward hop (send_fwd).
template <int PREC>
__global__ void dd_pack_kernel(char* send_bwd, char* send_fwd, const char* in, const Geom gl, int mu, int dagger) {
  using T = typename Real<PREC>::T;
  const int F = face_volume(gl, mu);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * F) return;
  const int side = i >= F, fi = i - side * F;  // side 0: slice 0, side 1: last slice
  int x[4];
  face_coords(gl, fi, mu, side ? gl.L[mu] - 1 : 0, x);
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int cb = cb_index(gl, x);
  T psi[24];
  SpinorIO<PREC, 24>::load(in + (size_t)par * SpinorIO<PREC, 24>::half_bytes(gl.Vh), gl.Vh, cb, psi);
  const T sf = dagger ? (T)1 : (T)-1;
  const T s = side ? -sf : sf;  // slice 0 feeds a forward hop, the last slice a backward hop
  C<T> h0[3], h1[3];
  if (mu == 0) wilson_project<0, T>(psi, s, h0, h1);
  else if (mu == 1) wilson_project<1, T>(psi, s, h0, h1);
  else if (mu == 2) wilson_project<2, T>(psi, s, h0, h1);
  else wilson_project<3, T>(psi, s, h0, h1);
  T* h = reinterpret_cast<T*>((side ? send_fwd : send_bwd) + (size_t)fi * Face<PREC>::site_bytes);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h[2 * c] = h0[c].r; h[2 * c + 1] = h0[c].i;
    h[6 + 2 * c] = h1[c].r; h[6 + 2 * c + 1] = h1[c].i;
  }
}

struct DDArg {
  char* out;                   // local full field
  const char* in;
  const char* gauge;           // local links
  const char* clover;          // local Ahat (null: 1)
  const char* ghost_fwd[4];    // per cut dimension: projected spinors of the next rank's slice 0
  const char* ghost_bwd[4];    // projected spinors of the previous rank's last slice
  const char* ghost_links[4];  // U_mu of the previous rank's last slice (face plane)
  Geom g;                      // local geometry
  double kappa;
  int dagger;
  int cut[4];                  // 1: dimension mu is partitioned (ghost zones), 0: local wrap
  int tfirst, tlast;           // this rank holds the global t = 0 / t = LT - 1 slice
  int apbc;
  int lo[4], n[4], step[4];    // the box of local sites this launch computes:
                               // x_mu = lo_mu + k step_mu, 0 <= k < n_mu
};

// M (or M^dagger) at one local site, the operation order of wilson_site<PREC,R,true>.
// CUT >= 0: the cut dimensions as a compile-time bit mask (bit mu), so that the ghost
// branches of whole dimensions are compiled out; CUT < 0: read from a.cut.
template <int PREC, int R, int CUT>
__global__ void __launch_bounds__(WilsonShape<PREC>::threads, WilsonShape<PREC>::minb) dd_wilson_kernel(const DDArg a) {
  using T = typename Real<PREC>::T;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n[0] * a.n[1] * a.n[2] * a.n[3]) return;
  int x[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    x[mu] = a.lo[mu] + (i % a.n[mu]) * a.step[mu];
    i /= a.n[mu];
  }
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
      const bool cut = CUT >= 0 ? ((CUT >> mu) & 1) != 0 : a.cut[mu] != 0;
      if (cut && x[mu] == g.L[mu] - 1) {
        const T* h = reinterpret_cast<const T*>(a.ghost_fwd[mu] + (size_t)face_index(g, x, mu) * Face<PREC>::site_bytes);
#pragma unroll
        for (int k = 0; k < 12; ++k) { psi[k] = h[k]; psi[12 + k] = 0; }
        if (mu == 3 && a.tlast && a.apbc) bc = -1;
        // [h; 0] projects to h + s B 0 = h exactly
      } else {
        int y[4] = {x[0], x[1], x[2], x[3]};
        if (++y[mu] == g.L[mu]) {  // a dimension that is not cut wraps on this rank
          y[mu] = 0;
          if (mu == 3 && a.apbc) bc = -1;
        }
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
      const bool cut = CUT >= 0 ? ((CUT >> mu) & 1) != 0 : a.cut[mu] != 0;
      if (cut && x[mu] == 0) {
        const int fi = face_index(g, x, mu);
        const T* h = reinterpret_cast<const T*>(a.ghost_bwd[mu] + (size_t)fi * Face<PREC>::site_bytes);
#pragma unroll
        for (int k = 0; k < 12; ++k) { psi[k] = h[k]; psi[12 + k] = 0; }
        LinkIO<PREC, R>::template load_plane<true>(a.ghost_links[mu], face_volume(g, mu), fi, U);
        if (mu == 3 && a.tfirst && a.apbc) bc = -1;
      } else {
        int y[4] = {x[0], x[1], x[2], x[3]};
        if (y[mu]-- == 0) {
          y[mu] = g.L[mu] - 1;
          if (mu == 3 && a.apbc) bc = -1;
        }
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

template <int PREC, int CUT>
void launch_dd_cut(int recon, const DDArg& a, dim3 grid, cudaStream_t st) {
  constexpr int T = WilsonShape<PREC>::threads;  // the single-domain kernel's launch shape
  if (recon == 18) dd_wilson_kernel<PREC, 18, CUT><<<grid, T, 0, st>>>(a);
  else if (recon == 12) dd_wilson_kernel<PREC, 12, CUT><<<grid, T, 0, st>>>(a);
  else dd_wilson_kernel<PREC, 8, CUT><<<grid, T, 0, st>>>(a);
}

template <int PREC>
void launch_dd(int recon, const DDArg& a, cudaStream_t st) {
  const long n = (long)a.n[0] * a.n[1] * a.n[2] * a.n[3];
  if (n <= 0) return;
  constexpr int T = WilsonShape<PREC>::threads;
  dim3 grid((unsigned)((n + T - 1) / T));
  const bool t_only = !a.cut[0] && !a.cut[1] && !a.cut[2] && a.cut[3];
  if (t_only) launch_dd_cut<PREC, 8>(recon, a, grid, st);  // t-slabs, the common case
  else launch_dd_cut<PREC, -1>(recon, a, grid, st);
}

void launch_dd_any(int prec, int recon, const DDArg& a, cudaStream_t st) {
  if (prec == P64) launch_dd<P64>(recon, a, st);
  else if (prec == P32) launch_dd<P32>(recon, a, st);
  else launch_dd<P16>(recon, a, st);
}

void launch_pack_any(int prec, char* sb, char* sf, const char* in, const Geom& gl, int mu, int dagger,
                     cudaStream_t st) {
  const int F = face_volume(gl, mu);
  dim3 grid((2 * F + DD_THREADS - 1) / DD_THREADS);
  if (prec == P64) dd_pack_kernel<P64><<<grid, DD_THREADS, 0, st>>>(sb, sf, in, gl, mu, dagger);
  else if (prec == P32) dd_pack_kernel<P32><<<grid, DD_THREADS, 0, st>>>(sb, sf, in, gl, mu, dagger);
  else dd_pack_kernel<P16><<<grid, DD_THREADS, 0, st>>>(sb, sf, in, gl, mu, dagger);
}

size_t face_site_bytes(int prec) { return prec == P64 ? 96 : 48; }

}  // namespace
}  // namespace dirac

using namespace dirac;

struct dirac_dd {
  dirac_ctx* c = nullptr;
  int P = 0, prec = 0, recon = 0;
  int grid[4] = {1, 1, 1, 1};  // ranks per dimension
  Geom gl{};                   // local geometry (identical on every rank)
  int F[4] = {0, 0, 0, 0};     // face sites per dimension
  struct Rank {
    int co[4] = {0, 0, 0, 0};  // coordinates in the rank grid
    char *gauge = nullptr, *clover = nullptr, *in = nullptr, *out = nullptr;
    char* send_fwd[4] = {};
    char* send_bwd[4] = {};
    char* ghost_fwd[4] = {};
    char* ghost_bwd[4] = {};
    char* ghost_links[4] = {};
    cudaStream_t st = nullptr;
    cudaEvent_t packed = nullptr, done = nullptr;
  };
  std::vector<Rank> r;
  cudaEvent_t start = nullptr;
  int rank_of(const int co[4]) const { return co[0] + grid[0] * (co[1] + grid[1] * (co[2] + grid[2] * co[3])); }
  // the neighbour of rank q one step along +mu (dir = +1) or -mu (dir = -1), periodic
  int neighbour(int q, int mu, int dir) const {
    int co[4] = {r[q].co[0], r[q].co[1], r[q].co[2], r[q].co[3]};
    co[mu] = (co[mu] + dir + grid[mu]) % grid[mu];
    return rank_of(co);
  }
};

namespace {

void dd_free(dirac_dd* d) {
  for (auto& k : d->r) {
    for (char* p : {k.gauge, k.clover, k.in, k.out})
      if (p) cudaFree(p);
    for (int mu = 0; mu < 4; ++mu)
      for (char* p : {k.send_fwd[mu], k.send_bwd[mu], k.ghost_fwd[mu], k.ghost_bwd[mu], k.ghost_links[mu]})
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
  const int* co = d->r[rank].co;
  const int4 o = make_int4(co[0] * d->gl.L[0], co[1] * d->gl.L[1], co[2] * d->gl.L[2], co[3] * d->gl.L[3]);
  dd_copy_kernel<<<(V + DD_THREADS - 1) / DD_THREADS, DD_THREADS, 0, st>>>(loc, d->gl, glob, d->c->g, lay, o,
                                                                          to_local);
  return DIRAC_OK;
}

}  // namespace

extern "C" int dirac_dd_create_grid(dirac_ctx* c, const int* grid, dirac_prec prec, dirac_dd** out) {
  if (!c || !out || !grid) return set_err(c, DIRAC_ERR_ARG, "bad dd arguments");
  *out = nullptr;
  if (c->p.kind != DIRAC_WILSON_CLOVER) return set_err(c, DIRAC_ERR_UNSUPPORTED, "dd: Wilson-clover only");
  int rc = check_op(c, prec, false);
  if (rc) return rc;
  int P = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int L = c->p.dims[mu], g = grid[mu];
    if (g < 1 || L % g || (L / g) % 2 || L / g < 2)
      return set_err(c, DIRAC_ERR_ARG, "dd: every L_mu / grid_mu must be an even integer >= 2");
    P *= g;
  }
  if (P > DD_MAX_RANKS) return set_err(c, DIRAC_ERR_ARG, "dd: at most 256 virtual ranks");
  dirac_dd* d = new dirac_dd();
  d->c = c;
  d->P = P;
  d->prec = prec;
  d->recon = c->p.recon[prec];
  d->gl = c->g;
  for (int mu = 0; mu < 4; ++mu) {
    d->grid[mu] = grid[mu];
    d->gl.L[mu] = c->p.dims[mu] / grid[mu];
  }
  d->gl.Lxh = d->gl.L[0] / 2;
  d->gl.Vh = c->g.Vh / P;
  for (int mu = 0; mu < 4; ++mu) d->F[mu] = face_volume(d->gl, mu);
  d->r.resize(P);
  for (int q = 0; q < P; ++q) {
    int rem = q;
    for (int mu = 0; mu < 4; ++mu) {
      d->r[q].co[mu] = rem % grid[mu];
      rem /= grid[mu];
    }
  }
  const SiteLayout ls = spinor_layout(prec), lc = clover_layout(prec), ll = link_layout(prec, d->recon);
  const size_t sb = 2 * ls.plane_bytes(d->gl.Vh), cbytes = 2 * lc.plane_bytes(d->gl.Vh);
  const size_t lbytes = 8 * ll.plane_bytes(d->gl.Vh);
  bool ok = cudaEventCreateWithFlags(&d->start, cudaEventDisableTiming) == cudaSuccess;
  const bool clov = c->clover[prec] != nullptr;
  for (auto& k : d->r) {
    ok = ok && cudaMalloc(&k.gauge, lbytes) == cudaSuccess && cudaMalloc(&k.in, sb) == cudaSuccess &&
         cudaMalloc(&k.out, sb) == cudaSuccess && (!clov || cudaMalloc(&k.clover, cbytes) == cudaSuccess) &&
         cudaStreamCreateWithFlags(&k.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&k.packed, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming) == cudaSuccess;
    for (int mu = 0; mu < 4 && ok; ++mu) {
      if (grid[mu] == 1) continue;
      const size_t fb = (size_t)d->F[mu] * face_site_bytes(prec), flb = (size_t)d->F[mu] * ll.n * ll.e;
      ok = cudaMalloc(&k.send_fwd[mu], fb) == cudaSuccess && cudaMalloc(&k.send_bwd[mu], fb) == cudaSuccess &&
           cudaMalloc(&k.ghost_fwd[mu], fb) == cudaSuccess && cudaMalloc(&k.ghost_bwd[mu], fb) == cudaSuccess &&
           cudaMalloc(&k.ghost_links[mu], flb) == cudaSuccess;
    }
  }
  if (!ok) {
    cudaGetLastError();
    dd_free(d);
    return set_err(c, DIRAC_ERR_OOM, "dd: rank storage");
  }
  // local links and clover from the context's storage; then the gauge ghosts: for every
  // cut dimension each rank packs the mu-links of its last mu-slice and the next rank in
  // mu copies them in (once)
  for (int q = 0; q < P; ++q) {
    dd_copy(d, q, d->r[q].gauge, c->gauge[prec], ll, 1, nullptr);
    if (clov) dd_copy(d, q, d->r[q].clover, c->clover[prec], lc, 1, nullptr);
  }
  for (int mu = 0; mu < 4; ++mu) {
    if (grid[mu] == 1) continue;
    const size_t flb = (size_t)d->F[mu] * ll.n * ll.e;
    char* lface = nullptr;
    if (cudaMalloc(&lface, flb) != cudaSuccess) {
      cudaGetLastError();
      dd_free(d);
      return set_err(c, DIRAC_ERR_OOM, "dd: link face");
    }
    for (int q = 0; q < P; ++q) {
      dd_pack_links_kernel<<<(d->F[mu] + DD_THREADS - 1) / DD_THREADS, DD_THREADS>>>(lface, d->r[q].gauge, d->gl,
                                                                                     ll, mu);
      cudaMemcpy(d->r[d->neighbour(q, mu, 1)].ghost_links[mu], lface, flb, cudaMemcpyDeviceToDevice);
    }
    cudaFree(lface);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    dd_free(d);
    return cuda_check(c, "dd create");
  }
  *out = d;
  return DIRAC_OK;
}

extern "C" int dirac_dd_create(dirac_ctx* c, int nranks, dirac_prec prec, dirac_dd** out) {
  const int grid[4] = {1, 1, 1, nranks};
  return dirac_dd_create_grid(c, grid, prec, out);
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
  cudaEventRecord(d->start, caller);
  // 1. pack every cut dimension's two faces (every rank, its own stream)
  for (int q = 0; q < P; ++q) {
    auto& k = d->r[q];
    cudaStreamWaitEvent(k.st, d->start, 0);
    for (int mu = 0; mu < 4; ++mu)
      if (d->grid[mu] > 1) launch_pack_any(d->prec, k.send_bwd[mu], k.send_fwd[mu], k.in, d->gl, mu, dagger, k.st);
    cudaEventRecord(k.packed, k.st);
  }
  for (int q = 0; q < P; ++q) {
    auto& k = d->r[q];
    DDArg a{};
    a.out = k.out;
    a.in = k.in;
    a.gauge = k.gauge;
    a.clover = k.clover;
    for (int mu = 0; mu < 4; ++mu) {
      a.ghost_fwd[mu] = k.ghost_fwd[mu];
      a.ghost_bwd[mu] = k.ghost_bwd[mu];
      a.ghost_links[mu] = k.ghost_links[mu];
      a.cut[mu] = d->grid[mu] > 1;
    }
    a.g = d->gl;
    a.kappa = c->p.kappa;
    a.dagger = dagger;
    a.tfirst = k.co[3] == 0;
    a.tlast = k.co[3] == d->grid[3] - 1;
    a.apbc = c->g.apbc;
    // 2. the interior box (1 .. L_mu - 2 in every cut dimension): no ghost needed, overlaps
    //    the exchange
    for (int mu = 0; mu < 4; ++mu) {
      a.lo[mu] = a.cut[mu] ? 1 : 0;
      a.n[mu] = a.cut[mu] ? d->gl.L[mu] - 2 : d->gl.L[mu];
      a.step[mu] = 1;
    }
    launch_dd_any(d->prec, d->recon, a, k.st);
    // 3. exchange: for every cut dimension the next rank's first slice and the previous
    //    rank's last slice
    for (int mu = 0; mu < 4; ++mu) {
      if (!a.cut[mu]) continue;
      const int nx = d->neighbour(q, mu, 1), pv = d->neighbour(q, mu, -1);
      const size_t fb = (size_t)d->F[mu] * face_site_bytes(d->prec);
      cudaStreamWaitEvent(k.st, d->r[nx].packed, 0);
      cudaStreamWaitEvent(k.st, d->r[pv].packed, 0);
      cudaMemcpyAsync(k.ghost_fwd[mu], d->r[nx].send_bwd[mu], fb, cudaMemcpyDeviceToDevice, k.st);
      cudaMemcpyAsync(k.ghost_bwd[mu], d->r[pv].send_fwd[mu], fb, cudaMemcpyDeviceToDevice, k.st);
    }
    // 4. the boundary: box m holds the sites on an edge of cut dimension m that are
    //    interior in every cut dimension before m (disjoint, together every edge site)
    for (int m = 0; m < 4; ++m) {
      if (!a.cut[m]) continue;
      for (int mu = 0; mu < 4; ++mu) {
        if (mu < m && a.cut[mu]) {
          a.lo[mu] = 1; a.n[mu] = d->gl.L[mu] - 2; a.step[mu] = 1;
        } else if (mu == m) {
          a.lo[mu] = 0; a.n[mu] = 2; a.step[mu] = d->gl.L[mu] - 1;
        } else {
          a.lo[mu] = 0; a.n[mu] = d->gl.L[mu]; a.step[mu] = 1;
        }
      }
      launch_dd_any(d->prec, d->recon, a, k.st);
    }
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
  if (face_bytes) {
    long long fb = 0;
    for (int mu = 0; mu < 4; ++mu)
      if (d->grid[mu] > 1) fb += 2LL * d->F[mu] * (long long)face_site_bytes(d->prec);
    *face_bytes = fb;
  }
  return DIRAC_OK;
}

extern "C" int dirac_dd_destroy(dirac_dd* d) {
  if (!d) return DIRAC_OK;
  dirac_ctx* c = d->c;
  cudaDeviceSynchronize();
  dd_free(d);
  return cuda_check(c, "dd destroy");
}
