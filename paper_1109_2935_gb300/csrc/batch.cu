// Batched application of the Wilson-clover operator: many right-hand sides on one
// lattice, and several lattices of different sizes, in one persistent launch.
//
// A CTA works on tiles of 32 sites x RG right-hand sides (blockDim = (32, RG)): warp y
// applies M to right-hand side rg*RG + y on the tile's 32 sites, so the links and the
// clover of those sites are fetched from DRAM once and served to the other RG-1 warps
// from L1. Every output site runs the same stencil code as the single-RHS kernel, so
// results are bitwise identical. The tile shape (RG and the number of resident CTAs)
// is chosen per batch plan by timing the candidates once (the autotuner below), and a
// plan can record its launches in a CUDA graph for replay. With FP16 storage the plan
// also times the tensor-core kernel of mrhs_tc.cu (all right-hand sides of a site in
// one dense contraction) and keeps the faster of the two.
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"
#include "mrhs_tc.h"
#include "wilson_ds.cuh"
#include "wilson.cuh"

namespace dirac {

static constexpr int kTileSites = 32;
static constexpr int kMaxRG = 16;
static constexpr int kMaxLat = 16;

// one lattice of a batch, as the kernel sees it
struct BatchLat {
  Geom g;
  const char* gauge;
  const char* clover;
  double kappa;
  const char* in;       // nrhs consecutive full fields
  char* out;
  size_t field_bytes;
  int nrhs;
  int tiles_site;       // 32-site groups over the 2 Vh output sites
  int tiles;            // tiles_site * ceil(nrhs / RG)
  int tile_begin;       // first tile of this lattice in the batch
  int rhs0;             // plan-wide index of this lattice's first right-hand side
  const double* mask;   // null, or mask[(rhs0 + r) * mstride] == 0: right-hand side r is skipped
  int mstride;
};

template <int PREC, int R>
__device__ __forceinline__ void batch_tile(const BatchLat& L, int t, int RG) {
  const int rgroups_site = L.tiles_site;
  const int rg = t / rgroups_site, sg = t - rg * rgroups_site;
  const int rhs = rg * RG + threadIdx.y;
  if (rhs >= L.nrhs) return;
  if (L.mask && L.mask[(size_t)(L.rhs0 + rhs) * L.mstride] == 0.0) return;
  WilsonArg a;
  a.g = L.g;
  a.gauge = L.gauge;
  a.clover = L.clover;
  a.kappa = L.kappa;
  a.dagger = 0;
  a.out_parity = 0;
  const size_t hb = L.field_bytes / 2;
  const char* in = L.in + (size_t)rhs * L.field_bytes;
  char* out = L.out + (size_t)rhs * L.field_bytes;
  a.in[0] = in;
  a.in[1] = in + hb;
  a.out[0] = out;
  a.out[1] = out + hb;
  wilson_site<PREC, R, true>(a, sg * kTileSites + threadIdx.x);
}

// one lattice, descriptor by value
template <int PREC, int R>
__global__ void __launch_bounds__(kTileSites * kMaxRG, 1) mrhs_kernel(const BatchLat L, int RG) {
  for (int t = blockIdx.x; t < L.tiles; t += gridDim.x) batch_tile<PREC, R>(L, t, RG);
}

// several lattices: descriptor table in device memory, tiles numbered across lattices
template <int PREC, int R>
__global__ void __launch_bounds__(kTileSites * kMaxRG, 1)
    batch_kernel(const BatchLat* __restrict__ lats, int nlat, int ntiles, int RG) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int l = 0;
    while (l + 1 < nlat && t >= lats[l + 1].tile_begin) ++l;
    const BatchLat L = lats[l];
    batch_tile<PREC, R>(L, t - L.tile_begin, RG);
  }
}

// the double-single form (FP64 fields): 4 right-hand sides per CTA (the untimed default
// shape), so that a thread may hold the float-float values in up to 255 registers
__global__ void __launch_bounds__(kTileSites * 4, 1)
    batch_kernel_ds(const BatchLat* __restrict__ lats, int nlat, int ntiles) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int l = 0;
    while (l + 1 < nlat && t >= lats[l + 1].tile_begin) ++l;
    const BatchLat L = lats[l];
    batch_tile<P64DS, 18>(L, t - L.tile_begin, 4);
  }
}

template <int PREC>
static void launch_mrhs_prec(int recon, const BatchLat& L, int RG, int grid, cudaStream_t st) {
  dim3 block(kTileSites, RG);
  if (recon == 18) mrhs_kernel<PREC, 18><<<grid, block, 0, st>>>(L, RG);
  else if (recon == 12) mrhs_kernel<PREC, 12><<<grid, block, 0, st>>>(L, RG);
  else mrhs_kernel<PREC, 8><<<grid, block, 0, st>>>(L, RG);
}
template <int PREC>
static void launch_batch_prec(int recon, const BatchLat* d, int nlat, int ntiles, int RG, int grid,
                              cudaStream_t st) {
  dim3 block(kTileSites, RG);
  if (recon == 18) batch_kernel<PREC, 18><<<grid, block, 0, st>>>(d, nlat, ntiles, RG);
  else if (recon == 12) batch_kernel<PREC, 12><<<grid, block, 0, st>>>(d, nlat, ntiles, RG);
  else batch_kernel<PREC, 8><<<grid, block, 0, st>>>(d, nlat, ntiles, RG);
}

static BatchLat describe(const dirac_ctx* c, int prec, const void* in, void* out, int nrhs, int RG) {
  BatchLat L;
  L.g = c->g;
  L.gauge = c->gauge[prec];
  L.clover = c->p.csw != 0.0 ? c->clover[prec] : nullptr;
  L.kappa = c->p.kappa;
  L.in = (const char*)in;
  L.out = (char*)out;
  L.field_bytes = 2 * spinor_half_bytes(prec, 24, c->Vh);
  L.nrhs = nrhs;
  L.tiles_site = (int)((2 * c->Vh + kTileSites - 1) / kTileSites);
  L.tiles = L.tiles_site * ((nrhs + RG - 1) / RG);
  L.tile_begin = 0;
  L.rhs0 = 0;
  L.mask = nullptr;
  L.mstride = 0;
  return L;
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// CTAs for a shape: `per_sm` resident CTAs on every SM, no more than the tiles
static int grid_for(int per_sm, int tiles) {
  long g = (long)sm_count() * per_sm;
  return (int)(g < tiles ? g : tiles);
}

}  // namespace dirac

using namespace dirac;

struct dirac_batch {
  std::vector<dirac_ctx*> ctxs;
  std::vector<BatchLat> lats;    // host copy (RG-dependent fields refreshed by the tuner)
  BatchLat* d_lats = nullptr;    // device table
  int prec = 0, recon = 12, ntiles = 0;
  bool ds = false;               // FP64 fields: double-single arithmetic (18-real links)
  int RG = 1, per_sm = 1, grid = 1;
  double tuned_ms = 0;
  std::vector<double> cand_ms;   // autotuner timings, candidate order
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_napply = 0;
  // tensor-core kernel (FP16 storage): its lattice table, grid and creation timing
  bool use_tc = false;
  TcLat* d_tc = nullptr;
  std::vector<int*> tc_nbr;      // per-lattice neighbour tables of the tensor-core kernel
  int tc_ntiles = 0, tc_grid = 0;
  double tc_ms = -1, cc_ms = -1;
  std::string err;
};

namespace dirac {

// the tile-shape candidates: (right-hand sides per CTA, resident CTAs per SM)
static const int kCand[][2] = {{1, 16}, {2, 8}, {4, 4}, {8, 2}, {16, 1}, {2, 16}, {4, 8}, {8, 4}};
static constexpr int kDefaultCand = 2;  // the shape the full tuning picks on the batched workloads

static int batch_layout(dirac_batch* b, int RG, cudaStream_t st) {
  int begin = 0;
  for (size_t l = 0; l < b->lats.size(); ++l) {
    BatchLat& L = b->lats[l];
    L.tiles = L.tiles_site * ((L.nrhs + RG - 1) / RG);
    L.tile_begin = begin;
    begin += L.tiles;
  }
  b->ntiles = begin;
  // pageable source: the copy is staged before the call returns, so the host vector
  // may change afterwards
  if (cudaMemcpyAsync(b->d_lats, b->lats.data(), sizeof(BatchLat) * b->lats.size(), cudaMemcpyHostToDevice,
                      st) != cudaSuccess) {
    b->err = "descriptor copy failed";
    return DIRAC_ERR_CUDA;
  }
  return DIRAC_OK;
}

static void batch_launch_direct(dirac_batch* b, cudaStream_t st) {
  const int nlat = (int)b->lats.size();
  if (b->use_tc) {
    launch_mrhs_tc(b->recon, b->d_tc, nlat, b->tc_ntiles, b->tc_grid, st);
    return;
  }
  if (b->prec == P64 && b->ds)
    batch_kernel_ds<<<b->grid, dim3(kTileSites, 4), 0, st>>>(b->d_lats, nlat, b->ntiles);
  else if (b->prec == P64) launch_batch_prec<P64>(b->recon, b->d_lats, nlat, b->ntiles, b->RG, b->grid, st);
  else if (b->prec == P32) launch_batch_prec<P32>(b->recon, b->d_lats, nlat, b->ntiles, b->RG, b->grid, st);
  else launch_batch_prec<P16>(b->recon, b->d_lats, nlat, b->ntiles, b->RG, b->grid, st);
}

}  // namespace dirac

extern "C" {

int dirac_apply_multi(dirac_ctx* c, void* out, const void* in, int nrhs, dirac_prec prec, void* stream) {
  int rc = check_op(c, prec, false);
  if (rc) return rc;
  if (c->p.kind != DIRAC_WILSON_CLOVER)
    return set_err(c, DIRAC_ERR_UNSUPPORTED, "multi-RHS apply is defined for Wilson-clover");
  if (!out || !in || nrhs < 1) return set_err(c, DIRAC_ERR_ARG, "bad multi-RHS arguments");
  const size_t fb = 2 * spinor_half_bytes(prec, 24, c->Vh);
  const char *i0 = (const char*)in, *o0 = (const char*)out;
  if (i0 < o0 + fb * nrhs && o0 < i0 + fb * nrhs) return set_err(c, DIRAC_ERR_ARG, "in and out overlap");
  const int RG = nrhs < kMaxRG ? nrhs : kMaxRG;
  BatchLat L = describe(c, prec, in, out, nrhs, RG);
  const int per_sm = kMaxRG / RG;  // 16 resident warps per SM at the 128-register cap
  const int grid = grid_for(per_sm, L.tiles);
  cudaStream_t st = (cudaStream_t)stream;
  if ((int)prec == P64) launch_mrhs_prec<P64>(c->p.recon[prec], L, RG, grid, st);
  else if ((int)prec == P32) launch_mrhs_prec<P32>(c->p.recon[prec], L, RG, grid, st);
  else launch_mrhs_prec<P16>(c->p.recon[prec], L, RG, grid, st);
  return cuda_check(c, "multi-RHS kernel");
}

int dirac_batch_create(dirac_ctx* const* ctxs, int nlat, void* const* out, const void* const* in,
                       const int* nrhs, dirac_prec prec, void* stream, dirac_batch** plan) {
  return dirac::batch_create(ctxs, nlat, out, in, nrhs, prec, (cudaStream_t)stream, plan, 2, false);
}

}  // extern "C"

namespace dirac {

int batch_create(dirac_ctx* const* ctxs, int nlat, void* const* out, const void* const* in, const int* nrhs,
                 int prec, cudaStream_t stream, dirac_batch** plan, int tune, bool ds) {
  if (!ctxs || !out || !in || !nrhs || !plan || nlat < 1 || nlat > kMaxLat) return DIRAC_ERR_ARG;
  *plan = nullptr;
  int recon = -1;
  for (int l = 0; l < nlat; ++l) {
    dirac_ctx* c = ctxs[l];
    if (!c || !out[l] || !in[l] || nrhs[l] < 1) return DIRAC_ERR_ARG;
    int rc = check_op(c, prec, false);
    if (rc) return rc;
    if (c->p.kind != DIRAC_WILSON_CLOVER) return set_err(c, DIRAC_ERR_UNSUPPORTED, "batch: Wilson-clover only");
    if (recon >= 0 && c->p.recon[prec] != recon)
      return set_err(c, DIRAC_ERR_ARG, "batch: every lattice needs the same link compression");
    recon = c->p.recon[prec];
  }
  if (ds && (prec != P64 || recon != 18 || tune != 0))
    return set_err(ctxs[0], DIRAC_ERR_UNSUPPORTED, "batch: double-single needs FP64 18-real links, untimed");
  dirac_batch* b = new dirac_batch();
  b->prec = prec;
  b->recon = recon;
  b->ds = ds;
  for (int l = 0, r0 = 0; l < nlat; ++l) {
    b->ctxs.push_back(ctxs[l]);
    b->lats.push_back(describe(ctxs[l], prec, in[l], out[l], nrhs[l], 1));
    b->lats.back().rhs0 = r0;
    r0 += nrhs[l];
  }
  if (cudaMalloc(&b->d_lats, sizeof(BatchLat) * nlat) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return DIRAC_ERR_OOM;
  }
  // autotune: time every candidate shape once (after one warm-up launch) and keep the
  // fastest; the launches write the plan's outputs, which the caller owns anyway
  cudaStream_t st = stream;
  int max_rhs = 1;
  for (int l = 0; l < nlat; ++l) max_rhs = nrhs[l] > max_rhs ? nrhs[l] : max_rhs;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = INFINITY;
  int bi = 0;
  const int ncand = (int)(sizeof(kCand) / sizeof(kCand[0]));
  for (int k = 0; k < ncand; ++k) {
    const int RG = kCand[k][0], per_sm = kCand[k][1];
    // tune < 2: only the shape (4 right-hand sides per CTA, 4 CTAs per SM)
    // (the default shape also serves plans with fewer right-hand sides: idle warps exit)
    if ((tune == 2 && RG > max_rhs && RG > 1) || (tune < 2 && k != kDefaultCand)) {
      b->cand_ms.push_back(-1);
      continue;
    }
    if (tune <= 0) {  // no timing at all
      best = 0;
      bi = k;
      b->cand_ms.push_back(-1);
      continue;
    }
    b->RG = RG;
    if (batch_layout(b, RG, st)) break;
    b->grid = grid_for(per_sm, b->ntiles);
    batch_launch_direct(b, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) batch_launch_direct(b, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      b->err = "autotune launch failed";
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    b->cand_ms.push_back(ms / 3);
    if (ms / 3 < best) { best = ms / 3; bi = k; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!b->err.empty() || best == INFINITY) {
    cudaGetLastError();
    cudaFree(b->d_lats);
    delete b;
    return DIRAC_ERR_CUDA;
  }
  b->RG = kCand[bi][0];
  b->per_sm = kCand[bi][1];
  if (batch_layout(b, b->RG, st)) {
    cudaFree(b->d_lats);
    delete b;
    return DIRAC_ERR_CUDA;
  }
  b->grid = grid_for(b->per_sm, b->ntiles);
  b->tuned_ms = best;
  b->cc_ms = best;
  // the tensor-core kernel (FP16 storage, 12- or 18-real links): timed the same way; the
  // plan keeps whichever kernel is faster
  if (prec == DIRAC_PREC_F16 && (recon == 12 || recon == 18) && tune >= 0) {
    std::vector<TcLat> tl(nlat);
    int begin = 0;
    for (int l = 0; l < nlat; ++l) {
      const BatchLat& L = b->lats[l];
      TcLat& T = tl[l];
      T.g = L.g;
      T.gauge = L.gauge;
      T.clover = L.clover;
      T.kappa = (float)L.kappa;
      T.in = L.in;
      T.out = L.out;
      T.field_bytes = L.field_bytes;
      T.nrhs = L.nrhs;
      T.ctiles = tc_ctiles(L.g.Vh);
      T.tiles = tc_tiles(T);
      T.tile_begin = begin;
      int* nb = nullptr;
      if (tc_build_nbr(L.g, &nb, st) == DIRAC_OK) b->tc_nbr.push_back(nb);
      T.nbr = nb;
      begin += T.tiles;
    }
    b->tc_ntiles = begin;
    const long g = (long)sm_count() * tc_ctas_per_sm(recon);
    b->tc_grid = (int)(g < begin ? g : begin);
    bool tables = true;
    for (int l = 0; l < nlat; ++l) tables = tables && tl[l].nbr != nullptr;
    if (!tables || cudaMalloc(&b->d_tc, sizeof(TcLat) * nlat) != cudaSuccess ||
        cudaMemcpyAsync(b->d_tc, tl.data(), sizeof(TcLat) * nlat, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      if (b->d_tc) cudaFree(b->d_tc);
      b->d_tc = nullptr;
    } else if (tune == 0) {
      b->use_tc = true;  // untimed plans take the tensor-core kernel where there is one
    } else {
      cudaEvent_t f0, f1;
      cudaEventCreate(&f0);
      cudaEventCreate(&f1);
      b->use_tc = true;
      batch_launch_direct(b, st);
      cudaEventRecord(f0, st);
      for (int r = 0; r < 3; ++r) batch_launch_direct(b, st);
      cudaEventRecord(f1, st);
      float ms = 0;
      if (cudaEventSynchronize(f1) == cudaSuccess && cudaGetLastError() == cudaSuccess &&
          cudaEventElapsedTime(&ms, f0, f1) == cudaSuccess) {
        b->tc_ms = ms / 3;
        b->use_tc = b->tc_ms < best;
        if (b->use_tc) b->tuned_ms = b->tc_ms;
      } else {
        cudaGetLastError();
        b->use_tc = false;
      }
      cudaEventDestroy(f0);
      cudaEventDestroy(f1);
      if (b->tc_ms < 0) {
        // the tensor-core launch failed: the plan keeps the CUDA-core kernel
        cudaStreamSynchronize(st);
        cudaGetLastError();
      }
    }
  }
  *plan = b;
  return cudaStreamSynchronize(st) == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}

// Right-hand sides whose mask entry is 0 are skipped by the CUDA-core kernels (their
// outputs are left as they are); a masked plan uses the CUDA-core kernel. The mask is
// read at every launch, so it may change between launches and inside captured graphs.
int batch_set_mask(dirac_batch* b, const double* mask, int stride, cudaStream_t st) {
  if (!b) return DIRAC_ERR_ARG;
  for (BatchLat& L : b->lats) {
    L.mask = mask;
    L.mstride = stride;
  }
  if (mask && b->use_tc) {
    b->use_tc = false;
    b->tuned_ms = b->cc_ms;
  }
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->graph_napply = 0;
  return batch_layout(b, b->RG, st);
}

}  // namespace dirac

extern "C" {

int dirac_batch_apply(dirac_batch* b, void* stream) {
  if (!b) return DIRAC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) {
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return DIRAC_ERR_CUDA;
    return DIRAC_OK;
  }
  batch_launch_direct(b, st);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}

int dirac_batch_capture(dirac_batch* b, int napply, void* stream) {
  if (!b || napply < 1) return DIRAC_ERR_ARG;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return DIRAC_ERR_CUDA;
  // the capture stream waits for the caller's stream so the descriptor table is in place
  cudaEvent_t ready;
  cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  cudaEventRecord(ready, (cudaStream_t)stream);
  cudaStreamWaitEvent(cap, ready, 0);
  cudaStreamSynchronize(cap);
  cudaEventDestroy(ready);
  int rc = DIRAC_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = DIRAC_ERR_CUDA;
  for (int k = 0; rc == DIRAC_OK && k < napply; ++k) batch_launch_direct(b, cap);
  if (rc == DIRAC_OK && cudaStreamEndCapture(cap, &b->graph) != cudaSuccess) rc = DIRAC_ERR_CUDA;
  if (rc == DIRAC_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = DIRAC_ERR_CUDA;
  cudaStreamDestroy(cap);
  if (rc) {
    cudaGetLastError();
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->exec = nullptr;
    return rc;
  }
  b->graph_napply = napply;
  return DIRAC_OK;
}

int dirac_batch_info(const dirac_batch* b, int* rhs_per_cta, int* ctas_per_sm, int* grid, double* tuned_ms) {
  if (!b) return DIRAC_ERR_ARG;
  if (rhs_per_cta) *rhs_per_cta = b->RG;
  if (ctas_per_sm) *ctas_per_sm = b->per_sm;
  if (grid) *grid = b->grid;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return DIRAC_OK;
}

int dirac_batch_set_tensor_cores(dirac_batch* b, int on) {
  if (!b) return DIRAC_ERR_ARG;
  if (on && !b->d_tc) return DIRAC_ERR_UNSUPPORTED;
  if (b->use_tc != (on != 0)) {
    // a captured graph holds the other kernel: drop it (capture again)
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_napply = 0;
  }
  b->use_tc = on != 0;
  b->tuned_ms = b->use_tc ? b->tc_ms : b->cc_ms;
  return DIRAC_OK;
}

int dirac_batch_kernel_info(const dirac_batch* b, int* tensor_cores, double* cuda_core_ms, double* tensor_core_ms) {
  if (!b) return DIRAC_ERR_ARG;
  if (tensor_cores) *tensor_cores = b->use_tc ? 1 : 0;
  if (cuda_core_ms) *cuda_core_ms = b->cc_ms;
  if (tensor_core_ms) *tensor_core_ms = b->tc_ms;
  return DIRAC_OK;
}

int dirac_batch_destroy(dirac_batch* b) {
  if (!b) return DIRAC_ERR_ARG;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_tc) cudaFree(b->d_tc);
  for (int* t : b->tc_nbr) cudaFree(t);
  if (b->d_lats) cudaFree(b->d_lats);
  delete b;
  cudaGetLastError();
  return DIRAC_OK;
}

}  // extern "C"
