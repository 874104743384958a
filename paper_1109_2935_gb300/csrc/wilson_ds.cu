// The Wilson-clover operator M (Eq. 2, kappa form) on FP64 fields evaluated in
// double-single arithmetic: the stencil of wilson.cuh instantiated with a float-float
// value type. The solvers can use it for the FP64 true residual r = b - M x of their
// restarts and reliable updates (Sec. 8.2: only that residual, the solution and the
// global sums need more than the sloppy precision): the binary32 pipes run about 60x the
// FP64 rate, and the ~48-bit products keep the residual accurate to ~1e-14 of |M x|. The
// float-float value doubles the register footprint and its add is a chain of ~10
// dependent operations, so at 8 resident warps per SM the kernel measured slower than the
// FP64 one; it is therefore off by default (dirac_set_ds_residual).
// Storage (spinors, 18-real links, clover) is the FP64 storage of the context.
#include "wilson_ds.cuh"

#include "internal.h"
#include "wilson.cuh"

namespace dirac {

void launch_wilson_ds(const WilsonArg& a, cudaStream_t st) {
  constexpr int T = WilsonShape<P64DS>::threads;
  const int n = 2 * a.g.Vh;
  wilson_kernel<P64DS, 18, true><<<(n + T - 1) / T, T, 0, st>>>(a);
}

}  // namespace dirac
