// Wilson-clover stencil instantiations for P32 storage (kernel template in wilson.cuh).
#include "wilson.cuh"
#include "internal.h"

namespace dirac {
void launch_wilson_p32(int recon, bool fullm, const WilsonArg& a, cudaStream_t st) {
  launch_wilson_prec<P32>(recon, fullm, a, st);
}
}  // namespace dirac
