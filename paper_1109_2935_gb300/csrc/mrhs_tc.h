// Tensor-core multi-right-hand-side Wilson-clover operator (mrhs_tc.cu): the lattice
// descriptor its persistent kernel walks and the host-side launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "field.cuh"

namespace dirac {

// One lattice of a tensor-core batch: nrhs consecutive FP16 full fields in `in` / `out`
// (field_bytes apart), links in FP16 with 12 or 18 reals, Ahat in FP16 (null: Ahat = 1).
struct TcLat {
  Geom g;
  const char* gauge;
  const char* clover;
  float kappa;
  const char* in;
  char* out;
  size_t field_bytes;
  int nrhs;
  int ctiles;      // tiles of sites per parity
  int tiles;       // ctiles * 2 parities * right-hand-side groups of 16
  int tile_begin;  // first tile of this lattice in the batch
  const int* nbr;  // [parity][Vh][hop]: neighbour cb of each hop (hop = 2 mu + dir, dir 0
                   // forward), bit 31 set when the hop crosses the antiperiodic t edge
};

// the neighbour table of a lattice for TcLat::nbr (device memory the caller frees)
int tc_build_nbr(const Geom& g, int** table, cudaStream_t st);

int tc_ctiles(int Vh);
int tc_tiles(const TcLat& L);
// resident CTAs per SM of the kernel (occupancy calculator)
int tc_ctas_per_sm(int recon);
void launch_mrhs_tc(int recon, const TcLat* d_lats, int nlat, int ntiles, int grid, cudaStream_t st);

}  // namespace dirac
