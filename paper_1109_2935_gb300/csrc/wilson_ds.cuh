// Double-single instantiation of the FP64-storage field access (P64DS): FP64 spinors,
// 18-real FP64 links and FP64 clover read into float-float values (dsfloat.cuh), results
// written back as FP64. Included by the translation units that instantiate the stencil
// with P64DS (the single-field operator and the batched kernel).
#pragma once
#include "dsfloat.cuh"
#include "field.cuh"

namespace dirac {

template <> struct Real<P64DS> { using T = dsf; };

template <> struct SpinorIO<P64DS, 24> {
  template <bool NC = true>
  __device__ static void load(const char* b, int Vh, int cb, dsf v[24]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double2 q = ld_chunk<double2, NC>(b + ((size_t)k * Vh + cb) * 16);
      v[2 * k] = dsf(q.x);
      v[2 * k + 1] = dsf(q.y);
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const dsf v[24]) {
#pragma unroll
    for (int k = 0; k < 12; ++k)
      *reinterpret_cast<double2*>(b + ((size_t)k * Vh + cb) * 16) =
          make_double2(v[2 * k].to_double(), v[2 * k + 1].to_double());
  }
};

template <> struct LinkIO<P64DS, 18> {
  __device__ static void load(const char* base, int Vh, int mu, int par, int cb, Link<dsf>& U) {
    const char* plane = base + (size_t)(mu * 2 + par) * (size_t)18 * 8 * Vh;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 q = __ldg(reinterpret_cast<const double2*>(plane + ((size_t)k * Vh + cb) * 16));
      U.m[k / 3][k % 3] = C<dsf>{dsf(q.x), dsf(q.y)};
    }
  }
};

template <> struct CloverIO<P64DS> {
  __host__ __device__ static constexpr size_t parity_bytes(int64_t Vh) { return (size_t)576 * Vh; }
};

}  // namespace dirac
