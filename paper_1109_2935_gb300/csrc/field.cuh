// Device-side field access: precision traits, chunked spinor/link/clover loads and
// stores, and the SU(3) arithmetic used by the stencils.
//
// Storage follows the paper's memory-traffic reductions (Sec. 5): fields are
// reordered into chunk-major arrays so that a warp's loads of one chunk are
// contiguous, SU(3) links are stored with 18, 12 or 8 reals and rebuilt in
// registers, and 16-bit storage keeps a per-site FP32 norm.
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

namespace dirac {

enum { P64 = 0, P32 = 1, P16 = 2 };
// a fourth arithmetic for stencils only: FP64 storage read into double-single (float-float)
// arithmetic (dsfloat.cuh, wilson_ds.cu); fields and storage are those of P64
enum { P64DS = 3 };

template <int PREC> struct Real { using T = float; };
template <> struct Real<P64> { using T = double; };

// ---------------------------------------------------------------- lattice geometry
struct Geom {
  int L[4];      // LX, LY, LZ, LT
  int Lxh;       // LX / 2
  int Vh;        // sites per parity
  int apbc;      // antiperiodic t for fermion hops
};

// Coordinates of checkerboard site cb of parity par.
__device__ __forceinline__ void cb_coords(const Geom& g, int cb, int par, int x[4]) {
  int xh = cb % g.Lxh;
  int r = cb / g.Lxh;
  x[1] = r % g.L[1]; r /= g.L[1];
  x[2] = r % g.L[2];
  x[3] = r / g.L[2];
  x[0] = 2 * xh + ((par + x[1] + x[2] + x[3]) & 1);
}

__device__ __forceinline__ int cb_index(const Geom& g, const int x[4]) {
  return ((x[3] * g.L[2] + x[2]) * g.L[1] + x[1]) * g.Lxh + (x[0] >> 1);
}

// ---------------------------------------------------------------- complex helpers
template <typename T> struct C { T r, i; };
template <typename T> __device__ __forceinline__ C<T> cmk(T r, T i) { return C<T>{r, i}; }
template <typename T> __device__ __forceinline__ C<T> operator+(C<T> a, C<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ C<T> operator-(C<T> a, C<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ C<T> operator*(C<T> a, C<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T> __device__ __forceinline__ C<T> operator*(T s, C<T> a) { return {s * a.r, s * a.i}; }
template <typename T> __device__ __forceinline__ C<T> conj(C<T> a) { return {a.r, -a.i}; }
template <typename T> __device__ __forceinline__ C<T> times_i(C<T> a) { return {-a.i, a.r}; }
// a += b * c
template <typename T> __device__ __forceinline__ void cmac(C<T>& a, C<T> b, C<T> c) {
  a.r = fma(b.r, c.r, a.r); a.r = fma(-b.i, c.i, a.r);
  a.i = fma(b.r, c.i, a.i); a.i = fma(b.i, c.r, a.i);
}
// a += conj(b) * c
template <typename T> __device__ __forceinline__ void cmacc(C<T>& a, C<T> b, C<T> c) {
  a.r = fma(b.r, c.r, a.r); a.r = fma(b.i, c.i, a.r);
  a.i = fma(b.r, c.i, a.i); a.i = fma(-b.i, c.r, a.i);
}

template <typename T> struct Link { C<T> m[3][3]; };

// v = U h (3-vector)
template <typename T>
__device__ __forceinline__ void su3_mv(const Link<T>& U, const C<T> h[3], C<T> v[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v[a] = U.m[a][0] * h[0];
    cmac(v[a], U.m[a][1], h[1]);
    cmac(v[a], U.m[a][2], h[2]);
  }
}
// v = U^dagger h
template <typename T>
__device__ __forceinline__ void su3_mv_dag(const Link<T>& U, const C<T> h[3], C<T> v[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v[a] = conj(U.m[0][a]) * h[0];
    cmacc(v[a], U.m[1][a], h[1]);
    cmacc(v[a], U.m[2][a], h[2]);
  }
}

// fma of one binary16 half of word a and one of word b into an FP32 accumulator: the two
// binary16 factors enter the fused multiply-add exactly (their product is exact in FP32),
// so this equals converting both and one FP32 fma, without the conversions.
template <int HA, int HB>
__device__ __forceinline__ float fma_hh(uint32_t a, uint32_t b, float c) {
  float d;
  asm("{\n\t.reg .b16 a0, a1, b0, b1;\n\t"
      "mov.b32 {a0, a1}, %1;\n\t"
      "mov.b32 {b0, b1}, %2;\n\t"
      "fma.rn.f32.f16 %0, a%4, b%5, %3;\n\t}"
      : "=f"(d) : "r"(a), "r"(b), "f"(c), "n"(HA), "n"(HB));
  return d;
}

// ---------------------------------------------------------------- raw chunk I/O
template <typename V> __device__ __forceinline__ V ldg_chunk(const char* p) {
  return __ldg(reinterpret_cast<const V*>(p));
}
// Read-only-cache load (NC) for fields no thread writes during the kernel, plain
// coherent load otherwise (BLAS kernels update fields in place).
template <typename V, bool NC> __device__ __forceinline__ V ld_chunk(const char* p) {
  if constexpr (NC) return __ldg(reinterpret_cast<const V*>(p));
  else return *reinterpret_cast<const V*>(p);
}

__device__ __forceinline__ void unpack_half8(int4 q, float v[8]) {
  const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 f = __half22float2(h[k]);
    v[2 * k] = f.x; v[2 * k + 1] = f.y;
  }
}
__device__ __forceinline__ int4 pack_half8(const float v[8]) {
  int4 q;
  __half2* h = reinterpret_cast<__half2*>(&q);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
  return q;
}

// ---------------------------------------------------------------- spinor I/O
// NR = reals per site: 24 (Wilson) or 6 (staggered).
template <int PREC, int NR> struct SpinorIO;

template <int NR> struct SpinorIO<P64, NR> {
  __host__ __device__ static constexpr size_t half_bytes(int64_t Vh) { return (size_t)NR * 8 * Vh; }
  template <bool NC = true>
  __device__ static void load(const char* b, int Vh, int cb, double v[NR]) {
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      double2 q = ld_chunk<double2, NC>(b + ((size_t)k * Vh + cb) * 16);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const double v[NR]) {
#pragma unroll
    for (int k = 0; k < NR / 2; ++k)
      *reinterpret_cast<double2*>(b + ((size_t)k * Vh + cb) * 16) = make_double2(v[2 * k], v[2 * k + 1]);
  }
};

template <> struct SpinorIO<P32, 24> {
  __host__ __device__ static constexpr size_t half_bytes(int64_t Vh) { return (size_t)96 * Vh; }
  template <bool NC = true>
  __device__ static void load(const char* b, int Vh, int cb, float v[24]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 q = ld_chunk<float4, NC>(b + ((size_t)k * Vh + cb) * 16);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const float v[24]) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
      *reinterpret_cast<float4*>(b + ((size_t)k * Vh + cb) * 16) =
          make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  }
};

template <> struct SpinorIO<P32, 6> {
  __host__ __device__ static constexpr size_t half_bytes(int64_t Vh) { return (size_t)24 * Vh; }
  template <bool NC = true>
  __device__ static void load(const char* b, int Vh, int cb, float v[6]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 q = ld_chunk<float2, NC>(b + ((size_t)k * Vh + cb) * 8);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const float v[6]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      *reinterpret_cast<float2*>(b + ((size_t)k * Vh + cb) * 8) = make_float2(v[2 * k], v[2 * k + 1]);
  }
};

__device__ __forceinline__ float site_norm_scale(const float* v, int n, float& inv) {
  float m = 0.f;
  for (int k = 0; k < n; ++k) m = fmaxf(m, fabsf(v[k]));
  inv = m > 0.f ? 1.0f / m : 0.f;
  return m;
}

template <> struct SpinorIO<P16, 24> {
  __host__ __device__ static constexpr size_t half_bytes(int64_t Vh) { return (size_t)52 * Vh; }
  // the 24 stored values without the per-site norm, which is returned
  template <bool NC = true>
  __device__ static float load_raw(const char* b, int Vh, int cb, float v[24]) {
    const float n = ld_chunk<float, NC>(b + (size_t)48 * Vh + (size_t)cb * 4);
#pragma unroll
    for (int k = 0; k < 3; ++k) unpack_half8(ld_chunk<int4, NC>(b + ((size_t)k * Vh + cb) * 16), v + 8 * k);
    return n;
  }
  template <bool NC = true>
  __device__ static void load(const char* b, int Vh, int cb, float v[24]) {
    float n = ld_chunk<float, NC>(b + (size_t)48 * Vh + (size_t)cb * 4);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int4 q = ld_chunk<int4, NC>(b + ((size_t)k * Vh + cb) * 16);
      unpack_half8(q, v + 8 * k);
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] *= n;
  }
  __device__ static void store(char* b, int Vh, int cb, const float v[24]) {
    float inv, w[24];
    float n = site_norm_scale(v, 24, inv);
#pragma unroll
    for (int k = 0; k < 24; ++k) w[k] = v[k] * inv;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      *reinterpret_cast<int4*>(b + ((size_t)k * Vh + cb) * 16) = pack_half8(w + 8 * k);
    reinterpret_cast<float*>(b + (size_t)48 * Vh)[cb] = n;
  }
};

template <> struct SpinorIO<P16, 6> {
  __host__ __device__ static constexpr size_t half_bytes(int64_t Vh) { return (size_t)16 * Vh; }
  // the 6 stored values without the per-site norm, which is returned
  template <bool NC = true>
  __device__ static float load_raw(const char* b, int Vh, int cb, float v[6]) {
    const float n = ld_chunk<float, NC>(b + (size_t)12 * Vh + (size_t)cb * 4);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 q = __half22float2(ld_chunk<__half2, NC>(b + ((size_t)k * Vh + cb) * 4));
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
    return n;
  }
  template <bool NC = true>
  __device__ static void load(const char* b, int Vh, int cb, float v[6]) {
    float n = ld_chunk<float, NC>(b + (size_t)12 * Vh + (size_t)cb * 4);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      __half2 q = ld_chunk<__half2, NC>(b + ((size_t)k * Vh + cb) * 4);
      float2 f = __half22float2(q);
      v[2 * k] = f.x * n; v[2 * k + 1] = f.y * n;
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const float v[6]) {
    float inv;
    float n = site_norm_scale(v, 6, inv);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      *reinterpret_cast<__half2*>(b + ((size_t)k * Vh + cb) * 4) =
          __floats2half2_rn(v[2 * k] * inv, v[2 * k + 1] * inv);
    reinterpret_cast<float*>(b + (size_t)12 * Vh)[cb] = n;
  }
};

// ---------------------------------------------------------------- gauge links
// Layout per precision: [mu][parity][chunk][Vh]; R stored reals per link.
//   R = 18: all entries, row-major (re, im)
//   R = 12: rows 0 and 1; row 2 = conj(row0 x row1)
//   R = 8 : Re/Im a2, a3, b1, arg(a1)/pi, arg(c1)/pi  (a, b, c = rows)
template <int PREC, int R> struct LinkIO;

__device__ __forceinline__ size_t link_plane_bytes(int R, int w, int Vh) { return (size_t)R * w * Vh; }

// row 2 = conj(row 0 x row 1): c = a_p b_q - a_q b_p as two chains of three fused
// multiply-adds after one product per real part
template <typename T>
__device__ __forceinline__ void reconstruct12(Link<T>& U) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int p = (j + 1) % 3, q = (j + 2) % 3;
    const C<T> ap = U.m[0][p], aq = U.m[0][q], bp = U.m[1][p], bq = U.m[1][q];
    T cr = ap.r * bq.r;
    cr = fma(-ap.i, bq.i, cr);
    cr = fma(-aq.r, bp.r, cr);
    cr = fma(aq.i, bp.i, cr);
    T ci = ap.r * bq.i;
    ci = fma(ap.i, bq.r, ci);
    ci = fma(-aq.r, bp.i, ci);
    ci = fma(-aq.i, bp.r, ci);
    U.m[2][j] = C<T>{cr, -ci};
  }
}

__device__ __forceinline__ void sincos_pi(double a, double* s, double* c) { sincospi(a, s, c); }
__device__ __forceinline__ void sincos_pi(float a, float* s, float* c) { sincospif(a, s, c); }

template <typename T>
__device__ __forceinline__ void reconstruct8(const T p[8], Link<T>& U) {
  C<T> a2 = {p[0], p[1]}, a3 = {p[2], p[3]}, b1 = {p[4], p[5]};
  T N = a2.r * a2.r + a2.i * a2.i + a3.r * a3.r + a3.i * a3.i;
  T sa, ca, sc, cc;
  sincos_pi(p[6], &sa, &ca);
  sincos_pi(p[7], &sc, &cc);
  T ma1 = sqrt(fmax((T)1 - N, (T)0));
  C<T> a1 = {ma1 * ca, ma1 * sa};
  T mc1 = sqrt(fmax((T)1 - ma1 * ma1 - (b1.r * b1.r + b1.i * b1.i), (T)0));
  C<T> c1 = {mc1 * cc, mc1 * sc};
  T invN = (T)1 / N;
  C<T> ca1 = conj(a1), ca2 = conj(a2), ca3 = conj(a3), cb1 = conj(b1), cc1 = conj(c1);
  C<T> a1b1 = ca1 * b1, a1c1 = ca1 * c1;
  U.m[0][0] = a1; U.m[0][1] = a2; U.m[0][2] = a3;
  U.m[1][0] = b1;
  U.m[1][1] = (-invN) * (ca3 * cc1 + a2 * a1b1);
  U.m[1][2] = invN * (ca2 * cc1 - a3 * a1b1);
  U.m[2][0] = c1;
  U.m[2][1] = invN * (ca3 * cb1 - a2 * a1c1);
  U.m[2][2] = (-invN) * (ca2 * cb1 + a3 * a1c1);
}

template <int PREC, int R>
struct LinkIO {
  using T = typename Real<PREC>::T;
  static constexpr int W = PREC == P64 ? 8 : (PREC == P32 ? 4 : 2);
  // storage chunks per link: bytes per chunk and chunk count
  static constexpr int kChunkBytes = PREC == P64 ? 16
                                   : PREC == P32 ? (R == 18 ? 8 : 16)
                                   : (R == 18 ? 4 : (R == 12 ? 8 : 16));
  static constexpr int kChunks = R * W / kChunkBytes;

  // load the link at index i of a plane whose chunk arrays have `stride` entries
  // (NC: read-only-cache loads from global memory; otherwise plain loads, e.g. smem)
  template <bool NC = true>
  __device__ static void load_plane(const char* plane, int stride, int i, Link<T>& U) {
    T v[R];
    if constexpr (PREC == P64) {
#pragma unroll
      for (int k = 0; k < R / 2; ++k) {
        double2 q = ld_chunk<double2, NC>(plane + ((size_t)k * stride + i) * 16);
        v[2 * k] = (T)q.x; v[2 * k + 1] = (T)q.y;
      }
    } else if constexpr (PREC == P32) {
      if constexpr (R == 18) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          float2 q = ld_chunk<float2, NC>(plane + ((size_t)k * stride + i) * 8);
          v[2 * k] = q.x; v[2 * k + 1] = q.y;
        }
      } else {
#pragma unroll
        for (int k = 0; k < R / 4; ++k) {
          float4 q = ld_chunk<float4, NC>(plane + ((size_t)k * stride + i) * 16);
          v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
        }
      }
    } else {
      if constexpr (R == 18) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          float2 f = __half22float2(ld_chunk<__half2, NC>(plane + ((size_t)k * stride + i) * 4));
          v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
      } else if constexpr (R == 12) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          uint2 q = ld_chunk<uint2, NC>(plane + ((size_t)k * stride + i) * 8);
          const __half2* h = reinterpret_cast<const __half2*>(&q);
          float2 f0 = __half22float2(h[0]), f1 = __half22float2(h[1]);
          v[4 * k] = f0.x; v[4 * k + 1] = f0.y; v[4 * k + 2] = f1.x; v[4 * k + 3] = f1.y;
        }
      } else {
        int4 q = ld_chunk<int4, NC>(plane + (size_t)i * 16);
        float f[8];
        unpack_half8(q, f);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = f[k];
      }
    }
    if constexpr (R == 8) {
      reconstruct8(v, U);
    } else {
#pragma unroll
      for (int a = 0; a < R / 6; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) U.m[a][b] = C<T>{v[6 * a + 2 * b], v[6 * a + 2 * b + 1]};
      if constexpr (R == 12) reconstruct12(U);
    }
  }
  // load link (mu, par, cb) from the gauge base pointer
  __device__ static void load(const char* base, int Vh, int mu, int par, int cb, Link<T>& U) {
    load_plane<true>(base + (size_t)(mu * 2 + par) * link_plane_bytes(R, W, Vh), Vh, cb, U);
  }
  // store the compressed form of a full FP64 link
  __device__ static void store(char* base, int Vh, int mu, int par, int cb, const double u[18]) {
    char* plane = base + (size_t)(mu * 2 + par) * link_plane_bytes(R, W, Vh);
    double v[18];
    if constexpr (R == 8) {
      v[0] = u[2]; v[1] = u[3]; v[2] = u[4]; v[3] = u[5]; v[4] = u[6]; v[5] = u[7];
      v[6] = atan2(u[1], u[0]) / 3.14159265358979323846;
      v[7] = atan2(u[13], u[12]) / 3.14159265358979323846;
    } else {
      for (int k = 0; k < R; ++k) v[k] = u[k];
    }
    if constexpr (PREC == P64) {
      for (int k = 0; k < R / 2; ++k)
        *reinterpret_cast<double2*>(plane + ((size_t)k * Vh + cb) * 16) = make_double2(v[2 * k], v[2 * k + 1]);
    } else if constexpr (PREC == P32) {
      if constexpr (R == 18) {
        for (int k = 0; k < 9; ++k)
          *reinterpret_cast<float2*>(plane + ((size_t)k * Vh + cb) * 8) = make_float2((float)v[2 * k], (float)v[2 * k + 1]);
      } else {
        for (int k = 0; k < R / 4; ++k)
          *reinterpret_cast<float4*>(plane + ((size_t)k * Vh + cb) * 16) =
              make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
      }
    } else {
      if constexpr (R == 18) {
        for (int k = 0; k < 9; ++k)
          *reinterpret_cast<__half2*>(plane + ((size_t)k * Vh + cb) * 4) =
              __floats2half2_rn((float)v[2 * k], (float)v[2 * k + 1]);
      } else if constexpr (R == 12) {
        for (int k = 0; k < 3; ++k) {
          uint2 q;
          __half2* h = reinterpret_cast<__half2*>(&q);
          h[0] = __floats2half2_rn((float)v[4 * k], (float)v[4 * k + 1]);
          h[1] = __floats2half2_rn((float)v[4 * k + 2], (float)v[4 * k + 3]);
          *reinterpret_cast<uint2*>(plane + ((size_t)k * Vh + cb) * 8) = q;
        }
      } else {
        float f[8];
        for (int k = 0; k < 8; ++k) f[k] = (float)v[k];
        *reinterpret_cast<int4*>(plane + (size_t)cb * 16) = pack_half8(f);
      }
    }
  }
};

// ---------------------------------------------------------------- clover I/O
// Per site: two Hermitian 6x6 blocks (chirality +: spins 0,1; chirality -: spins
// 2,3), each stored as 6 real diagonal entries followed by the 15 complex entries
// below the diagonal in row-major order (i > j): 36 reals per block, 72 per site.
// Layout [parity][chunk][Vh]; F16 adds Vh FP32 per-site scales after the chunks.
template <int PREC> struct CloverIO;

template <> struct CloverIO<P64> {
  __host__ __device__ static constexpr size_t parity_bytes(int64_t Vh) { return (size_t)576 * Vh; }
  __device__ static void load(const char* b, int Vh, int cb, double v[72]) {
#pragma unroll
    for (int k = 0; k < 36; ++k) {
      double2 q = ldg_chunk<double2>(b + ((size_t)k * Vh + cb) * 16);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const double v[72]) {
    for (int k = 0; k < 36; ++k)
      *reinterpret_cast<double2*>(b + ((size_t)k * Vh + cb) * 16) = make_double2(v[2 * k], v[2 * k + 1]);
  }
};
template <> struct CloverIO<P32> {
  __host__ __device__ static constexpr size_t parity_bytes(int64_t Vh) { return (size_t)288 * Vh; }
  __device__ static void load(const char* b, int Vh, int cb, float v[72]) {
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      float4 q = ldg_chunk<float4>(b + ((size_t)k * Vh + cb) * 16);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  }
  __device__ static void store(char* b, int Vh, int cb, const double v[72]) {
    for (int k = 0; k < 18; ++k)
      *reinterpret_cast<float4*>(b + ((size_t)k * Vh + cb) * 16) =
          make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
  }
};
template <> struct CloverIO<P16> {
  __host__ __device__ static constexpr size_t parity_bytes(int64_t Vh) { return (size_t)148 * Vh; }
  // the 72 stored values without the per-site norm, which is returned
  __device__ static float load_raw(const char* b, int Vh, int cb, float v[72]) {
    const float n = __ldg(reinterpret_cast<const float*>(b + (size_t)144 * Vh) + cb);
#pragma unroll
    for (int k = 0; k < 9; ++k) unpack_half8(ldg_chunk<int4>(b + ((size_t)k * Vh + cb) * 16), v + 8 * k);
    return n;
  }
  __device__ static void load(const char* b, int Vh, int cb, float v[72]) {
    float n = __ldg(reinterpret_cast<const float*>(b + (size_t)144 * Vh) + cb);
#pragma unroll
    for (int k = 0; k < 9; ++k) unpack_half8(ldg_chunk<int4>(b + ((size_t)k * Vh + cb) * 16), v + 8 * k);
#pragma unroll
    for (int k = 0; k < 72; ++k) v[k] *= n;
  }
  __device__ static void store(char* b, int Vh, int cb, const double v[72]) {
    float m = 0.f;
    for (int k = 0; k < 72; ++k) m = fmaxf(m, fabsf((float)v[k]));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    for (int k = 0; k < 9; ++k) {
      float f[8];
      for (int j = 0; j < 8; ++j) f[j] = (float)v[8 * k + j] * inv;
      *reinterpret_cast<int4*>(b + ((size_t)k * Vh + cb) * 16) = pack_half8(f);
    }
    reinterpret_cast<float*>(b + (size_t)144 * Vh)[cb] = m;
  }
};

// The 36 reals of chirality block `blk` (0 or 1) of site i, from a clover array with
// chunk stride `stride` (global memory with NC, shared memory without).
template <int PREC, bool NC, typename T>
__device__ __forceinline__ void clover_block(const char* b, int stride, int i, int blk, T v[36]) {
  if constexpr (PREC == P64) {
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      double2 q = ld_chunk<double2, NC>(b + ((size_t)(18 * blk + k) * stride + i) * 16);
      v[2 * k] = (T)q.x; v[2 * k + 1] = (T)q.y;
    }
  } else if constexpr (PREC == P32) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float4 q = ld_chunk<float4, NC>(b + ((size_t)(9 * blk + k) * stride + i) * 16);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else {
    // reals 36*blk .. 36*blk+35 live in 8-half chunks 4*blk .. 4*blk+4
    const float n = ld_chunk<float, NC>(b + (size_t)144 * stride + (size_t)i * 4);
    float f[40];
#pragma unroll
    for (int k = 0; k < 5; ++k) unpack_half8(ld_chunk<int4, NC>(b + ((size_t)(4 * blk + k) * stride + i) * 16), f + 8 * k);
    const int off = 4 * blk;  // block 1 starts 4 halves into chunk 4
#pragma unroll
    for (int k = 0; k < 36; ++k) v[k] = f[k + off] * n;
  }
}

// y = A x for one Hermitian 6x6 block stored as above (d[6], then 15 complex L_ij, i>j)
template <typename T>
__device__ __forceinline__ void herm6_mv(const T* blk, const C<T> x[6], C<T> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = blk[i] * x[i];
  int o = 6;
#pragma unroll
  for (int i = 1; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) {
      C<T> l = {blk[o], blk[o + 1]};
      o += 2;
      cmac(y[i], l, x[j]);   // y_i += L_ij x_j
      cmacc(y[j], l, x[i]);  // y_j += conj(L_ij) x_i
    }
  }
}

}  // namespace dirac
