// BLAS-1 and global reductions on spinor fields (Sec. 6.1: fields stored
// contiguously so that BLAS-like routines and global reductions run efficiently;
// Sec. 8.2: this linear algebra is bandwidth-bound).
//
// Every kernel works site by site on fields of any storage precision (FP64, FP32,
// FP16 + per-site norm). Arithmetic is FP32 when no FP64 field takes part and FP64
// otherwise; every reduction accumulates in FP64. Reductions are deterministic:
// each block writes a partial sum, the last block to finish adds the partials in a
// fixed order and writes the result into mapped pinned host memory.
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "internal.h"

namespace dirac {

static constexpr int kRedBlocks = 152 * 4;
static constexpr int kThreads = 256;
static constexpr int kMaxMulti = 16;

struct Blas {
  double* partials = nullptr;  // device [kRedBlocks][3]
  unsigned* ticket = nullptr;  // device counter, returns to 0 after each reduction
  double* host_res = nullptr;  // pinned, mapped
  double* dev_res = nullptr;   // device alias of host_res
  std::string err;
};

Blas* blas_create() {
  Blas* b = new Blas();
  if (cudaMalloc(&b->partials, sizeof(double) * 3 * kRedBlocks) != cudaSuccess ||
      cudaMalloc(&b->ticket, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(b->ticket, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaHostAlloc(&b->host_res, sizeof(double) * 4, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&b->dev_res, b->host_res, 0) != cudaSuccess) {
    blas_destroy(b);
    return nullptr;
  }
  return b;
}

void blas_destroy(Blas* b) {
  if (!b) return;
  if (b->partials) cudaFree(b->partials);
  if (b->ticket) cudaFree(b->ticket);
  if (b->host_res) cudaFreeHost(b->host_res);
  delete b;
}

const char* blas_error(Blas* b) { return b ? b->err.c_str() : "no blas context"; }

// ---------------------------------------------------------------- site access
template <int NR, typename T>
__device__ __forceinline__ void site_load(const FieldRef& f, int s, T v[NR]) {
  int q = s >= f.Vh ? 1 : 0;
  int cb = s - q * f.Vh;
  const char* b = f.p + q * f.hb;
  if (f.prec == P64) {
    double t[NR];
    SpinorIO<P64, NR>::template load<false>(b, f.Vh, cb, t);
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = (T)t[k];
  } else if (f.prec == P32) {
    float t[NR];
    SpinorIO<P32, NR>::template load<false>(b, f.Vh, cb, t);
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = (T)t[k];
  } else {
    float t[NR];
    SpinorIO<P16, NR>::template load<false>(b, f.Vh, cb, t);
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = (T)t[k];
  }
}

template <int NR, typename T>
__device__ __forceinline__ void site_store(const FieldRef& f, int s, const T v[NR]) {
  int q = s >= f.Vh ? 1 : 0;
  int cb = s - q * f.Vh;
  char* b = f.p + q * f.hb;
  if (f.prec == P64) {
    double t[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) t[k] = (double)v[k];
    SpinorIO<P64, NR>::store(b, f.Vh, cb, t);
  } else {
    float t[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) t[k] = (float)v[k];
    if (f.prec == P32) SpinorIO<P32, NR>::store(b, f.Vh, cb, t);
    else SpinorIO<P16, NR>::store(b, f.Vh, cb, t);
  }
}

// Stores v like site_store and leaves in v the values as stored, so that a reduction
// over the result needs no reload: for FP16 the binary16 values times the per-site
// norm, computed exactly as a load decodes them; FP32 / FP64 storage leaves v as it is.
template <int NR, typename T>
__device__ __forceinline__ void site_store_q(const FieldRef& f, int s, T v[NR]) {
  if (f.prec != P16) {
    site_store<NR>(f, s, v);
    return;
  }
  int q = s >= f.Vh ? 1 : 0;
  int cb = s - q * f.Vh;
  char* b = f.p + q * f.hb;
  float t[NR], inv;
#pragma unroll
  for (int k = 0; k < NR; ++k) t[k] = (float)v[k];
  const float n = site_norm_scale(t, NR, inv);
  if constexpr (NR == 24) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = t[8 * k + j] * inv;
      const int4 h = pack_half8(w);
      *reinterpret_cast<int4*>(b + ((size_t)k * f.Vh + cb) * 16) = h;
      unpack_half8(h, w);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[8 * k + j] = (T)(w[j] * n);
    }
    reinterpret_cast<float*>(b + (size_t)48 * f.Vh)[cb] = n;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const __half2 h = __floats2half2_rn(t[2 * k] * inv, t[2 * k + 1] * inv);
      *reinterpret_cast<__half2*>(b + ((size_t)k * f.Vh + cb) * 4) = h;
      const float2 w = __half22float2(h);
      v[2 * k] = (T)(w.x * n);
      v[2 * k + 1] = (T)(w.y * n);
    }
    reinterpret_cast<float*>(b + (size_t)12 * f.Vh)[cb] = n;
  }
}

// ---------------------------------------------------------------- operations
// Each op: void operator()(int site, double acc[3]) const. Complex coefficients are
// `Cf`: a host value, or (scale x) a device value that an earlier reduction or a
// solver's scalar kernel wrote, so solvers need not bring scalars to the host.
template <typename T>
__device__ __forceinline__ void cf_get(const Cf& c, T& r, T& i) {
  if (c.p) {
    r = (T)(c.s * c.p[0]);
    i = (T)(c.s * c.p[1]);
  } else {
    r = (T)c.r;
    i = (T)c.i;
  }
}

template <int NR, typename T> struct OpCopy {
  FieldRef d, s;
  __device__ void operator()(int i, double*) const { T v[NR]; site_load<NR>(s, i, v); site_store<NR>(d, i, v); }
};
// y = a x + b y
template <int NR, typename T> struct OpAxpby {
  FieldRef x, y; Cf a, b;
  __device__ void operator()(int i, double*) const {
    T ar, ai, br, bi;
    cf_get(a, ar, ai);
    cf_get(b, br, bi);
    T u[NR], v[NR];
    site_load<NR>(x, i, u); site_load<NR>(y, i, v);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      T xr = u[2 * k], xi = u[2 * k + 1], yr = v[2 * k], yi = v[2 * k + 1];
      v[2 * k] = ar * xr - ai * xi + br * yr - bi * yi;
      v[2 * k + 1] = ar * xi + ai * xr + br * yi + bi * yr;
    }
    site_store<NR>(y, i, v);
  }
};
// p = r + b p + c v   (BiCGstab direction update with b = beta, c = -beta omega)
template <int NR, typename T> struct OpPUpdate {
  FieldRef r, v, p; Cf b, c;
  __device__ void operator()(int i, double*) const {
    T br, bi, cr, ci;
    cf_get(b, br, bi);
    cf_get(c, cr, ci);
    T ur[NR], uv[NR], up[NR];
    site_load<NR>(r, i, ur); site_load<NR>(v, i, uv); site_load<NR>(p, i, up);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      T pr = up[2 * k], pi = up[2 * k + 1], vr = uv[2 * k], vi = uv[2 * k + 1];
      up[2 * k] = ur[2 * k] + br * pr - bi * pi + cr * vr - ci * vi;
      up[2 * k + 1] = ur[2 * k + 1] + br * pi + bi * pr + cr * vi + ci * vr;
    }
    site_store<NR>(p, i, up);
  }
};
template <int NR, typename T> struct OpNorm2 {
  FieldRef x;
  __device__ void operator()(int i, double* acc) const {
    T u[NR];
    site_load<NR>(x, i, u);
    T s = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) s = fma(u[k], u[k], s);
    acc[0] += (double)s;
  }
};
// (x, y) and ||x||^2
template <int NR, typename T> struct OpCdotNorm {
  FieldRef x, y;
  __device__ void operator()(int i, double* acc) const {
    T u[NR], v[NR];
    site_load<NR>(x, i, u); site_load<NR>(y, i, v);
    T re = 0, im = 0, nn = 0;
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      T xr = u[2 * k], xi = u[2 * k + 1], yr = v[2 * k], yi = v[2 * k + 1];
      re = fma(xr, yr, re); re = fma(xi, yi, re);
      im = fma(xr, yi, im); im = fma(-xi, yr, im);
      nn = fma(xr, xr, nn); nn = fma(xi, xi, nn);
    }
    acc[0] += (double)re; acc[1] += (double)im; acc[2] += (double)nn;
  }
};
template <int NR, typename T>
__device__ __forceinline__ void acc_norm_dot(const T* v, const T* ww, double* acc) {
  T nn = 0;
#pragma unroll
  for (int k = 0; k < NR; ++k) nn = fma(v[k], v[k], nn);
  acc[0] += (double)nn;
  if (ww) {
    T re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      re = fma(ww[2 * k], v[2 * k], re); re = fma(ww[2 * k + 1], v[2 * k + 1], re);
      im = fma(ww[2 * k], v[2 * k + 1], im); im = fma(-ww[2 * k + 1], v[2 * k], im);
    }
    acc[1] += (double)re; acc[2] += (double)im;
  }
}
// y += a x ; ||y||^2, (w, y). Every input is loaded before the store; a w that is y
// itself means the updated y.
template <int NR, typename T, bool DOT> struct OpCaxpyNorm {
  static constexpr int kMinBlocks = sizeof(T) == 4 ? 2 : 1;
  FieldRef x, y, w; Cf a;
  __device__ void operator()(int i, double* acc) const {
    T ar, ai;
    cf_get(a, ar, ai);
    T u[NR], v[NR], ww[DOT ? NR : 1];
    site_load<NR>(x, i, u); site_load<NR>(y, i, v);
    const bool wy = DOT && w.p == y.p;
    if constexpr (DOT) if (!wy) site_load<NR>(w, i, ww);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      T xr = u[2 * k], xi = u[2 * k + 1];
      v[2 * k] += ar * xr - ai * xi;
      v[2 * k + 1] += ar * xi + ai * xr;
    }
    site_store_q<NR>(y, i, v);  // reduce what is stored
    if constexpr (DOT) {
      if (wy)
#pragma unroll
        for (int k = 0; k < NR; ++k) ww[k] = v[k];
      acc_norm_dot<NR, T>(v, ww, acc);
    } else {
      acc_norm_dot<NR, T>(v, nullptr, acc);
    }
  }
};
// ---- all-FP16 Wilson fields (the FP16 Krylov spaces of the mixed solvers): every input
// of a site is loaded as its raw binary16 chunks and norm (13 registers instead of 24) and
// decoded where it is used, so three CTAs fit per SM with all loads of a site in flight.
struct RawH { int4 q[3]; float n; };

__device__ __forceinline__ RawH raw_h(const FieldRef& f, int s) {
  const int q = s >= f.Vh ? 1 : 0;
  const int cb = s - q * f.Vh;
  const char* b = f.p + q * f.hb;
  RawH r;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.q[k] = *reinterpret_cast<const int4*>(b + ((size_t)k * f.Vh + cb) * 16);
  r.n = reinterpret_cast<const float*>(b + (size_t)48 * f.Vh)[cb];
  return r;
}

// decoded exactly as SpinorIO<P16, 24>::load decodes a site
__device__ __forceinline__ void dec_h(const RawH& r, float v[24]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) unpack_half8(r.q[k], v + 8 * k);
#pragma unroll
  for (int k = 0; k < 24; ++k) v[k] *= r.n;
}

static bool all_h24(std::initializer_list<const FieldRef*> fs) {
  for (auto f : fs) if (f->prec != P16 || f->nr != 24) return false;
  return true;
}

// OpCaxpyNorm on all-FP16 Wilson fields
template <bool DOT> struct OpCaxpyNormH {
  static constexpr int kMinBlocks = 3;
  FieldRef x, y, w; Cf a;
  __device__ void operator()(int i, double* acc) const {
    float ar, ai;
    cf_get(a, ar, ai);
    const RawH rx = raw_h(x, i), ry = raw_h(y, i);
    const bool wy = DOT && w.p == y.p;
    RawH rw = rx;  // unused when w is y itself
    if (DOT && !wy) rw = raw_h(w, i);
    float v[24];
    {
      float u[24];
      dec_h(rx, u);
      dec_h(ry, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float xr = u[2 * k], xi = u[2 * k + 1];
        v[2 * k] += ar * xr - ai * xi;
        v[2 * k + 1] += ar * xi + ai * xr;
      }
    }
    site_store_q<24>(y, i, v);  // reduce what is stored
    if constexpr (DOT) {
      float ww[24];
      if (wy) {
#pragma unroll
        for (int k = 0; k < 24; ++k) ww[k] = v[k];
      } else {
        dec_h(rw, ww);
      }
      acc_norm_dot<24, float>(v, ww, acc);
    } else {
      acc_norm_dot<24, float>(v, nullptr, acc);
    }
  }
};

// OpBicgXR with p, s, t, w all-FP16 Wilson fields (xs any non-FP64 precision)
struct OpBicgXRH {
  static constexpr int kMinBlocks = 2;
  FieldRef p, s, t, xs, w; Cf a, b, c;
  __device__ void operator()(int i, double* acc) const {
    float ar, ai, br, bi, cr, ci;
    cf_get(a, ar, ai);
    cf_get(b, br, bi);
    cf_get(c, cr, ci);
    const RawH rp = raw_h(p, i), rs = raw_h(s, i), rt = raw_h(t, i), rw = raw_h(w, i);
    float ux[24], us[24];
    site_load<24>(xs, i, ux);
    dec_h(rs, us);
    {
      float up[24];
      dec_h(rp, up);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        ux[2 * k] += ar * up[2 * k] - ai * up[2 * k + 1] + br * us[2 * k] - bi * us[2 * k + 1];
        ux[2 * k + 1] += ar * up[2 * k + 1] + ai * up[2 * k] + br * us[2 * k + 1] + bi * us[2 * k];
      }
    }
    site_store<24>(xs, i, ux);
    {
      float ut[24];
      dec_h(rt, ut);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float tr = ut[2 * k], ti = ut[2 * k + 1];
        us[2 * k] += cr * tr - ci * ti;
        us[2 * k + 1] += cr * ti + ci * tr;
      }
    }
    site_store_q<24>(s, i, us);
    float ww[24];
    dec_h(rw, ww);
    acc_norm_dot<24, float>(us, ww, acc);
  }
};

// OpScaleCdot on all-FP16 Wilson fields
struct OpScaleCdotH {
  static constexpr int kMinBlocks = 3;
  FieldRef x, y; Cf s;
  __device__ void operator()(int i, double* acc) const {
    float sr, si;
    cf_get(s, sr, si);
    const bool xy = x.p == y.p;
    const RawH rx = raw_h(x, i);
    RawH ry = rx;  // unused when y is x itself
    if (!xy) ry = raw_h(y, i);
    float u[24], v[24];
    dec_h(rx, u);
#pragma unroll
    for (int k = 0; k < 24; ++k) u[k] *= sr;
    site_store_q<24>(x, i, u);
    if (xy) {
#pragma unroll
      for (int k = 0; k < 24; ++k) v[k] = u[k];
    } else {
      dec_h(ry, v);
    }
    float re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re = fma(u[2 * k], v[2 * k], re); re = fma(u[2 * k + 1], v[2 * k + 1], re);
      im = fma(u[2 * k], v[2 * k + 1], im); im = fma(-u[2 * k + 1], v[2 * k], im);
    }
    acc[0] += (double)re; acc[1] += (double)im;
  }
};

// OpCdotNorm on all-FP16 Wilson fields: (x, y) and ||x||^2
struct OpCdotNormH {
  static constexpr int kMinBlocks = 3;
  FieldRef x, y;
  __device__ void operator()(int i, double* acc) const {
    const RawH rx = raw_h(x, i), ry = raw_h(y, i);
    float u[24], v[24];
    dec_h(rx, u);
    dec_h(ry, v);
    float re = 0, im = 0, nn = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float xr = u[2 * k], xi = u[2 * k + 1], yr = v[2 * k], yi = v[2 * k + 1];
      re = fma(xr, yr, re); re = fma(xi, yi, re);
      im = fma(xr, yi, im); im = fma(-xi, yr, im);
      nn = fma(xr, xr, nn); nn = fma(xi, xi, nn);
    }
    acc[0] += (double)re; acc[1] += (double)im; acc[2] += (double)nn;
  }
};

// OpPUpdate on all-FP16 Wilson fields: p = r + b p + c v
struct OpPUpdateH {
  static constexpr int kMinBlocks = 3;
  FieldRef r, v, p; Cf b, c;
  __device__ void operator()(int i, double*) const {
    float br, bi, cr, ci;
    cf_get(b, br, bi);
    cf_get(c, cr, ci);
    const RawH rr = raw_h(r, i), rv = raw_h(v, i), rp = raw_h(p, i);
    float ur[24], up[24];
    dec_h(rp, up);
    dec_h(rr, ur);
    {
      float uv[24];
      dec_h(rv, uv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float pr = up[2 * k], pi = up[2 * k + 1], vr = uv[2 * k], vi = uv[2 * k + 1];
        up[2 * k] = ur[2 * k] + br * pr - bi * pi + cr * vr - ci * vi;
        up[2 * k + 1] = ur[2 * k + 1] + br * pi + bi * pr + cr * vi + ci * vr;
      }
    }
    site_store<24>(p, i, up);
  }
};

// xs += a p + b s ;  s += c t (s becomes r) ; ||r||^2, (w, r)     (BiCGstab; p, s, t
// and xs are distinct and loaded before the first store, w after the last)
template <int NR, typename T> struct OpBicgXR {
  static constexpr int kMinBlocks = sizeof(T) == 4 ? 2 : 1;
  FieldRef p, s, t, xs, w; Cf a, b, c;
  __device__ void operator()(int i, double* acc) const {
    T ar, ai, br, bi, cr, ci;
    cf_get(a, ar, ai);
    cf_get(b, br, bi);
    cf_get(c, cr, ci);
    T up[NR], us[NR], ux[NR], ut[NR];
    site_load<NR>(p, i, up); site_load<NR>(s, i, us); site_load<NR>(xs, i, ux);
    site_load<NR>(t, i, ut);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      ux[2 * k] += ar * up[2 * k] - ai * up[2 * k + 1] + br * us[2 * k] - bi * us[2 * k + 1];
      ux[2 * k + 1] += ar * up[2 * k + 1] + ai * up[2 * k] + br * us[2 * k + 1] + bi * us[2 * k];
    }
    site_store<NR>(xs, i, ux);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      T tr = ut[2 * k], ti = ut[2 * k + 1];
      us[2 * k] += cr * tr - ci * ti;
      us[2 * k + 1] += cr * ti + ci * tr;
    }
    site_store_q<NR>(s, i, us);
    T ww[NR];
    site_load<NR>(w, i, ww);
    acc_norm_dot<NR, T>(us, ww, acc);
  }
};
// xs += a p ; r += c Ap ; ||r||^2     (CG, c = -a; distinct fields, all loaded first)
template <int NR, typename T> struct OpCgUpdate {
  static constexpr int kMinBlocks = sizeof(T) == 4 ? 2 : 1;
  FieldRef p, Ap, xs, r; Cf a, c;
  __device__ void operator()(int i, double* acc) const {
    T ar, ai, cr, ci;
    cf_get(a, ar, ai);
    cf_get(c, cr, ci);
    T up[NR], ux[NR], ua[NR], ur[NR];
    site_load<NR>(p, i, up); site_load<NR>(xs, i, ux);
    site_load<NR>(Ap, i, ua); site_load<NR>(r, i, ur);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      ux[2 * k] += ar * up[2 * k] - ai * up[2 * k + 1];
      ux[2 * k + 1] += ar * up[2 * k + 1] + ai * up[2 * k];
    }
    site_store<NR>(xs, i, ux);
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      ur[2 * k] += cr * ua[2 * k] - ci * ua[2 * k + 1];
      ur[2 * k + 1] += cr * ua[2 * k + 1] + ci * ua[2 * k];
    }
    site_store_q<NR>(r, i, ur);
    acc_norm_dot<NR, T>(ur, nullptr, acc);
  }
};
// x *= s (real part of the coefficient) ; (x, y). y is loaded before the store; a y
// that is x itself means the scaled x.
template <int NR, typename T> struct OpScaleCdot {
  static constexpr int kMinBlocks = sizeof(T) == 4 ? 2 : 1;
  FieldRef x, y; Cf s;
  __device__ void operator()(int i, double* acc) const {
    T sr, si;
    cf_get(s, sr, si);
    T u[NR], v[NR];
    const bool xy = x.p == y.p;
    site_load<NR>(x, i, u);
    if (!xy) site_load<NR>(y, i, v);
#pragma unroll
    for (int k = 0; k < NR; ++k) u[k] *= sr;
    site_store_q<NR>(x, i, u);
    if (xy)
#pragma unroll
      for (int k = 0; k < NR; ++k) v[k] = u[k];
    T re = 0, im = 0;
#pragma unroll
    for (int k = 0; k < NR / 2; ++k) {
      re = fma(u[2 * k], v[2 * k], re); re = fma(u[2 * k + 1], v[2 * k + 1], re);
      im = fma(u[2 * k], v[2 * k + 1], im); im = fma(-u[2 * k + 1], v[2 * k], im);
    }
    acc[0] += (double)re; acc[1] += (double)im;
  }
};
// y = b - y ; ||y||^2
template <int NR, typename T> struct OpXmyNorm {
  FieldRef b, y;
  __device__ void operator()(int i, double* acc) const {
    T u[NR], v[NR];
    site_load<NR>(b, i, u); site_load<NR>(y, i, v);
    T nn = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      v[k] = u[k] - v[k];
      nn = fma(v[k], v[k], nn);
    }
    site_store<NR>(y, i, v);
    acc[0] += (double)nn;
  }
};
struct MultiCoef { FieldRef x[kMaxMulti]; Cf c[kMaxMulti]; int n; };
// y += sum_j c_j x_j. The sum is formed in TS (FP32 when no x_j is FP64) and added to
// y in T, so a GCR restart's FP64 solution update over low-precision directions runs
// at the FP32 rate.
template <int NR, typename T, typename TS> struct OpMultiCaxpy {
  MultiCoef m; FieldRef y;
  __device__ void operator()(int i, double*) const {
    TS s[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) s[k] = 0;
    for (int j = 0; j < m.n; ++j) {
      TS u[NR];
      site_load<NR>(m.x[j], i, u);
      TS cr, ci;
      cf_get(m.c[j], cr, ci);
#pragma unroll
      for (int k = 0; k < NR / 2; ++k) {
        s[2 * k] += cr * u[2 * k] - ci * u[2 * k + 1];
        s[2 * k + 1] += cr * u[2 * k + 1] + ci * u[2 * k];
      }
    }
    T v[NR];
    site_load<NR>(y, i, v);
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] += (T)s[k];
    site_store<NR>(y, i, v);
  }
};

// Multi-shift CG (Eq. 4) update of every still-active shifted system j in one pass:
//   x_j += a_j p_j ;  p_j = z_j r + b_j p_j
// with (a_j, z_j, b_j, active_j) = coef[4 j .. 4 j + 3] written on the device.
struct ShiftFields { FieldRef x[kMaxMulti], p[kMaxMulti]; int n; };
template <int NR, typename T> struct OpMultiShift {
  ShiftFields f; FieldRef r; const double* coef;
  __device__ void operator()(int i, double*) const {
    T ur[NR];
    site_load<NR>(r, i, ur);
    for (int j = 0; j < f.n; ++j) {
      if (coef[4 * j + 3] == 0.0) continue;  // converged: no longer updated
      const T a = (T)coef[4 * j], z = (T)coef[4 * j + 1], b = (T)coef[4 * j + 2];
      T up[NR], ux[NR];
      site_load<NR>(f.p[j], i, up);
      site_load<NR>(f.x[j], i, ux);
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        ux[k] = fma(a, up[k], ux[k]);
        up[k] = fma(b, up[k], z * ur[k]);
      }
      site_store<NR>(f.x[j], i, ux);
      site_store<NR>(f.p[j], i, up);
    }
  }
};

// ---------------------------------------------------------------- kernels
// Resident CTAs per SM that an op asks the register allocator for (its kMinBlocks,
// else 1): the FP32 update-and-reduce ops keep two 256-thread CTAs per SM.
template <class Op, class = void> struct MinBlocks { static constexpr int value = 1; };
template <class Op> struct MinBlocks<Op, std::void_t<decltype(Op::kMinBlocks)>> {
  static constexpr int value = Op::kMinBlocks;
};

template <class Op>
__global__ void __launch_bounds__(kThreads, MinBlocks<Op>::value) blas_map_kernel(Op op, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) op(i, nullptr);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of three values; the result is valid in thread 0.
__device__ __forceinline__ void block_sum3(double acc[3], double (*sh)[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) acc[k] = warp_sum(acc[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) sh[warp][k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      double s = 0;
      for (int w = 0; w < kThreads / 32; ++w) s += sh[w][k];
      acc[k] = s;
    }
  }
  __syncthreads();
}

template <class Op>
__global__ void __launch_bounds__(kThreads, MinBlocks<Op>::value) blas_reduce_kernel(Op op, int n, double* partials,
                                                          unsigned* ticket, double* res) {
  __shared__ double sh[kThreads / 32][3];
  __shared__ bool last;
  double acc[3] = {0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) op(i, acc);
  block_sum3(acc, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) partials[3 * blockIdx.x + k] = acc[k];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s[3] = {0, 0, 0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] += __ldcg(partials + 3 * b + k);
  block_sum3(s, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) res[k] = s[k];
    *ticket = 0;
  }
}

// ---------------------------------------------------------------- host dispatch
static int nsites(const FieldRef& f) { return f.npar * f.Vh; }

static bool any64(std::initializer_list<const FieldRef*> fs) {
  for (auto f : fs) if (f->prec == P64) return true;
  return false;
}

static int check(Blas* b, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
    return DIRAC_ERR_CUDA;
  }
  return DIRAC_OK;
}

template <class Op>
static int run_map(Blas* b, const Op& op, int n, cudaStream_t st) {
  constexpr int kMaxGrid = MinBlocks<Op>::value > 1 ? 152 * MinBlocks<Op>::value : 152 * 16;
  int grid = (n + kThreads - 1) / kThreads;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) grid = 1;
  blas_map_kernel<Op><<<grid, kThreads, 0, st>>>(op, n);
  return check(b, "blas map kernel");
}

template <class Op>
static int run_reduce(Blas* b, const Op& op, int n, double* out, int nout, cudaStream_t st,
                      double* dres) {
  // one wave of resident CTAs when the op asks for several per SM, else 4 per SM
  constexpr int kMaxGrid = MinBlocks<Op>::value > 1 ? 152 * MinBlocks<Op>::value : kRedBlocks;
  static_assert(kMaxGrid <= kRedBlocks, "partials buffer");
  int grid = (n + kThreads - 1) / kThreads;
  if (grid > kMaxGrid) grid = kMaxGrid;
  if (grid < 1) grid = 1;
  blas_reduce_kernel<Op><<<grid, kThreads, 0, st>>>(op, n, b->partials, b->ticket, dres ? dres : b->dev_res);
  int rc = check(b, "blas reduce kernel");
  if (rc || dres) return rc;  // device-resident result: no synchronisation
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    b->err = std::string("reduction sync: ") + cudaGetErrorString(e);
    return DIRAC_ERR_CUDA;
  }
  for (int k = 0; k < nout; ++k) out[k] = ((volatile double*)b->host_res)[k];
  return DIRAC_OK;
}

// Dispatch on (reals per site, arithmetic type).
#define DISPATCH(nr, dbl, BODY)                               \
  do {                                                        \
    if ((nr) == 24) {                                         \
      constexpr int NR = 24;                                  \
      if (dbl) { using T = double; BODY; } else { using T = float; BODY; } \
    } else {                                                  \
      constexpr int NR = 6;                                   \
      if (dbl) { using T = double; BODY; } else { using T = float; BODY; } \
    }                                                         \
  } while (0)

int blas_copy(Blas* b, const FieldRef& dst, const FieldRef& src, cudaStream_t st) {
  DISPATCH(dst.nr, any64({&dst, &src}), return run_map(b, (OpCopy<NR, T>{dst, src}), nsites(dst), st));
}
int blas_zero(Blas* b, const FieldRef& x, cudaStream_t st) {
  if (cudaMemsetAsync(x.p, 0, x.hb * x.npar, st) != cudaSuccess) return check(b, "memset");
  return DIRAC_OK;
}
int blas_axpby(Blas* b, Cf a, const FieldRef& x, Cf bb, const FieldRef& y, cudaStream_t st) {
  DISPATCH(y.nr, any64({&x, &y}), return run_map(b, (OpAxpby<NR, T>{x, y, a, bb}), nsites(y), st));
}
int blas_pupdate(Blas* b, const FieldRef& r, Cf beta, Cf c, const FieldRef& v, const FieldRef& p,
                 cudaStream_t st) {
  if (all_h24({&r, &v, &p})) return run_map(b, (OpPUpdateH{r, v, p, beta, c}), nsites(p), st);
  DISPATCH(p.nr, any64({&r, &v, &p}), return run_map(b, (OpPUpdate<NR, T>{r, v, p, beta, c}), nsites(p), st));
}
int blas_norm2(Blas* b, const FieldRef& x, double* out, cudaStream_t st, double* dres) {
  DISPATCH(x.nr, any64({&x}), return run_reduce(b, (OpNorm2<NR, T>{x}), nsites(x), out, 1, st, dres));
}
int blas_cdot(Blas* b, const FieldRef& x, const FieldRef& y, double out[2], cudaStream_t st, double* dres) {
  if (all_h24({&x, &y})) return run_reduce(b, (OpCdotNormH{x, y}), nsites(x), out, 2, st, dres);
  DISPATCH(x.nr, any64({&x, &y}),
           return run_reduce(b, (OpCdotNorm<NR, T>{x, y}), nsites(x), out, 2, st, dres));
}
int blas_cdot_norm(Blas* b, const FieldRef& x, const FieldRef& y, double out[3], cudaStream_t st,
                   double* dres) {
  if (all_h24({&x, &y})) return run_reduce(b, (OpCdotNormH{x, y}), nsites(x), out, 3, st, dres);
  DISPATCH(x.nr, any64({&x, &y}),
           return run_reduce(b, (OpCdotNorm<NR, T>{x, y}), nsites(x), out, 3, st, dres));
}
int blas_caxpy_norm(Blas* b, Cf a, const FieldRef& x, const FieldRef& y, double* out, cudaStream_t st,
                    double* dres) {
  if (all_h24({&x, &y})) return run_reduce(b, (OpCaxpyNormH<false>{x, y, y, a}), nsites(y), out, 1, st, dres);
  DISPATCH(y.nr, any64({&x, &y}),
           return run_reduce(b, (OpCaxpyNorm<NR, T, false>{x, y, y, a}), nsites(y), out, 1, st, dres));
}
int blas_caxpy_norm_dot(Blas* b, Cf a, const FieldRef& x, const FieldRef& y, const FieldRef& w,
                        double out[3], cudaStream_t st, double* dres) {
  if (all_h24({&x, &y, &w})) return run_reduce(b, (OpCaxpyNormH<true>{x, y, w, a}), nsites(y), out, 3, st, dres);
  DISPATCH(y.nr, any64({&x, &y, &w}),
           return run_reduce(b, (OpCaxpyNorm<NR, T, true>{x, y, w, a}), nsites(y), out, 3, st, dres));
}
int blas_bicg_xr(Blas* b, Cf a, const FieldRef& p, Cf bb, const FieldRef& s, Cf c, const FieldRef& t,
                 const FieldRef& xs, const FieldRef& w, double out[3], cudaStream_t st, double* dres) {
  if (all_h24({&p, &s, &t, &w}) && xs.prec != P64 && xs.nr == 24)
    return run_reduce(b, (OpBicgXRH{p, s, t, xs, w, a, bb, c}), nsites(s), out, 3, st, dres);
  DISPATCH(s.nr, any64({&p, &s, &t, &xs, &w}),
           return run_reduce(b, (OpBicgXR<NR, T>{p, s, t, xs, w, a, bb, c}), nsites(s), out, 3, st, dres));
}
int blas_cg_update(Blas* b, Cf a, const FieldRef& p, Cf c, const FieldRef& Ap, const FieldRef& xs,
                   const FieldRef& r, double* out, cudaStream_t st, double* dres) {
  DISPATCH(r.nr, any64({&p, &Ap, &xs, &r}),
           return run_reduce(b, (OpCgUpdate<NR, T>{p, Ap, xs, r, a, c}), nsites(r), out, 1, st, dres));
}
int blas_scale_cdot(Blas* b, Cf s, const FieldRef& x, const FieldRef& y, double out[2], cudaStream_t st,
                    double* dres) {
  if (all_h24({&x, &y})) return run_reduce(b, (OpScaleCdotH{x, y, s}), nsites(x), out, 2, st, dres);
  DISPATCH(x.nr, any64({&x, &y}),
           return run_reduce(b, (OpScaleCdot<NR, T>{x, y, s}), nsites(x), out, 2, st, dres));
}
int blas_xmy_norm(Blas* b, const FieldRef& bb, const FieldRef& y, double* out, cudaStream_t st, double* dres) {
  DISPATCH(y.nr, any64({&bb, &y}),
           return run_reduce(b, (OpXmyNorm<NR, T>{bb, y}), nsites(y), out, 1, st, dres));
}
int blas_multishift_update(Blas* b, int n, const FieldRef* xs, const FieldRef* ps, const FieldRef& r,
                           const double* coef, cudaStream_t st) {
  if (n < 1 || n > kMaxMulti) {
    b->err = "multi-shift update: 1..16 shifts";
    return DIRAC_ERR_ARG;
  }
  ShiftFields f;
  f.n = n;
  bool dbl = r.prec == P64;
  for (int j = 0; j < n; ++j) {
    f.x[j] = xs[j];
    f.p[j] = ps[j];
    dbl = dbl || xs[j].prec == P64 || ps[j].prec == P64;
  }
  DISPATCH(r.nr, dbl, return run_map(b, (OpMultiShift<NR, T>{f, r, coef}), nsites(r), st));
}

int blas_multi_caxpy(Blas* b, int n, const Cf* c, const FieldRef* xs, const FieldRef& y, cudaStream_t st) {
  for (int j0 = 0; j0 < n; j0 += kMaxMulti) {
    MultiCoef m;
    m.n = n - j0 < kMaxMulti ? n - j0 : kMaxMulti;
    bool xdbl = false;
    for (int j = 0; j < m.n; ++j) {
      m.x[j] = xs[j0 + j];
      m.c[j] = c[j0 + j];
      xdbl = xdbl || xs[j0 + j].prec == P64;
    }
    int rc;
    if (y.prec == P64 && !xdbl) {
      if (y.nr == 24) rc = run_map(b, (OpMultiCaxpy<24, double, float>{m, y}), nsites(y), st);
      else rc = run_map(b, (OpMultiCaxpy<6, double, float>{m, y}), nsites(y), st);
    } else {
      DISPATCH(y.nr, xdbl || y.prec == P64, rc = run_map(b, (OpMultiCaxpy<NR, T, T>{m, y}), nsites(y), st));
    }
    if (rc) return rc;
  }
  return DIRAC_OK;
}

}  // namespace dirac

// ======================================================================== no-alloc
// dirac_cdot_noalloc: the reduction above, for callers that must not allocate GPU
// memory. Its scratch (per-block partial sums and the last-block ticket) is the
// file-scope array below, which every GPU that loads the library holds until exit.
namespace dirac {

static constexpr int kNoAllocThreads = 256;
static constexpr int kNoAllocSitesPerThread = 8;
static constexpr int kNoAllocMaxBlocks = 4096;
// sites one call may cover: 4096 blocks x 256 threads x 8 sites = 8,388,608
static constexpr long long kNoAllocMaxSites =
    (long long)kNoAllocMaxBlocks * kNoAllocThreads * kNoAllocSitesPerThread;
// 3 partial sums per block, then one 64-bit slot for the ticket: 98,312 bytes
static __device__ __align__(256) unsigned long long g_noalloc_scratch[3 * kNoAllocMaxBlocks + 1];

static std::mutex g_noalloc_mu;
// Device address of the array per device, and the id of the CUDA context it was looked
// up in: a device reset (or another context on the same device) loads the module again,
// possibly at another address, so the address is looked up again when the id changes.
static void* g_noalloc_addr[128] = {};
static unsigned long long g_noalloc_ctx[128] = {};

// Id of the current CUDA context (0 if none is current or the driver lacks the call),
// through the runtime's driver entry points so that the library needs no -lcuda.
static unsigned long long noalloc_ctx_id() {
  typedef int (*get_current_t)(void**);
  typedef int (*get_id_t)(void*, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (get_current_t)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (get_id_t)f;
    cudaGetLastError();
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// true when the GPU can address p as device memory (device or managed allocation)
static bool noalloc_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // the query's own error, nothing was pending before it
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int noalloc_fail(char* err, size_t len, int code, const std::string& msg) {
  if (err && len) {
    size_t n = msg.size() < len - 1 ? msg.size() : len - 1;
    std::memcpy(err, msg.data(), n);
    err[n] = 0;
  }
  return code;
}

}  // namespace dirac

extern "C" int dirac_cdot_noalloc(const void* x, const void* y, dirac_prec prec, int reals_per_site,
                                  long long sites_per_parity, dirac_parity parity, double* result,
                                  void* stream, char* err, size_t err_len) {
  using namespace dirac;
  if (err && err_len) err[0] = 0;
  if (!x || !y || !result)
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG, "dirac_cdot_noalloc: null pointer");
  if (prec != DIRAC_PREC_F64 && prec != DIRAC_PREC_F32 && prec != DIRAC_PREC_F16)
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG, "dirac_cdot_noalloc: unknown precision");
  if (reals_per_site != 24 && reals_per_site != 6)
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG, "dirac_cdot_noalloc: reals_per_site must be 24 or 6");
  if (parity < DIRAC_PARITY_FULL || parity > DIRAC_PARITY_ODD || sites_per_parity < 1 ||
      sites_per_parity > 0x3fffffffLL)
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG, "dirac_cdot_noalloc: bad parity or size");
  const long long n = (parity == DIRAC_PARITY_FULL ? 2 : 1) * sites_per_parity;
  if (n > kNoAllocMaxSites)
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG,
                        "dirac_cdot_noalloc: " + std::to_string(n) + " sites exceed the maximum of " +
                            std::to_string(kNoAllocMaxSites) + " for its fixed scratch array");
  // an error left by earlier asynchronous work is reported, not taken over: peek (the
  // caller can still read it) and queue nothing
  cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return noalloc_fail(err, err_len, DIRAC_ERR_CUDA,
                        std::string("dirac_cdot_noalloc: an earlier CUDA error is pending (") +
                            cudaGetErrorString(pending) + "); nothing was queued");
  // the kernel dereferences all three pointers: a host pointer would fault the GPU
  if (!noalloc_device_ptr(x) || !noalloc_device_ptr(y))
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG, "dirac_cdot_noalloc: x and y must be device memory");
  if (!noalloc_device_ptr(result))
    return noalloc_fail(err, err_len, DIRAC_ERR_ARG,
                        "dirac_cdot_noalloc: result must be device memory (3 doubles)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128)
    return noalloc_fail(err, err_len, DIRAC_ERR_CUDA, "dirac_cdot_noalloc: cudaGetDevice failed");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = noalloc_ctx_id();
    if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
      // set-up, with the device current: the host-side name of the array is not a
      // device address, so ask the runtime for the real one (again after a reset)
      void* a = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        return noalloc_fail(err, err_len, DIRAC_ERR_CUDA,
                            std::string("dirac_cdot_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_noalloc_addr[dev] = a;
      g_noalloc_ctx[dev] = noalloc_ctx_id();
    }
    base = g_noalloc_addr[dev];
  }
  double* partials = reinterpret_cast<double*>(base);
  unsigned* ticket = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned long long*>(base) + 3 * kNoAllocMaxBlocks);
  cudaStream_t st = (cudaStream_t)stream;
  // the ticket must start at zero; the partial sums are written before they are read
  if (cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return noalloc_fail(err, err_len, DIRAC_ERR_CUDA, "dirac_cdot_noalloc: clearing the ticket failed");
  FieldRef fx, fy;
  fx.p = (char*)x;
  fy.p = (char*)y;
  fx.prec = fy.prec = prec;
  fx.nr = fy.nr = reals_per_site;
  fx.Vh = fy.Vh = (int)sites_per_parity;
  fx.npar = fy.npar = parity == DIRAC_PARITY_FULL ? 2 : 1;
  fx.hb = fy.hb = spinor_half_bytes(prec, reals_per_site, sites_per_parity);
  const long long per_block = (long long)kNoAllocThreads * kNoAllocSitesPerThread;
  const int grid = (int)((n + per_block - 1) / per_block);
  const bool dbl = prec == DIRAC_PREC_F64;
  if (reals_per_site == 24) {
    if (dbl) blas_reduce_kernel<OpCdotNorm<24, double>><<<grid, kNoAllocThreads, 0, st>>>(
        OpCdotNorm<24, double>{fx, fy}, (int)n, partials, ticket, result);
    else blas_reduce_kernel<OpCdotNorm<24, float>><<<grid, kNoAllocThreads, 0, st>>>(
        OpCdotNorm<24, float>{fx, fy}, (int)n, partials, ticket, result);
  } else {
    if (dbl) blas_reduce_kernel<OpCdotNorm<6, double>><<<grid, kNoAllocThreads, 0, st>>>(
        OpCdotNorm<6, double>{fx, fy}, (int)n, partials, ticket, result);
    else blas_reduce_kernel<OpCdotNorm<6, float>><<<grid, kNoAllocThreads, 0, st>>>(
        OpCdotNorm<6, float>{fx, fy}, (int)n, partials, ticket, result);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(err, err_len, DIRAC_ERR_CUDA, std::string("dirac_cdot_noalloc: launch: ") + cudaGetErrorString(e));
  return DIRAC_OK;
}
