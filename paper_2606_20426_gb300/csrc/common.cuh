// Shared device helpers for the TaCauchy sm_103a kernels.
//
// R is the compute type of a kernel (float in TC_FP32_MIXED, double in
// TC_FP64); every reduction accumulates in double.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tacauchy.h"

#define TC_HD __host__ __device__ __forceinline__
#define TC_D __device__ __forceinline__

namespace tc {

constexpr int kBlock = 256;  // threads per block of the streaming kernels
constexpr int kWarp = 32;

// Device status bits, OR-ed into Scalars::status by kernels.
enum : int {
  ST_NONFINITE = 1,
  ST_INVALID_MESH = 2,
  ST_CAPACITY = 4,
  ST_PENETRATION = 8,
};

// Per-env device scalars (one struct in device memory).
struct Scalars {
  double energy;       // last evaluated total energy
  double gnorm2;       // |g_free|^2
  double rz, rz_next;  // PCG r.z (current, and the value of the next iteration)
  double pq;           // PCG p.(A p)
  double rr;           // PCG r.r
  double pcg_tol2;     // (eta |g|)^2
  double pmax;         // max-norm of the Newton direction
  double ccd_t;        // conservative fraction of the motion (min over pairs)
  double reduce_tmp[8];
  double force[3];     // contact force accumulator
  int status;          // ST_* bits
  int pcg_done;        // set when |r| <= tol
  int pcg_iters;       // iterations taken by the last solve
  int overflow;        // grid/pair capacity overflow
  int pcg_capped;      // the last solve stopped at the env's pcg_max above its tolerance
};

template <class R> struct Vec3 {
  R x, y, z;
};

template <class R> TC_HD Vec3<R> v3(R x, R y, R z) { return Vec3<R>{x, y, z}; }
template <class R> TC_HD Vec3<R> operator+(Vec3<R> a, Vec3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R> TC_HD Vec3<R> operator-(Vec3<R> a, Vec3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R> TC_HD Vec3<R> operator*(R s, Vec3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class R> TC_HD R dot(Vec3<R> a, Vec3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> TC_HD Vec3<R> cross(Vec3<R> a, Vec3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class R> TC_HD R& at(Vec3<R>& a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// SoA triple of arrays (x, y, z components).
template <class R> struct SoA3 {
  R* x;
  R* y;
  R* z;
  TC_HD Vec3<R> get(int64_t i) const { return {x[i], y[i], z[i]}; }
  TC_HD void set(int64_t i, Vec3<R> v) const { x[i] = v.x; y[i] = v.y; z[i] = v.z; }
};

// ---------------------------------------------------------------- reductions

TC_D double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
TC_D double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
TC_D double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------- double-float
// On this part FP64 instructions issue at a small fraction of the FP32 rate,
// so accumulators that must carry more than 24 bits use an unevaluated pair
// of floats (hi + lo, Dekker / Knuth error-free transformations): products of
// two floats are exact (FMA residual), sums keep ~48 bits.
struct DF {
  float hi, lo;
};
TC_D DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
TC_D DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  const float e = s.lo + x.lo + y.lo;
  const float h = s.hi + e;
  return {h, e - (h - s.hi)};
}
TC_D DF df_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
// a / b rounded to float from double-float operands (b != 0): the quotient
// of the leading parts, corrected once by the FMA residual of a - q b.
TC_D float df_ratio(DF a, DF b) {
  const float q0 = a.hi / b.hi;
  const float e = fmaf(-q0, b.hi, a.hi) + (a.lo - q0 * b.lo);
  return q0 + e / b.hi;
}
TC_D DF df_from_double(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
TC_D DF df_shfl_xor(DF v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// Asynchronous global -> shared copy of one 4- or 8-byte word (no register
// holds it in flight); complete once the issuing thread passes
// cp_async_wait_all.
template <class T> TC_D void cp_async_word(T* smem_dst, const T* gmem_src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte words");
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const size_t g = __cvta_generic_to_global(gmem_src);
  if (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(g) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(g) : "memory");
}
TC_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Accumulator of a precision: double-float for FP32 work, double for FP64.
template <class R> struct Acc;
template <> struct Acc<float> {
  using T = DF;
  static TC_D T zero() { return {0.f, 0.f}; }
  static TC_D T prod(float a, float b) { return df_prod(a, b); }
  static TC_D T add(T a, T b) { return df_add(a, b); }
  static TC_D T shfl_xor(T v, int o) { return df_shfl_xor(v, o); }
  static TC_D double to_double(T v) { return (double)v.hi + (double)v.lo; }
  static TC_D T from_double(double x) { return df_from_double(x); }
  static TC_D float ratio(T a, T b) { return df_ratio(a, b); }
  static TC_D bool positive(T a) { return a.hi > 0.f; }
};
template <> struct Acc<double> {
  using T = double;
  static TC_D T zero() { return 0.0; }
  static TC_D T prod(double a, double b) { return a * b; }
  static TC_D T add(T a, T b) { return a + b; }
  static TC_D T shfl_xor(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  static TC_D double to_double(T v) { return v; }
  static TC_D T from_double(double x) { return x; }
  static TC_D double ratio(T a, T b) { return a / b; }
  static TC_D bool positive(T a) { return a > 0.0; }
};

// Block sums of NV accumulators per thread (fixed tree); totals in s[k][0]
// after the call, visible to every thread.
template <class R, int NV> TC_D void block_acc_sum(typename Acc<R>::T* v, typename Acc<R>::T (*s)[32]) {
  using A = Acc<R>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    typename A::T x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = A::add(x, A::shfl_xor(x, o));
    if (lane == 0) s[k][w] = x;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      typename A::T x = lane < (int)(blockDim.x >> 5) ? s[k][lane] : A::zero();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = A::add(x, A::shfl_xor(x, o));
      if (lane == 0) s[k][0] = x;
    }
  }
  __syncthreads();
}

// Block sum of one double per thread; result valid in thread 0.
// Fixed combination order -> deterministic.
template <int NT> TC_D double block_sum(double v) {
  __shared__ double s[NT / kWarp];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < NT / kWarp ? s[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}
template <int NT> TC_D double block_max(double v) {
  __shared__ double s[NT / kWarp];
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s[w] = v;
  __syncthreads();
  double r = -1e308;
  if (w == 0) {
    r = lane < NT / kWarp ? s[lane] : -1e308;
    r = warp_max(r);
  }
  __syncthreads();
  return r;
}
template <int NT> TC_D double block_min(double v) {
  __shared__ double s[NT / kWarp];
  v = warp_min(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s[w] = v;
  __syncthreads();
  double r = 1e308;
  if (w == 0) {
    r = lane < NT / kWarp ? s[lane] : 1e308;
    r = warp_min(r);
  }
  __syncthreads();
  return r;
}

inline unsigned grid_for(int64_t n, int nt = kBlock) {
  int64_t b = (n + nt - 1) / nt;
  return (unsigned)(b < 1 ? 1 : b);
}

// Index of (i, j), i <= j, in packed upper-triangular storage of an N x N
// symmetric matrix (row-major upper triangle).
TC_HD int sym_index(int i, int j, int N) {
  if (i > j) { int t = i; i = j; j = t; }
  return i * N - (i * (i - 1)) / 2 + (j - i);
}

TC_D bool finite_d(double v) { return isfinite(v); }

}  // namespace tc
