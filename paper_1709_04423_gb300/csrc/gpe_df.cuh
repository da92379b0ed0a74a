// gpe_df.cuh -- double-float ("df64") real numbers for the FP64-accuracy form
// that runs on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  Arithmetic uses the error-free transformations
// of floating-point sums and products: two-sum (Knuth, TAOCP vol. 2, 4.2.2:
// s = a + b exactly as s + e) and two-product via a fused multiply-add
// (p = a b exactly as p + fma(a, b, -p)), followed by renormalisation.  Every
// float operation is written with the round-to-nearest intrinsics so that the
// compiler cannot contract or reassociate the error terms.
//
// On this GPU the FP32 pipes are about 70 times faster than FP64, so a
// double-float operation of 5-20 float instructions still outpaces a native
// FP64 one several times over; the state keeps 16 bytes per complex value.
// Accuracy: relative error of a few 2^-48 per operation, against 2^-53 for
// FP64.  Range: that of float (magnitudes below ~1e-38 flush to zero, and the
// low word loses precision below ~1e-31).
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace gpe {
// The type and its functions live in their own namespace: argument-dependent
// lookup finds them for df64 arguments, while unqualified calls on double
// and float inside namespace gpe keep resolving to the standard functions.
namespace dfl {

struct __align__(8) df64 {
  float hi, lo;
  __host__ __device__ constexpr df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // constexpr so that literal constants are split at compile time
  __host__ __device__ constexpr df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr df64(int v) : df64((double)v) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

#if defined(__CUDA_ARCH__)
#define GPE_FADD(a, b) __fadd_rn(a, b)
#define GPE_FSUB(a, b) __fsub_rn(a, b)
#define GPE_FMUL(a, b) __fmul_rn(a, b)
#define GPE_FFMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define GPE_FADD(a, b) ((a) + (b))
#define GPE_FSUB(a, b) ((a) - (b))
#define GPE_FMUL(a, b) ((a) * (b))
#define GPE_FFMA(a, b, c) std::fma(a, b, c)
#endif

// s + e = a + b exactly (Knuth two-sum)
__host__ __device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = GPE_FADD(a, b);
  const float bb = GPE_FSUB(s, a);
  e = GPE_FADD(GPE_FSUB(a, GPE_FSUB(s, bb)), GPE_FSUB(b, bb));
}
// s + e = a + b exactly, given |a| >= |b|
__host__ __device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = GPE_FADD(a, b);
  e = GPE_FSUB(b, GPE_FSUB(s, a));
}

__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e = GPE_FADD(e, GPE_FADD(a.lo, b.lo));
  float h, l;
  df_fast_two_sum(s, e, h, l);
  return df64(h, l);
}
__host__ __device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = GPE_FMUL(a.hi, b.hi);
  float e = GPE_FFMA(a.hi, b.hi, -p);                 // exact error of the leading product
  e = GPE_FFMA(a.hi, b.lo, e);
  e = GPE_FFMA(a.lo, b.hi, e);
  float h, l;
  df_fast_two_sum(p, e, h, l);
  return df64(h, l);
}
__host__ __device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__host__ __device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__host__ __device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__host__ __device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) { return a * b + c; }
__host__ __device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }
__host__ __device__ __forceinline__ bool operator<(df64 a, df64 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }

// Transcendentals are only reached outside the polynomial ranges of the
// sub-step N; they go through FP64.
__device__ __forceinline__ df64 exp(df64 a) { return df64(::exp((double)a)); }
__device__ __forceinline__ void sincos(df64 a, df64* s, df64* c) {
  double sd, cd;
  ::sincos((double)a, &sd, &cd);
  *s = df64(sd);
  *c = df64(cd);
}
__device__ __forceinline__ df64 sqrt(df64 a) { return df64(::sqrt((double)a)); }

__device__ __forceinline__ df64 shfl_xor_t(df64 v, int o) {
  return df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ df64 shfl_up_t(df64 v, int o) {
  return df64(__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ df64 shfl_down_t(df64 v, int o) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}

struct __align__(16) df64x2 {  // one 16-byte access per complex value
  df64 x, y;
};

// cache-hinted loads of the complex value (the overloads of the float4 forms)
__device__ __forceinline__ df64x2 __ldcg(const df64x2* p) {
  const float4 v = ::__ldcg(reinterpret_cast<const float4*>(p));
  return df64x2{df64(v.x, v.y), df64(v.z, v.w)};
}
__device__ __forceinline__ df64x2 __ldg(const df64x2* p) {
  const float4 v = ::__ldg(reinterpret_cast<const float4*>(p));
  return df64x2{df64(v.x, v.y), df64(v.z, v.w)};
}

// Exact multiple by a power of two (no rounding: both words scale exactly).
__host__ __device__ __forceinline__ df64 df_scale(df64 a, float pow2) {
  return df64(GPE_FMUL(a.hi, pow2), GPE_FMUL(a.lo, pow2));
}
// a * b with a plain float b (one partial product fewer than df64 * df64)
__host__ __device__ __forceinline__ df64 df_mulf(df64 a, float b) {
  const float p = GPE_FMUL(a.hi, b);
  float e = GPE_FFMA(a.hi, b, -p);
  e = GPE_FFMA(a.lo, b, e);
  float h, l;
  df_fast_two_sum(p, e, h, l);
  return df64(h, l);
}

// Triple-float complex factor: re = re[0] + re[1] + re[2] (likewise im), ~72
// significant bits, so that it holds an FP64 value exactly.  The potential
// factors of the sub-step N are kept in this form: a factor applied every
// step would otherwise repeat its own 48-bit rounding coherently, step after
// step, while the rounding of each product with the evolving state is not
// correlated from one step to the next.
struct __align__(8) tf3c {
  float re[3];
  float im[3];
};

// Exact split of a double into three floats (the remainders v - t0 and
// v - t0 - t1 are exact in double; the last one has at most 5 significant bits
// left over).
__host__ __device__ inline void tf_split(double v, float* t) {
  t[0] = (float)v;
  const double r = v - (double)t[0];
  t[1] = (float)r;
  t[2] = (float)(r - (double)t[1]);
}

// Error of f * p accumulated in one float (f triple, p double-float); the
// partial products below f2 p.hi are under 2^-72 relative and dropped.
__device__ __forceinline__ float tf_err(const float* f, df64 p, float e) {
  e = GPE_FFMA(f[0], p.lo, e);
  e = GPE_FFMA(f[1], p.hi, e);
  e = GPE_FFMA(f[1], p.lo, e);
  e = GPE_FFMA(f[2], p.hi, e);
  return e;
}

// f * p for a real triple-float f
__device__ __forceinline__ df64 tf_mul(const float* f, df64 p) {
  const float P = GPE_FMUL(f[0], p.hi);
  const float e = tf_err(f, p, GPE_FFMA(f[0], p.hi, -P));
  float h, l;
  df_two_sum(P, e, h, l);
  return df64(h, l);
}

// f * p - g * q as one dot product with a single final renormalisation
__device__ __forceinline__ df64 tf_dot2(const float* f, df64 p, const float* g, df64 q) {
  const float P1 = GPE_FMUL(f[0], p.hi), P2 = GPE_FMUL(g[0], q.hi);
  float s, es;
  df_two_sum(P1, -P2, s, es);
  float e = tf_err(f, p, GPE_FFMA(f[0], p.hi, -P1));
  float e2 = tf_err(g, q, GPE_FFMA(g[0], q.hi, -P2));
  e = GPE_FADD(GPE_FSUB(e, e2), es);
  float h, l;
  df_two_sum(s, e, h, l);
  return df64(h, l);
}

}  // namespace dfl

using dfl::df64;
using dfl::df64x2;
using dfl::tf3c;
using dfl::tf_split;

// warp shuffles of the state's real type (df64 overloads found by lookup in dfl)
template <typename T>
__device__ __forceinline__ T shfl_xor_t(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <typename T>
__device__ __forceinline__ T shfl_up_t(T v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <typename T>
__device__ __forceinline__ T shfl_down_t(T v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

}  // namespace gpe
