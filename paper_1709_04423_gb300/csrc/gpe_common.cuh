// gpe_common.cuh -- shared device helpers of the GB300 split-step
// Crank-Nicolson GP library: complex types, line geometry, FP64 block
// reductions with a deterministic last-block finish.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "gpe_df.cuh"

namespace gpe {

// ---- the bounds-checking build (-DGPE_BOUNDS_CHECK, libgpe_check.so)
// GPE_CHECK(cond, code) tests an index before a global or shared-memory
// access; a failed test records its code (the first one per translation
// unit) in this unit's device flag and the caller skips the access -- no
// assert, no trap.  Each translation unit registers a reader of its flag at
// load time; gp_check_status collects them.  In the normal build the checks
// compile to nothing.
#ifdef GPE_BOUNDS_CHECK
static __device__ int g_check_first = 0;
#define GPE_CHECK(cond, code) ((cond) ? true : (atomicCAS(&::gpe::g_check_first, 0, (code)), false))
void register_check_reader(int (*reader)());
namespace {
int read_check_flag() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_check_first, sizeof(int)) != cudaSuccess) return -1;
  cudaMemcpyToSymbol(g_check_first, &z, sizeof(int));
  return v;
}
struct CheckReaderReg {
  CheckReaderReg() { register_check_reader(&read_check_flag); }
};
CheckReaderReg g_check_reader_reg;
}  // namespace
#else
#define GPE_CHECK(cond, code) true
#endif

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };
template <> struct C2<df64> { using type = df64x2; };
template <typename T> struct is_df { static constexpr bool value = false; };
template <> struct is_df<df64> { static constexpr bool value = true; };
template <typename T> using c2_t = typename C2<T>::type;

template <typename T> __device__ __forceinline__ c2_t<T> mk(T x, T y) { c2_t<T> r; r.x = x; r.y = y; return r; }
// Complex product with its fused multiply-adds spelled out, so that the
// rounding does not depend on how the compiler contracts the expression in a
// given kernel (the batched and the single-grid kernels then agree bit for bit).
template <typename T> __device__ __forceinline__ c2_t<T> cmul(c2_t<T> a, c2_t<T> b) {
  if constexpr (is_df<T>::value) return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  else return mk<T>(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}

// exp(-i th) p (FP32 and FP64 states), as p + ((c - 1) p + s (p.y, -p.x))
// with c - 1 = -2 sin^2(th/2) and s = 2 sin(th/2) cos(th/2) (or their series
// for small FP32 angles, rot_coefs).  The rounded
// pair (1 + (c - 1), s) has modulus 1 + O(th^2 eps); a rounded cos(th) next
// to 1 would instead carry an error of up to half an ulp of 1 in the
// modulus, the same at a point step after step (th changes slowly), so that
// |phi| would drift linearly with the number of steps.  What remains is the
// rounding of the final sums, which is unbiased.
// The Taylor series of s = sin th and cm1 = cos th - 1: for FP32 angles
// |th| < 1/8 s to th^7 and cm1 to th^8, for |th| < 1/32 s to th^5 and cm1 to
// th^6; in both ranges the first omitted terms are below 2e-13 relative.
__device__ __forceinline__ void rot_coefs_series(float th, float& s, float& cm1) {
  const float t2 = th * th;
  s = th * fmaf(t2, fmaf(t2, fmaf(t2, float(-1.0 / 5040), float(1.0 / 120)), float(-1.0 / 6)), 1.0f);
  cm1 = t2 * fmaf(t2, fmaf(t2, fmaf(t2, float(1.0 / 40320), float(-1.0 / 720)), float(1.0 / 24)), -0.5f);
}
__device__ __forceinline__ void rot_coefs_series_short(float th, float& s, float& cm1) {
  const float t2 = th * th;
  s = th * fmaf(t2, fmaf(t2, float(1.0 / 120), float(-1.0 / 6)), 1.0f);
  cm1 = t2 * fmaf(t2, fmaf(t2, float(-1.0 / 720), float(1.0 / 24)), -0.5f);
}

// s = sin th and cm1 = cos th - 1 (the coefficients of rot_neg): FP32 with
// |th| < 1/8 their series (rot_coefs_series_short below 1/32), else from the
// half angle.
template <typename T> __device__ __forceinline__ void rot_coefs(T th, T& s, T& cm1) {
  if constexpr (std::is_same<T, float>::value) {
    const float a = fabsf(th);
    if (a < 0.03125f) {
      rot_coefs_series_short(th, s, cm1);
      return;
    }
    if (a < 0.125f) {
      rot_coefs_series(th, s, cm1);
      return;
    }
  }
  {
    T sh, ch;
    sincos(T(0.5) * th, &sh, &ch);
    s = T(2) * (sh * ch);
    cm1 = T(-2) * (sh * sh);
  }
}

// p + ((c - 1) p + s (p.y, -p.x)) for given coefficients
template <typename T> __device__ __forceinline__ c2_t<T> rot_apply(c2_t<T> p, T s, T cm1) {
  return mk<T>(p.x + fma(cm1, p.x, s * p.y), p.y + fma(cm1, p.y, -(s * p.x)));
}

template <typename T> __device__ __forceinline__ c2_t<T> rot_neg(c2_t<T> p, T th) {
  T s, cm1;
  rot_coefs<T>(th, s, cm1);
  return rot_apply<T>(p, s, cm1);
}

// Geometry of the lines of one sweep.  Line L of axis 0 starts at L*nx
// (L = j + ny*k); of axis 1 at (L % nx) + (L / nx)*nx*ny (L = i + nx*k); of
// axis 2 at L (L = i + nx*j).  Consecutive L of axes 1 and 2 are
// neighbouring x positions, so a warp of consecutive lines reads whole rows.
struct LineGeom {
  int axis;
  int n;        // points along the line
  long stride;  // element distance between consecutive points
  long nlines;
  int nx, ny, nz;
  // elements of the array the lines live in (the bounds the checks of the
  // checking build hold every index to)
  __host__ __device__ long points() const { return (long)nx * ny * nz; }
};

__device__ __forceinline__ long line_base(const LineGeom& g, long L) {
  if (g.axis == 0) return L * g.nx;
  if (g.axis == 1) return (L % g.nx) + (L / g.nx) * (long)g.nx * g.ny;
  return L;
}

// The two transverse indices (a, b) of line L: axis 0 -> (j, k), axis 1 ->
// (i, k), axis 2 -> (i, j).
__device__ __forceinline__ void line_transverse(const LineGeom& g, long L, int& a, int& b) {
  if (g.axis == 0) { a = (int)(L % g.ny); b = (int)(L / g.ny); }
  else { a = (int)(L % g.nx); b = (int)(L / g.nx); }
}

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel
// launched as a programmatic dependent of the previous kernel in its stream
// may start while that kernel is still running: pdl_wait() blocks until the
// previous grid has completed and its memory is visible (it returns at once
// when the kernel was launched normally), so everything before it may only
// touch data no earlier kernel writes (the coefficient tables); pdl_release()
// lets the next kernel be scheduled before this one ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums K per-thread doubles over the block; thread 0 gets the totals.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* >= 32*K */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) smem[warp * K + q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      double s = lane < nw ? smem[lane * K + q] : 0.0;
      v[q] = warp_sum(s);
    }
  }
}

// Writes the block's K totals to partials[blockIdx.x*K + q]; the last block to
// finish sums all partials in block order (deterministic) and returns true
// with the totals in tot[] (valid in thread 0 of that block only).  The
// counter is reset for the next launch.
template <int K>
__device__ __forceinline__ bool grid_sum_last(double (&v)[K], double* partials, unsigned int* counter,
                                              double (&tot)[K], double* smem) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) partials[(long)blockIdx.x * K + q] = v[q];
    __threadfence();
    unsigned int done = atomicAdd(counter, 1u);
    is_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // fixed-order sum: thread t takes blocks t, t+blockDim, ...; then the block tree
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] += __ldcg(&partials[(long)b * K + q]);
  }
  block_sum<K>(acc, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) tot[q] = acc[q];
    *counter = 0u;
  }
  return true;
}

// Pending renormalisation factor of an imaginary-time step's input.  The
// previous step's last sweep left one norm sum per block in parts[0..nparts);
// one warp of every block of the reading kernel sums them in the same fixed
// order (lane-strided FP64 sums, then a butterfly), so all blocks -- and every
// run -- obtain the same factor 1/sqrt(wscale * total).
__device__ __forceinline__ double pending_factor_warp(const double* parts, int nparts, double wscale) {
  double acc = 0.0;
  for (int b = threadIdx.x & 31; b < nparts; b += 32) acc += __ldcg(&parts[b]);
  return 1.0 / sqrt(warp_sum(acc) * wscale);
}

// The same for the whole block: parts == nullptr means no pending factor (1).
// Every thread of the block must call it (two block barriers).
__device__ __forceinline__ double pending_scale(const double* parts, int nparts, double wscale, double* smem) {
  if (!parts) return 1.0;
  if (threadIdx.x < 32) {
    const double f = pending_factor_warp(parts, nparts, wscale);
    if (threadIdx.x == 0) smem[0] = f;
  }
  __syncthreads();
  const double f = smem[0];
  __syncthreads();  // smem free again
  return f;
}

// Opts a kernel in to `bytes` of dynamic shared memory (beyond the default
// 48 KB) once per kernel and size.  The record is this library's own (an
// internal-linkage table keyed by the kernel's host stub): a function-local
// static in a launcher template would be one object for every copy of the
// library in the process, so that a second copy (the checking build) would
// skip the opt-in for its own kernels.
namespace {
inline void opt_in_smem(const void* kern, size_t bytes) {
  static std::mutex m;
  static std::vector<std::pair<const void*, size_t>> done;
  std::lock_guard<std::mutex> lock(m);
  for (auto& d : done)
    if (d.first == kern) {
      if (d.second >= bytes) return;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      d.second = bytes;
      return;
    }
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done.emplace_back(kern, bytes);
}
}  // namespace

// Launch with or without the programmatic-dependent-launch attribute (the
// kernel must call pdl_wait() before it reads what earlier kernels wrote).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace gpe
