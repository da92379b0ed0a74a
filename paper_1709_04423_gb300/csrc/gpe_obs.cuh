// gpe_obs.cuh -- FP64 Simpson-rule reductions for the observables the paper's
// programs report (abstract; "Summary of revisions": energy, chemical
// potential, root-mean-square sizes, densities).
//
// One pass over the grid accumulates, with tensor-product Simpson weights w,
//   S0 = sum w |phi|^2                       (norm)
//   S1 = sum w 1/2 sum_d |d_d phi|^2         (kinetic)
//   S2 = sum w V |phi|^2                     (potential)
//   S3 = sum w |phi|^4                       (interaction)
//   S4..S6 = sum w x_d^2 |phi|^2             (second moments)
// The weights are either the FP64 Simpson weights or, for an FP32 state,
// the exact Simpson coefficients (1, 2, 4) with the factor prod dx/3 applied
// to the FP64 totals.
// The per-point terms are formed in the arithmetic type R of the state (float
// for an FP32 state, double otherwise) and summed per thread in R over the
// thread's 10-100 points; the per-thread sums are then reduced over the
// block (warp shuffles) and the grid (fixed order) in FP64.  FP32 rounding
// of the terms is of the size of the FP32 state's own rounding and averages
// out over the grid; an FP64 term per point would cost more than the
// propagation steps themselves on a part whose FP64 rate is 1/70 of FP32.
// The host turns the sums into
// E = (S1+S2)/S0 + g/2 S3/S0^2, mu = (S1+S2)/S0 + g S3/S0^2, rms_d = sqrt(S_{4+d}/S0).
// Derivatives: 4th-order central differences for 2 <= i <= n-3, 2nd-order at
// i = 1, n-2, zero at the end points.  Optionally writes |phi|^2 (FP64).
#pragma once
#include "gpe_common.cuh"

namespace gpe {

// arithmetic type of the per-point terms
template <typename T> struct ObsReal { using type = double; };
template <> struct ObsReal<float> { using type = float; };
template <typename T> using obs_r = typename ObsReal<T>::type;

template <typename T>
struct ObsArgs {
  const c2_t<T>* psi;
  int dim, nx, ny, nz;
  double hx, hy, hz;        // grid spacings
  const double* V;          // full potential or nullptr
  // per-axis tables in the arithmetic type: separable trap terms, coordinates,
  // Simpson weights
  const obs_r<T>* vx; const obs_r<T>* vy; const obs_r<T>* vz;
  const obs_r<T>* cx; const obs_r<T>* cy; const obs_r<T>* cz;
  const obs_r<T>* wx; const obs_r<T>* wy; const obs_r<T>* wz;
  double wscale;            // factor of the FP64 totals (1, or prod dx/3 with coefficient weights)
  // radial problem of the spherical trap: weight of the |psi|^4 term per x
  // index (1/(4 pi r^2)); nullptr for the other grids.  x0: how the x
  // derivative treats the start of the axis -- 0 Cartesian (R8), 1 the
  // spherical u's odd extension (u'(0) = u_1/dx), 2 the even extension across
  // the axis of a circular or axial trap (point 0 is the mirror image of
  // point 1, so the stencils at i = 1, 2 read psi_0 as psi_1)
  const obs_r<T>* gx;
  int x0;
  double* density;          // optional |phi|^2 output
  double* partials;
  unsigned int* counter;
  double* out;              // [7] sums
};

// |d phi / d axis|^2 at point q (index i of n along the axis, stride s);
// f1 = 1/(2h), f4 = 1/(12h)
template <typename T, typename R>
__device__ __forceinline__ R grad2_axis(const c2_t<T>* psi, long q, int i, int n, long s, R f1, R f4, long lim) {
  if (i == 0 || i == n - 1) return R(0);
  R dx, dy;
  if (i == 1 || i == n - 2) {
    if (!GPE_CHECK(q - s >= 0 && q + s < lim, 271)) return R(0);
    const c2_t<T> a = psi[q - s], b = psi[q + s];
    dx = (R(b.x) - R(a.x)) * f1;
    dy = (R(b.y) - R(a.y)) * f1;
  } else {
    if (!GPE_CHECK(q - 2 * s >= 0 && q + 2 * s < lim, 272)) return R(0);
    const c2_t<T> a = psi[q - 2 * s], b = psi[q - s], c = psi[q + s], e = psi[q + 2 * s];
    dx = (R(a.x) - R(8) * R(b.x) + R(8) * R(c.x) - R(e.x)) * f4;
    dy = (R(a.y) - R(8) * R(b.y) + R(8) * R(c.y) - R(e.y)) * f4;
  }
  return dx * dx + dy * dy;
}

constexpr int kObsThreads = 256;
constexpr int kObsBlocks = 152 * 4;   // at most; 10-100 points per thread on large grids

// Per-thread sums of the seven terms over the thread's points.  Rows
// r = j + ny k of the grid are spread over nblk blocks (this block is blk);
// 2^tx_log2 threads of a row-group take consecutive x indices (coalesced),
// and each thread keeps its x-dependent table values across the rows it visits.
template <typename T>
__device__ __forceinline__ void obs_accumulate(const ObsArgs<T>& A, int tx_log2, int blk, int nblk,
                                               obs_r<T> (&acc)[7]) {
  using R = obs_r<T>;
  const int TX = 1 << tx_log2;
  const int tx = threadIdx.x & (TX - 1), ty = threadIdx.x >> tx_log2, rpb = blockDim.x >> tx_log2;
  const int nrows = A.ny * A.nz;
  const long sy = A.nx, sz = (long)A.nx * A.ny, lim = (long)A.nx * A.ny * A.nz;
  const R fx1 = R(1.0 / (2.0 * A.hx)), fx4 = R(1.0 / (12.0 * A.hx));
  const R fy1 = R(1.0 / (2.0 * A.hy)), fy4 = R(1.0 / (12.0 * A.hy));
  const R fz1 = R(1.0 / (2.0 * A.hz)), fz4 = R(1.0 / (12.0 * A.hz));
  for (int i = tx; i < A.nx; i += TX) {
    const R vxi = A.vx[i], cxi = A.cx[i], wxi = A.wx[i];
    for (int r = blk * rpb + ty; r < nrows; r += nblk * rpb) {
      const int j = r % A.ny, k = r / A.ny;
      const long q = (long)r * A.nx + i;
      if (!GPE_CHECK(q < lim && (A.nx < 3 || q + 2 < lim || i + 2 >= A.nx), 273)) continue;
      const c2_t<T> p = A.psi[q];
      const R px = R(p.x), py = R(p.y);
      const R dens = px * px + py * py;
      R g2;
      if (A.x0 == 1 && i == 0) {
        const c2_t<T> p1 = A.psi[q + 1];
        const R ux = R(p1.x) * (R(2) * fx1), uy = R(p1.y) * (R(2) * fx1);
        g2 = ux * ux + uy * uy;
      } else if (A.x0 == 2 && (i == 1 || (i == 2 && A.nx >= 5))) {
        const c2_t<T> m = A.psi[q - i + 1], b = A.psi[q + 1];  // psi_0 read as psi_1
        R ux, uy;
        if (i == 1) {
          ux = (R(b.x) - R(m.x)) * fx1;
          uy = (R(b.y) - R(m.y)) * fx1;
        } else {
          const c2_t<T> e = A.psi[q + 2];
          ux = (R(m.x) - R(8) * R(m.x) + R(8) * R(b.x) - R(e.x)) * fx4;
          uy = (R(m.y) - R(8) * R(m.y) + R(8) * R(b.y) - R(e.y)) * fx4;
        }
        g2 = ux * ux + uy * uy;
      } else {
        g2 = grad2_axis<T, R>(A.psi, q, i, A.nx, 1, fx1, fx4, lim);
      }
      if (A.dim > 1) g2 += grad2_axis<T, R>(A.psi, q, j, A.ny, sy, fy1, fy4, lim);
      if (A.dim > 2) g2 += grad2_axis<T, R>(A.psi, q, k, A.nz, sz, fz1, fz4, lim);
      const R Vq = A.V ? R(A.V[q]) : (vxi + A.vy[j] + A.vz[k]);
      const R w = wxi * A.wy[j] * A.wz[k];
      const R wd = w * dens;
      acc[0] += wd;
      acc[1] += R(0.5) * w * g2;
      acc[2] += wd * Vq;
      acc[3] += A.gx ? wd * dens * A.gx[i] : wd * dens;
      acc[4] += wd * cxi * cxi;
      const R cy = A.cy[j], cz = A.cz[k];
      acc[5] += wd * cy * cy;
      acc[6] += wd * cz * cz;
      if (A.density) A.density[q] = (double)dens;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kObsThreads) observables_kernel(ObsArgs<T> A, int tx_log2) {
  using R = obs_r<T>;
  __shared__ double smem[32 * 7];
  R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  pdl_wait();  // the state is the previous kernel's output
  pdl_release();
  obs_accumulate<T>(A, tx_log2, blockIdx.x, gridDim.x, acc);
  double v[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) v[q] = (double)acc[q];  // FP64 from here on
  block_sum<7>(v, smem);
  double tot[7];
  if (grid_sum_last<7>(v, A.partials, A.counter, tot, smem) && threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 7; ++q) A.out[q] = tot[q] * A.wscale;
  }
}

// Threads per row of the reduction: 32..256, enough for a row of nx points.
inline int obs_tx_log2(int nx) {
  int lg = 5;
  while ((1 << lg) < nx && lg < 8) ++lg;
  return lg;
}

// Many independent grids in one launch: block b takes item items[b] =
// (grid, block index within the grid, blocks of that grid) and stores its
// FP64 sums in parts[8 b + q]; obs_finish_kernel then sums each grid's blocks
// in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kObsThreads) batch_obs_kernel(const ObsArgs<T>* __restrict__ runs,
                                                               const int4* __restrict__ items,
                                                               double* __restrict__ parts) {
  using R = obs_r<T>;
  __shared__ double smem[32 * 7];
  const int4 it = items[blockIdx.x];  // (run, block, nblocks, tx_log2)
  const ObsArgs<T> A = runs[it.x];
  R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  obs_accumulate<T>(A, it.w, it.y, it.z, acc);
  double v[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) v[q] = (double)acc[q];
  block_sum<7>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 7; ++q) parts[8L * blockIdx.x + q] = v[q];
  }
}

// One block per grid: the sums of items first[g] .. first[g+1]-1, times the
// grid's weight factor, into out[8 g + q].
static __global__ void __launch_bounds__(kObsThreads) obs_finish_kernel(const double* __restrict__ parts,
                                                                const int* __restrict__ first,
                                                                const double* __restrict__ wscale,
                                                                double* __restrict__ out) {
  __shared__ double smem[32 * 7];
  const int g = blockIdx.x;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = first[g] + threadIdx.x; b < first[g + 1]; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] += parts[8L * b + q];
  block_sum<7>(v, smem);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < 7; ++q) out[8L * g + q] = v[q] * wscale[g];
}

// The one launch configuration of the reduction (every caller uses it, so
// that equal states give bitwise equal sums).
template <typename T>
inline void launch_observables(const ObsArgs<T>& a, cudaStream_t s, bool pdl = false) {
  const int lg = obs_tx_log2(a.nx);  // 32..256 threads per row
  const int rpb = kObsThreads >> lg;
  const long nrows = (long)a.ny * a.nz;
  const long want = (nrows + rpb - 1) / rpb;
  const int blocks = (int)(want < kObsBlocks ? want : kObsBlocks);
  launch_k(pdl, observables_kernel<T>, dim3(blocks), dim3(kObsThreads), 0, s, a, lg);
}

}  // namespace gpe
