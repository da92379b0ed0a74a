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
// all in FP64, whatever the state's precision; the host turns them into
// E = (S1+S2)/S0 + g/2 S3/S0^2, mu = (S1+S2)/S0 + g S3/S0^2, rms_d = sqrt(S_{4+d}/S0).
// Derivatives: 4th-order central differences for 2 <= i <= n-3, 2nd-order at
// i = 1, n-2, zero at the end points.  Optionally writes |phi|^2 (FP64).
#pragma once
#include "gpe_common.cuh"

namespace gpe {

template <typename T>
struct ObsArgs {
  const c2_t<T>* psi;
  int dim, nx, ny, nz;
  double hx, hy, hz;        // grid spacings
  const double* V;          // full potential or nullptr
  const double* vx; const double* vy; const double* vz;  // separable trap terms
  const double* cx; const double* cy; const double* cz;  // coordinates
  const double* wx; const double* wy; const double* wz;  // Simpson weights
  double* density;          // optional |phi|^2 output
  double* partials;
  unsigned int* counter;
  double* out;              // [7] sums
};

template <typename T>
__device__ __forceinline__ double2 ld2(const c2_t<T>* p, long q) {
  c2_t<T> v = p[q];
  return make_double2((double)v.x, (double)v.y);
}

template <typename T>
__device__ __forceinline__ double grad2_axis(const c2_t<T>* psi, long q, int i, int n, long s, double h) {
  if (i == 0 || i == n - 1) return 0.0;
  double2 d;
  if (i == 1 || i == n - 2) {
    double2 a = ld2<T>(psi, q - s), b = ld2<T>(psi, q + s);
    const double f = 1.0 / (2.0 * h);
    d = make_double2((b.x - a.x) * f, (b.y - a.y) * f);
  } else {
    double2 a = ld2<T>(psi, q - 2 * s), b = ld2<T>(psi, q - s), c = ld2<T>(psi, q + s), e = ld2<T>(psi, q + 2 * s);
    const double f = 1.0 / (12.0 * h);
    d = make_double2((a.x - 8.0 * b.x + 8.0 * c.x - e.x) * f, (a.y - 8.0 * b.y + 8.0 * c.y - e.y) * f);
  }
  return d.x * d.x + d.y * d.y;
}

template <typename T>
__global__ void __launch_bounds__(256) observables_kernel(ObsArgs<T> A) {
  __shared__ double smem[32 * 7];
  const long np = (long)A.nx * A.ny * A.nz;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (long)gridDim.x * blockDim.x) {
    const int i = (int)(q % A.nx);
    const long r = q / A.nx;
    const int j = (int)(r % A.ny);
    const int k = (int)(r / A.ny);
    const double2 p = ld2<T>(A.psi, q);
    const double dens = p.x * p.x + p.y * p.y;
    double g2 = grad2_axis<T>(A.psi, q, i, A.nx, 1, A.hx);
    if (A.dim > 1) g2 += grad2_axis<T>(A.psi, q, j, A.ny, A.nx, A.hy);
    if (A.dim > 2) g2 += grad2_axis<T>(A.psi, q, k, A.nz, (long)A.nx * A.ny, A.hz);
    const double Vq = A.V ? A.V[q] : (A.vx[i] + A.vy[j] + A.vz[k]);
    const double w = A.wx[i] * A.wy[j] * A.wz[k];
    const double wd = w * dens;
    v[0] += wd;
    v[1] += 0.5 * w * g2;
    v[2] += wd * Vq;
    v[3] += wd * dens;
    v[4] += wd * A.cx[i] * A.cx[i];
    v[5] += wd * A.cy[j] * A.cy[j];
    v[6] += wd * A.cz[k] * A.cz[k];
    if (A.density) A.density[q] = dens;
  }
  block_sum<7>(v, smem);
  double tot[7];
  if (grid_sum_last<7>(v, A.partials, A.counter, tot, smem) && threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 7; ++q) A.out[q] = tot[q];
  }
}

}  // namespace gpe
