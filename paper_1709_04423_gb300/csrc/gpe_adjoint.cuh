// gpe_adjoint.cuh -- adjoint of the real-time split-step Crank-Nicolson step
// (the differentiation form of the propagator).
//
// Conventions: real inner product <a, b> = Re sum conj(a) b over grid points;
// the adjoint state is lambda = dJ/dRe(phi) + i dJ/dIm(phi) (the gradient
// convention of torch.autograd for complex tensors).  One forward step is
// N, L_x, L_y, L_z with
//   N:   u = exp(-i th) p,  th = dt (V + g |p|^2)
//   L_d: u = C p,  C = (1 + iA)^-1 (1 - iA) with A real symmetric,
// so the reverse step applies L_z^H, L_y^H, L_x^H -- each the same
// Crank-Nicolson sweep with dt -> -dt, since C^H = conj(C) = C(-dt) -- and
// then the adjoint of N at the step's input p: with s = Im(conj(lam) u),
//   lam <- exp(+i th) lam + 2 g dt s p,
//   dJ/dV(point) += dt s,   dJ/dg += dt sum s |p|^2.
#pragma once
#include "gpe_common.cuh"

namespace gpe {

template <typename T>
struct AdjPhaseArgs {
  const c2_t<T>* phi;  // step input p
  c2_t<T>* lam;        // adjoint, updated in place
  long np;
  int nx, ny;
  const T* V;          // full potential or nullptr (separable harmonic trap)
  const T* vx; const T* vy; const T* vz;
  T dt, g;
  double* dJdV;        // [np] FP64 accumulator
  double* partials;
  unsigned int* counter;
  double* dJdg;        // FP64 accumulator (device scalar); the last block adds this step's sum
};

template <typename T>
__global__ void __launch_bounds__(256) adjoint_phase_kernel(AdjPhaseArgs<T> A) {
  __shared__ double red_smem[32];
  T gacc = T(0);
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < A.np; q += (long)gridDim.x * blockDim.x) {
    const c2_t<T> p = A.phi[q];
    c2_t<T> l = A.lam[q];
    T Vq;
    if (A.V) {
      Vq = A.V[q];
    } else {
      const int i = (int)(q % A.nx);
      const long r = q / A.nx;
      Vq = A.vx[i] + A.vy[(int)(r % A.ny)] + A.vz[(int)(r / A.ny)];
    }
    const T dens = p.x * p.x + p.y * p.y;
    const T th = A.dt * (Vq + A.g * dens);
    // rotations with the forward's coefficients (rot_coefs): cos th = 1 + cm1
    T sn, cm1;
    rot_coefs<T>(th, sn, cm1);
    const c2_t<T> u = rot_neg<T>(p, th);                                // exp(-i th) p
    const T s = l.x * u.y - l.y * u.x;                                  // Im(conj(lam) u)
    const T ds = A.dt * s;
    A.dJdV[q] += (double)ds;
    gacc += ds * dens;
    const T c2g = T(2) * A.g * ds;
    // exp(i th) lam + 2 g dt s p
    l = mk<T>((l.x + fma(cm1, l.x, -(sn * l.y))) + c2g * p.x, (l.y + fma(cm1, l.y, sn * l.x)) + c2g * p.y);
    A.lam[q] = l;
  }
  double v[1] = {(double)gacc}, tot[1];  // FP64 from the per-thread sums on
  block_sum<1>(v, red_smem);
  if (grid_sum_last<1>(v, A.partials, A.counter, tot, red_smem) && threadIdx.x == 0) *A.dJdg += tot[0];
}

}  // namespace gpe
