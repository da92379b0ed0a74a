// gpe_sweep.cuh -- Crank-Nicolson line sweeps of the split-step GP propagator.
//
// One step of the method ("Solution method": split-step Crank-Nicolson) is the
// nonlinear/potential sub-step N followed by one tridiagonal CN solve along
// each Cartesian axis.  Every CN solve here is a Thomas elimination with
// time-invariant coefficients precomputed on the host (m_k = 1/(b - a c'_{k-1}),
// c'_k = a m_k), run by one thread per line:
//
//   forward  d_k = (rhs_k - a d_{k-1}) m_k,      k = 1..n-2
//   back     u_k = d_k - c'_k u_{k+1},           u_{n-2} = d_{n-2}
//
// with a = -r, b = 1 + 2r, rhs_k = p_k + r (p_{k-1} - 2 p_k + p_{k+1}) and the
// end points held at zero.  In real time r = i beta (beta = dt/(4 dx^2)), in
// imaginary time r = beta, so the imaginary-time coefficients are real.
//
// The intermediate d_k is written in place over the line and read back by the
// back substitution, so each point is read and written twice by the same
// thread; the line's own second pass hits L1/L2.
//
// FIRST: the sweep along x also applies, as it loads each point, the pending
// imaginary-time renormalisation factor and the sub-step N,
//     p <- s p,   p <- exp(-i dt (V + g|p|^2)) p   or   exp(-dt (V + g|p|^2)) p.
// LAST (imaginary time): the sweep along the last axis accumulates the
// Simpson-weighted norm of its output in FP64, one sum per block, from which
// the next step's first sweep forms the factor 1/sqrt(norm).
#pragma once
#include <type_traits>
#include "gpe_common.cuh"

namespace gpe {

template <typename T>
struct SweepArgs {
  c2_t<T>* psi;
  LineGeom geom;
  const c2_t<T>* m;    // [n] elimination factors (complex; real part only in imaginary time)
  const c2_t<T>* cp;   // [n] c'_k
  T beta;              // dt/(4 dx^2), signed
  // sub-step N (FIRST only)
  const T* V;          // full potential [npoints] or nullptr for the separable trap
  const T* vx;         // [nx] nu^2 x^2/2
  const T* vy;         // [ny]
  const T* vz;         // [nz]
  T dt, g;
  const T* gw;             // nonlinear weight per point along the line (radial problem), or nullptr
  // pending renormalisation (imag FIRST): previous step's per-block norm sums
  const double* parts_in;
  int nparts_in;
  double parts_wscale;
  // norm (LAST, imaginary time): one FP64 sum per block into parts_out
  const double* w_axis;    // [n] Simpson weights along the line
  const double* w_a;       // weights of transverse index a
  const double* w_b;       // weights of transverse index b
  double* parts_out;
};

template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> apply_N(c2_t<T> p, T V, T dt, T g) {
  T dens = p.x * p.x + p.y * p.y;
  T th = dt * (V + g * dens);
  if (IMAG) {
    T f = exp(-th);
    return mk<T>(f * p.x, f * p.y);
  } else {
    return rot_neg<T>(p, th);
  }
}

template <typename T, bool IMAG, bool FIRST, bool LAST>
__global__ void __launch_bounds__(128) cn_sweep_kernel(SweepArgs<T> A) {
  using c2 = c2_t<T>;
  __shared__ double red_smem[32];
  const LineGeom& G = A.geom;
  const long L = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = L < G.nlines;
  const double pend = FIRST ? pending_scale(A.parts_in, A.nparts_in, A.parts_wscale, red_smem) : 1.0;
  double nacc = 0.0;
  if (active) {
    const long base = line_base(G, L);
    const long s = G.stride;
    const int n = G.n;
    const int M = n - 2;
    c2* line = A.psi + base;
    const T beta = A.beta;
    int ta = 0, tb = 0;
    line_transverse(G, L, ta, tb);
    // sub-step N parameters for this line (axis 0: transverse = (j, k))
    T vline = T(0), sc = T(1);
    if (FIRST) {
      if (A.V == nullptr) vline = A.vy[ta] + A.vz[tb];
      sc = (T)pend;
    }
    auto load = [&](int k) -> c2 {
      c2 p = line[(long)k * s];
      if (FIRST) {
        p.x *= sc; p.y *= sc;
        T V = A.V ? A.V[base + (long)k * s] : (A.vx[k] + vline);
        p = apply_N<T, IMAG>(p, V, A.dt, A.gw ? A.g * A.gw[k] : A.g);
      }
      return p;
    };
    // ---- forward elimination
    c2 pm = mk<T>(0, 0);
    c2 pc = load(1);
    c2 pn = (M >= 2) ? load(2) : mk<T>(0, 0);
    c2 d = mk<T>(0, 0);
    for (int k = 1; k <= M; ++k) {
      const c2 mk_ = A.m[k];
      c2 lap = mk<T>(pm.x + pn.x - T(2) * pc.x, pm.y + pn.y - T(2) * pc.y);
      c2 t;
      if (IMAG) {
        // rhs = p + beta lap ; t = rhs + beta d_prev ; d = t m (m real)
        t = mk<T>(pc.x + beta * (lap.x + d.x), pc.y + beta * (lap.y + d.y));
        d = mk<T>(t.x * mk_.x, t.y * mk_.x);
      } else {
        // rhs = p + i beta lap ; t = rhs + i beta d_prev ; d = t m
        t = mk<T>(pc.x - beta * (lap.y + d.y), pc.y + beta * (lap.x + d.x));
        d = cmul<T>(t, mk_);
      }
      line[(long)k * s] = d;
      pm = pc;
      pc = pn;
      pn = (k + 2 <= M) ? load(k + 2) : mk<T>(0, 0);
    }
    // ---- back substitution
    double wl = 0.0;
    if (LAST) wl = A.w_a[ta] * A.w_b[tb];
    c2 u = d;  // u_M = d_M
    if (LAST) nacc += A.w_axis[M] * ((double)u.x * u.x + (double)u.y * u.y);
    line[(long)M * s] = u;
    for (int k = M - 1; k >= 1; --k) {
      const c2 dk = line[(long)k * s];
      const c2 c = A.cp[k];
      if (IMAG) u = mk<T>(dk.x - c.x * u.x, dk.y - c.x * u.y);
      else u = mk<T>(dk.x - (c.x * u.x - c.y * u.y), dk.y - (c.x * u.y + c.y * u.x));
      line[(long)k * s] = u;
      if (LAST) nacc += A.w_axis[k] * ((double)u.x * u.x + (double)u.y * u.y);
    }
    line[0] = mk<T>(0, 0);
    line[(long)(n - 1) * s] = mk<T>(0, 0);
    if (LAST) nacc *= wl;
  }
  if (LAST) {
    double v[1] = {nacc};
    block_sum<1>(v, red_smem);
    if (threadIdx.x == 0) A.parts_out[blockIdx.x] = v[0];
  }
}

// psi *= the renormalisation left pending after the last imaginary-time step
template <typename T>
__global__ void scale_kernel(c2_t<T>* psi, long np, const double* parts, int nparts, double wscale) {
  __shared__ double smem[32];
  pdl_wait();
  pdl_release();
  const T s = (T)pending_scale(parts, nparts, wscale, smem);
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < np; q += (long)gridDim.x * blockDim.x) {
    c2_t<T> p = psi[q];
    p.x *= s; p.y *= s;
    psi[q] = p;
  }
}

// exp(-i dt V) and exp(-dt V) per point, evaluated in FP64 and stored in T
template <typename T>
__global__ void potential_factor_kernel(c2_t<T>* fr, c2_t<T>* fi, const double* V, double dt, long n) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    double s, c;
    sincos(dt * V[q], &s, &c);
    fr[q] = mk<T>((T)c, (T)(-s));
    fi[q] = mk<T>((T)exp(-dt * V[q]), T(0));
  }
}

static __global__ void to_float_kernel(float* dst, const double* src, long n) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    dst[q] = (float)src[q];
}

}  // namespace gpe
