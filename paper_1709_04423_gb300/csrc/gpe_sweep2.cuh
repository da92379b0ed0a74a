// gpe_sweep2.cuh -- segmented Crank-Nicolson line sweeps (the hot path).
//
// Each sweep L_d solves, on every line along axis d, the Crank-Nicolson system
// of the split-step method ("Solution method" of the paper)
//     (1 + A) u = (1 - A) p,      A = r T,  T = tridiag(-1, 2, -1),
// r = i dt/(4 dx^2) (real time) or dt/(4 dx^2) (imaginary time), ends held at
// zero.  It is computed in increment form,
//     u = p - z,   (1 + A) z = 2 A p = -2 r lap(p),
// so that the coefficients, which sit close to 1, only ever multiply the small
// increment: FP32 rounding of the coefficients then perturbs the kinetic term
// by O(eps) relative instead of O(eps/dt).  The Thomas elimination of
// (1 + A) with a = -r, b = 1 + 2r, m_k = 1/(b - a c'_{k-1}), c'_k = a m_k
// collapses, with alpha_k = r m_k (so that c'_k = -alpha_k), to two
// first-order recurrences
//     forward   e_k = alpha_k (e_{k-1} - 2 lap_k),        e_0 = 0
//     backward  z_k = e_k + alpha_k z_{k+1},              z_{M+1} = 0
// over the interior points k = 1..M = n-2.
//
// Both recurrences are linear with time-invariant coefficients, so a line is
// split into segments of SEG points, each run by its own thread with a zero
// carry-in; the true carries follow from the segment products
//     Gf_k = prod_{i=start..k} alpha_i,   Gb_k = prod_{i=k..end} alpha_i,
// (precomputed on the host) by a scan over segments:
//     e_k = e^_k + Gf_k E_{s-1},  E_s = e^_end + Gf_end E_{s-1},
//     z_k = z^_k + Gb_k Z_{s+1},  Z_s = z^_start + Gb_start Z_{s+1}.
// The result is the exact elimination, reassociated.  Everything a thread
// needs stays in registers: one read and one write of the state per point.
//
// Two mappings:
//  * x lines (contiguous): one warp per line, lane = segment; carries move by
//    warp shuffles (Kogge-Stone affine scan).  FIRST fuses the sub-step N
//    (and the pending imaginary-time renormalisation) into the load.
//  * y/z lines (strided): lane = line, warp = segment, so every load and store
//    of a warp is a contiguous row of 32 neighbouring lines; carries pass
//    through shared memory.
// LAST (imaginary time) accumulates the Simpson-weighted norm of the output:
// each thread sums its own SEG points in the state precision, and everything
// from there on (the line weight, warp, block and grid sums) is FP64; the
// last block stores the next step's factor 1/sqrt(norm).
#pragma once
#include "gpe_common.cuh"

namespace gpe {

template <typename T>
struct Sweep2Args {
  c2_t<T>* psi;
  LineGeom geom;
  const c2_t<T>* alpha;  // [n] alpha_k = r m_k (imaginary time: real part only)
  const c2_t<T>* gf;     // [n] forward segment products for this SEG
  const c2_t<T>* gb;     // [n] backward segment products for this SEG
  // sub-step N (FIRST)
  const T* V;            // full potential or nullptr (separable harmonic trap)
  const T* vx; const T* vy; const T* vz;
  T dt, g;
  const double* scale_in;
  // norm (LAST)
  const T* w_axis;     // Simpson weights along the line, state precision
  const double* w_a; const double* w_b;
  double* partials;
  unsigned int* counter;
  double* scale_out;
};

template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> phase_N(c2_t<T> p, T V, T dt, T g) {
  const T dens = p.x * p.x + p.y * p.y;
  const T th = dt * (V + g * dens);
  if (IMAG) {
    const T f = exp(-th);
    return mk<T>(f * p.x, f * p.y);
  } else {
    T s, c;
    sincos(th, &s, &c);
    return mk<T>(c * p.x + s * p.y, c * p.y - s * p.x);  // exp(-i th) p
  }
}

// a * b for the coefficient type: complex in real time, real in imaginary time
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> cf_mul(c2_t<T> a, c2_t<T> b) {
  if (IMAG) return mk<T>(a.x * b.x, a.x * b.y);
  return cmul<T>(a, b);
}
// c + a * b
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> cf_fma(c2_t<T> a, c2_t<T> b, c2_t<T> c) {
  if (IMAG) return mk<T>(fma(a.x, b.x, c.x), fma(a.x, b.y, c.y));
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// coefficient product a * b (both coefficients)
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> cf_cc(c2_t<T> a, c2_t<T> b) {
  if (IMAG) return mk<T>(a.x * b.x, T(0));
  return cmul<T>(a, b);
}

template <typename T>
__device__ __forceinline__ c2_t<T> shfl_up2(c2_t<T> v, int o) {
  return mk<T>(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o));
}
template <typename T>
__device__ __forceinline__ c2_t<T> shfl_down2(c2_t<T> v, int o) {
  return mk<T>(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}

// Segment-local forward/backward passes over SEG registers.  k0 = first
// interior index of the segment; points with k > M are padding (zero).
template <typename T, bool IMAG, int SEG>
__device__ __forceinline__ void local_forward(c2_t<T> (&p)[SEG], c2_t<T> (&e)[SEG], c2_t<T> pl, c2_t<T> pr,
                                              const c2_t<T>* __restrict__ alpha, int k0, int M) {
  c2_t<T> prev = mk<T>(0, 0);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    const c2_t<T> left = j == 0 ? pl : p[j - 1];
    const c2_t<T> right = j == SEG - 1 ? pr : p[j + 1];
    // t = e_{k-1} - 2 lap_k,  lap_k = left - 2 p_k + right
    const c2_t<T> t = mk<T>(prev.x - T(2) * (left.x + right.x) + T(4) * p[j].x,
                            prev.y - T(2) * (left.y + right.y) + T(4) * p[j].y);
    c2_t<T> v = mk<T>(0, 0);
    if (k <= M) v = cf_mul<T, IMAG>(__ldg(&alpha[k]), t);
    e[j] = v;
    prev = v;
  }
}

template <typename T, bool IMAG, int SEG>
__device__ __forceinline__ void local_backward(c2_t<T> (&e)[SEG], const c2_t<T>* __restrict__ alpha, int k0, int M) {
  c2_t<T> next = mk<T>(0, 0);
#pragma unroll
  for (int j = SEG - 1; j >= 0; --j) {
    const int k = k0 + j;
    if (k <= M) next = cf_fma<T, IMAG>(__ldg(&alpha[k]), next, e[j]);
    else next = mk<T>(0, 0);
    e[j] = next;
  }
}

// ---------------------------------------------------------------- x sweep
// One warp per line; lane j owns interior points k = 1 + j*SEG .. (j+1)*SEG.
template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG>
__global__ void __launch_bounds__(128) xsweep_kernel(Sweep2Args<T> A) {
  using c2 = c2_t<T>;
  __shared__ double red_smem[32];
  const LineGeom& G = A.geom;
  const int lane = threadIdx.x & 31;
  const long L = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const bool active = L < G.nlines;  // warp-uniform
  double nacc = 0.0;
  if (active) {
    const int M = G.n - 2;
    const long base = L * (long)G.nx;
    c2* line = A.psi + base;
    const int k0 = 1 + lane * SEG;
    int ta, tb;
    line_transverse(G, L, ta, tb);
    T vline = T(0), sc = T(1);
    if (FIRST) {
      if (A.V == nullptr) vline = A.vy[ta] + A.vz[tb];
      if (A.scale_in) sc = (T)(*A.scale_in);
    }
    c2 p[SEG], e[SEG];
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      c2 v = mk<T>(0, 0);
      if (k <= M) {
        v = line[k];
        if (FIRST) {
          v.x *= sc; v.y *= sc;
          const T Vk = A.V ? A.V[base + k] : (A.vx[k] + vline);
          v = phase_N<T, IMAG>(v, Vk, A.dt, A.g);
        }
      }
      p[j] = v;
    }
    // halo from the neighbouring lanes (zero at the Dirichlet ends)
    c2 pl = shfl_up2<T>(p[SEG - 1], 1);
    c2 pr = shfl_down2<T>(p[0], 1);
    if (lane == 0) pl = mk<T>(0, 0);
    if (lane == 31) pr = mk<T>(0, 0);
    local_forward<T, IMAG, SEG>(p, e, pl, pr, A.alpha, k0, M);
    // forward carries: C_j = e^_end(j) + P_j C_{j-1}
    const int kend = k0 + SEG - 1;
    c2 Pm = (k0 <= M) ? __ldg(&A.gf[min(kend, M)]) : mk<T>(1, 0);
    c2 Bc = e[SEG - 1];
    if (k0 <= M && kend > M) {
      // ragged last segment: its end value sits at index M - k0
#pragma unroll
      for (int j = 0; j < SEG; ++j) if (k0 + j == M) Bc = e[j];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const c2 Pp = shfl_up2<T>(Pm, o), Bp = shfl_up2<T>(Bc, o);
      if (lane >= o) {
        Bc = cf_fma<T, IMAG>(Pm, Bp, Bc);
        Pm = cf_cc<T, IMAG>(Pm, Pp);
      }
    }
    c2 Ein = shfl_up2<T>(Bc, 1);
    if (lane == 0) Ein = mk<T>(0, 0);
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) e[j] = cf_fma<T, IMAG>(__ldg(&A.gf[k]), Ein, e[j]);
    }
    local_backward<T, IMAG, SEG>(e, A.alpha, k0, M);
    // backward carries: D_j = z^_start(j) + Q_j D_{j+1}
    c2 Qm = (k0 <= M) ? __ldg(&A.gb[k0]) : mk<T>(1, 0);
    c2 Dc = e[0];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const c2 Qp = shfl_down2<T>(Qm, o), Dp = shfl_down2<T>(Dc, o);
      if (lane + o < 32) {
        Dc = cf_fma<T, IMAG>(Qm, Dp, Dc);
        Qm = cf_cc<T, IMAG>(Qm, Qp);
      }
    }
    c2 Zin = shfl_down2<T>(Dc, 1);
    if (lane == 31) Zin = mk<T>(0, 0);
    T tacc = T(0);  // this thread's few points, in the state precision
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) {
        const c2 z = cf_fma<T, IMAG>(__ldg(&A.gb[k]), Zin, e[j]);
        const c2 u = mk<T>(p[j].x - z.x, p[j].y - z.y);
        line[k] = u;
        if (LAST) tacc += A.w_axis[k] * (u.x * u.x + u.y * u.y);
      }
    }
    if (lane == 0) line[0] = mk<T>(0, 0);
    if (lane == 31) line[G.n - 1] = mk<T>(0, 0);
    if (LAST) nacc = (double)tacc * (A.w_a[ta] * A.w_b[tb]);  // FP64 from here on
  }
  if (LAST) {
    double v[1] = {nacc}, tot[1];
    block_sum<1>(v, red_smem);
    if (grid_sum_last<1>(v, A.partials, A.counter, tot, red_smem) && threadIdx.x == 0)
      *A.scale_out = 1.0 / sqrt(tot[0]);
  }
}

// ---------------------------------------------------------------- y/z sweep
// Lane = line (32 consecutive lines per block), warp s = segment of SEG points;
// blockDim.x = 32 * nseg with nseg <= 16.  KEEP holds the input segment in
// registers for the final u = p - z; otherwise the forward pass streams the
// loads and the final pass reads p again (from L2), halving register use.
template <typename T, bool IMAG, bool LAST, int SEG, bool KEEP>
__global__ void __launch_bounds__(512) colsweep_kernel(Sweep2Args<T> A) {
  using c2 = c2_t<T>;
  __shared__ c2 carry[16][33];
  __shared__ double red_smem[32];
  const LineGeom& G = A.geom;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5, nseg = blockDim.x >> 5;
  const long L = (long)blockIdx.x * 32 + lane;
  const bool active = L < G.nlines;
  const int M = G.n - 2;
  const long st = G.stride;
  const int k0 = 1 + s * SEG;
  const long base = active ? line_base(G, L) : 0;
  c2* line = A.psi + base;
  auto ld = [&](int k) -> c2 { return (active && k >= 1 && k <= M) ? line[(long)k * st] : mk<T>(0, 0); };
  c2 e[SEG];
  c2 p[KEEP ? SEG : 1];
  if constexpr (KEEP) {
#pragma unroll
    for (int j = 0; j < SEG; ++j) p[j] = ld(k0 + j);
    local_forward<T, IMAG, SEG>(p, e, ld(k0 - 1), ld(k0 + SEG), A.alpha, k0, M);
  } else {
    c2 pm = ld(k0 - 1), pc = ld(k0), prev = mk<T>(0, 0);
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      const c2 pn = ld(k + 1);
      const c2 t = mk<T>(prev.x - T(2) * (pm.x + pn.x) + T(4) * pc.x,
                         prev.y - T(2) * (pm.y + pn.y) + T(4) * pc.y);
      c2 v = mk<T>(0, 0);
      if (k <= M) v = cf_mul<T, IMAG>(__ldg(&A.alpha[k]), t);
      e[j] = v;
      prev = v;
      pm = pc;
      pc = pn;
    }
  }
  // segment end value -> shared; one warp runs the carry recurrence
  {
    c2 Bc = e[SEG - 1];
#pragma unroll
    for (int j = 0; j < SEG; ++j) if (k0 + j == M) Bc = e[j];
    carry[s][lane] = Bc;
  }
  __syncthreads();
  if (s == 0) {
    c2 C = mk<T>(0, 0);
    for (int q = 0; q < nseg; ++q) {
      const int kq0 = 1 + q * SEG;
      if (kq0 > M) break;
      const c2 Pq = __ldg(&A.gf[min(kq0 + SEG - 1, M)]);
      C = cf_fma<T, IMAG>(Pq, C, carry[q][lane]);
      carry[q][lane] = C;  // E_q
    }
  }
  __syncthreads();
  const c2 Ein = (s > 0) ? carry[s - 1][lane] : mk<T>(0, 0);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    if (k <= M) e[j] = cf_fma<T, IMAG>(__ldg(&A.gf[k]), Ein, e[j]);
  }
  local_backward<T, IMAG, SEG>(e, A.alpha, k0, M);
  __syncthreads();  // every warp has read its E before the slots are reused
  carry[s][lane] = e[0];
  __syncthreads();
  if (s == 0) {
    c2 D = mk<T>(0, 0);
    for (int q = nseg - 1; q >= 0; --q) {
      const int kq0 = 1 + q * SEG;
      if (kq0 > M) continue;
      const c2 Qq = __ldg(&A.gb[kq0]);
      D = cf_fma<T, IMAG>(Qq, D, carry[q][lane]);
      carry[q][lane] = D;  // Z_q
    }
  }
  __syncthreads();
  const c2 Zin = (s + 1 < nseg && k0 + SEG <= M) ? carry[s + 1][lane] : mk<T>(0, 0);
  double nacc = 0.0;
  if (active) {
    int ta = 0, tb = 0;
    if (LAST) line_transverse(G, L, ta, tb);
    T tacc = T(0);  // this thread's few points, in the state precision
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) {
        const c2 z = cf_fma<T, IMAG>(__ldg(&A.gb[k]), Zin, e[j]);
        c2 pk;
        if constexpr (KEEP) pk = p[j];
        else pk = __ldcg(&line[(long)k * st]);
        const c2 u = mk<T>(pk.x - z.x, pk.y - z.y);
        line[(long)k * st] = u;
        if (LAST) tacc += A.w_axis[k] * (u.x * u.x + u.y * u.y);
      }
    }
    if (s == 0) {
      line[0] = mk<T>(0, 0);
      line[(long)(G.n - 1) * st] = mk<T>(0, 0);
    }
    if (LAST) nacc = (double)tacc * (A.w_a[ta] * A.w_b[tb]);  // FP64 from here on
  }
  if (LAST) {
    double v[1] = {nacc}, tot[1];
    block_sum<1>(v, red_smem);
    if (grid_sum_last<1>(v, A.partials, A.counter, tot, red_smem) && threadIdx.x == 0)
      *A.scale_out = 1.0 / sqrt(tot[0]);
  }
}

}  // namespace gpe
