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
// over the interior points k = 1..M = n-2.  The kernels carry both at half
// scale, e~ = e/2 and z~ = z/2:
//     e~_k = alpha_k (e~_{k-1} + 2 p_k - p_{k-1} - p_{k+1}),   u_k = p_k - 2 z~_k,
// which saves a multiplication per point and component; scaling by 2
// commutes with rounding in binary floating point (away from overflow and
// subnormals), so every value is exactly half the full-scale one and u is
// bit for bit the same.
//
// Both recurrences are linear with time-invariant coefficients, so a line is
// split into segments of SEG points, each run by its own thread with a zero
// carry-in.  With the precomputed segment products
//     Gf_k = prod_{i=start..k} alpha_i,   Gb_k = prod_{i=k..end} alpha_i,
// and A_q = the product over all of segment q, the true values are
//     e_k = e^_k + Gf_k E_{s-1},   E_t = sum_{q<=t} (prod_{q<r<=t} A_r) e^_end(q),
//     z_k = z^_k + Gb_k Z_{s+1},   Z_t = sum_{q>=t} (prod_{t<=r<q} A_r) z^_start(q),
// where the products over segments are host-precomputed 16 x 16 tables, so
// every thread forms its own carry-in as a short dot product (no serial scan
// across segments).  The result is the exact elimination, reassociated.
//
// Three mappings:
//  * y/z lines (strided): lane = line (32 neighbouring lines per block, so
//    every warp load and store is one contiguous row), warp = segment; the
//    segment lives in registers.
//  * x lines in 2d/3d: a tile of 32 lines x n points is loaded row-wise with
//    coalesced accesses and transposed into shared memory (pitch 33), the
//    sub-step N and the pending renormalisation are applied on the way in
//    (FIRST), the segments are solved as above, and the tile is written back.
//  * x line in 1d: one warp per line, lane = segment, carries by shuffles.
// LAST (imaginary time) accumulates the Simpson-weighted norm of the output:
// each thread and then each block sums in the state precision, the per-block
// totals are summed over the grid in FP64 in a fixed order, and the last block
// stores the next step's factor 1/sqrt(norm).  (FP64 per point would cost more
// than the whole sweep on this part, whose FP64 rate is 1/70 of FP32; the
// factor only rescales the state, and the observables recompute the norm in
// FP64 from scratch.)
#pragma once
#include <type_traits>

#include "gpe_common.cuh"

namespace gpe {

template <typename T>
struct Sweep2Args {
  c2_t<T>* psi;          // lines are written here
  const c2_t<T>* src;    // and read from here (x sweeps; nullptr = psi)
  LineGeom geom;
  const c2_t<T>* alpha;  // [n] alpha_k = r m_k (imaginary time: real part only)
  const c2_t<T>* gf;     // [n] forward segment products for this SEG
  const c2_t<T>* gb;     // [n] backward segment products for this SEG
  const c2_t<T>* ptab;   // [2][16][16] carry tables Pf, Pb for this SEG
  // sub-step N (FIRST).  FP64 state: exp(-i dt V) (real time) or exp(-dt V)
  // (imaginary time, real part only) as a per-point factor array fV, or for
  // the separable harmonic trap as per-axis factors fx[i] fy[j] fz[k], and
  // dtg = dt g for the nonlinear part.  FP32 state: the potential V (array) or
  // vx[i] + vy[j] + vz[k], and dt, g: the phase angle is formed per point,
  // because FP32-rounded factors would be applied identically every step and
  // their |F| - 1 ~ 1e-7 would add up step after step.
  const c2_t<T>* fV;
  const c2_t<T>* fx; const c2_t<T>* fy; const c2_t<T>* fz;
  T dtg;
  const T* V;
  const T* vx; const T* vy; const T* vz;
  T dt, g;
  // weight of the nonlinear term per x index (the spherical trap's radial
  // problem: 1/(4 pi r^2)); nullptr = 1.  Used by the 1d sweep only.
  const T* gw;
  // double-float state: the same factors as exact triple-floats, per point
  // (tfV) or per x index (tfx) and per x line (tfyz = fy[j] fz[k], formed in FP64)
  const tf3c* tfV;
  const tf3c* tfx;
  const tf3c* tfyz;
  // pending renormalisation (FIRST, imaginary time): the previous step's
  // per-block norm sums, their number and factor (see pending_scale)
  const double* parts_in;
  int nparts_in;
  double parts_wscale;
  // norm of the output (LAST): Simpson coefficients (1, 2, 4: exact in any
  // precision) along the line and of the two transverse indices -- the grid
  // factor prod_d dx_d/3 is applied by the reader to the FP64 total, so no
  // rounded weight biases the norm -- and one sum per block into parts_out
  const T* w_axis;
  const T* w_a; const T* w_b;
  double* parts_out;
  // rho axis of a circular or axial trap (x sweeps with VAR): the matrix is
  // not symmetric -- row k of T is (-(1 - h_k), 2, -(1 + h_k)) -- so the
  // forward recurrence is e_k = alpha_k e_{k-1} + 2 r m_k lapv_k with alpha_k
  // = r (1 - h_k) m_k and lapv_k = 2 p_k - (1 - h_k) p_{k-1} - (1 + h_k)
  // p_{k+1} (vh_k = (1 - h_k, 1 + h_k)), carried at half scale like the
  // symmetric one (vbf_k = r m_k), and the backward one is z_k = e_k + vab_k
  // z_{k+1} with vab_k = r (1 + h_k) m_k; gf / gb and the carry tables are the
  // segment products of alpha / vab.
  const c2_t<T>* vab;
  const c2_t<T>* vbf;
  const c2_t<T>* vh;
  // how far the segment carries reach above the precision's threshold (the
  // host reads them off gf, gb and the carry tables): carries cross at most
  // cdepth segments and reach the first (last) cpts points of a segment, cpts
  // one of 4, 8, 12; 0 = every segment and point
  int cdepth, cpts;
};

// Sub-step N at one point: p <- F exp(-i a) p (real time) or F exp(-a) p
// (imaginary time), where F = exp(-i dt V) or exp(-dt V) is the precomputed
// potential factor and a = dt g |p|^2.  The exponential of the nonlinear part
// is its Taylor series: for |a| < 1/32 sin to a^7, cos to a^8, exp to a^7
// (first omitted terms below 2.3e-17 relative), for |a| < 1/8 sin to a^11,
// cos to a^12, exp to a^13 (below 1.2e-21) -- under FP64 rounding either
// way; larger |a| takes the library sincos/exp.  The multiply-adds are
// spelled out (Horner steps as fma, the products as cmul), so that the
// rounding does not depend on how the compiler contracts the expression in a
// given kernel: the batched and single-grid sweeps agree bit for bit.
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> phase_N(c2_t<T> p, c2_t<T> F, T dtg) {
  const T a = dtg * fma(p.x, p.x, p.y * p.y);
  if (IMAG) {
    T e;
    if (fabs(a) < T(0.03125)) {
      const T m = -a;
      T t = T(1.0 / 5040);
      t = fma(m, t, T(1.0 / 720));
      t = fma(m, t, T(1.0 / 120));
      t = fma(m, t, T(1.0 / 24));
      t = fma(m, t, T(1.0 / 6));
      t = fma(m, t, T(1.0 / 2));
      t = fma(m, t, T(1));
      e = fma(m, t, T(1));
    } else if (fabs(a) < T(0.125)) {
      const T m = -a;
      T t = T(1.0 / 6227020800.0);
      t = fma(m, t, T(1.0 / 479001600));
      t = fma(m, t, T(1.0 / 39916800));
      t = fma(m, t, T(1.0 / 3628800));
      t = fma(m, t, T(1.0 / 362880));
      t = fma(m, t, T(1.0 / 40320));
      t = fma(m, t, T(1.0 / 5040));
      t = fma(m, t, T(1.0 / 720));
      t = fma(m, t, T(1.0 / 120));
      t = fma(m, t, T(1.0 / 24));
      t = fma(m, t, T(1.0 / 6));
      t = fma(m, t, T(1.0 / 2));
      t = fma(m, t, T(1));
      e = fma(m, t, T(1));
    } else {
      e = exp(-a);
    }
    const T f = F.x * e;
    return mk<T>(f * p.x, f * p.y);
  } else {
    T sn, cs;
    if (fabs(a) < T(0.03125)) {
      const T a2 = a * a;
      T s = T(-1.0 / 5040);
      s = fma(a2, s, T(1.0 / 120));
      s = fma(a2, s, T(-1.0 / 6));
      sn = a * fma(a2, s, T(1));
      T c = T(1.0 / 40320);
      c = fma(a2, c, T(-1.0 / 720));
      c = fma(a2, c, T(1.0 / 24));
      c = fma(a2, c, T(-1.0 / 2));
      cs = fma(a2, c, T(1));
    } else if (fabs(a) < T(0.125)) {
      const T a2 = a * a;
      T s = T(-1.0 / 39916800);
      s = fma(a2, s, T(1.0 / 362880));
      s = fma(a2, s, T(-1.0 / 5040));
      s = fma(a2, s, T(1.0 / 120));
      s = fma(a2, s, T(-1.0 / 6));
      sn = a * fma(a2, s, T(1));
      T c = T(1.0 / 479001600);
      c = fma(a2, c, T(-1.0 / 3628800));
      c = fma(a2, c, T(1.0 / 40320));
      c = fma(a2, c, T(-1.0 / 720));
      c = fma(a2, c, T(1.0 / 24));
      c = fma(a2, c, T(-1.0 / 2));
      cs = fma(a2, c, T(1));
    } else {
      sincos(a, &sn, &cs);
    }
    // w = F exp(-i a) = (cs F.x + sn F.y) + i (cs F.y - sn F.x); return w p
    const c2_t<T> w = mk<T>(fma(cs, F.x, sn * F.y), fma(cs, F.y, -(sn * F.x)));
    return cmul<T>(w, p);
  }
}

// FP32 state: p <- exp(-i th) p or exp(-th) p with th = dt (V + g |p|^2)
// formed per point (library sincos / exp of the state precision).  Real time
// rotates with rot_neg, whose rounded rotation keeps |p| unbiased.
// (Imaginary time keeps the product form: applying the factor as
// p + (factor - 1) p with expm1 was measured to move the FP32 ground state's
// mu further from FP64 -- the FP32 iteration stops at an exact fixed point of
// the rounded map, whose mu depends on how each sub-step rounds, and that
// form stops 1.3e-6 away against 8e-9 for the product.)
// The FP32 factor is the library expf.  A correctly rounded factor (1 +
// expm1(-th), rounded once) was measured as well: on the 128^3 imaginary-time
// workload it moves the first 100 steps 180x closer to the FP64 oracle in mu
// (1.2e-8 against 2.1e-6) but leaves the FP32 iteration at a fixed point of the
// rounded map 1.9e-6 from FP64 at the 5000-step job end and 1.2e-6 converged,
// against 8.6e-7 and 3.8e-8 with expf -- both sit at the floor that rounding
// the state to FP32 sets (an FP32 emulation with exact factors wanders between
// 1e-8 and 8e-7 on a 64^3 version), and expf is the cheaper one and ends the
// job within 1e-6.
// th = dt (V + g |p|^2) as every FP32 phase forms it
template <typename T>
__device__ __forceinline__ T phase_angle(c2_t<T> p, T V, T dt, T g) {
  return dt * (V + g * (p.x * p.x + p.y * p.y));
}

template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> phase_direct(c2_t<T> p, T V, T dt, T g) {
  const T th = phase_angle<T>(p, V, dt, g);
  if (IMAG) {
    const T f = exp(-th);
    return mk<T>(f * p.x, f * p.y);
  }
  return rot_neg<T>(p, th);
}

// Double-float state: p <- exp(-i a) p (real time) or exp(-a) p (imaginary
// time), a = dt g |p|^2, then the potential factors (exact triple-floats).
// For |a| < 1/8 the exponential is its Taylor series; the terms of order a^6
// and up (at most 5.3e-9 here) only need float accuracy for a 2^-50 total
// and are summed in float, the leading ones in double-float.  Larger |a|
// goes through FP64.
template <bool IMAG>
__device__ __forceinline__ df64x2 phase_df(df64x2 p, const Sweep2Args<df64>& A, long gidx, int k, int L,
                                           df64 dtg) {
  const df64 a = dtg * (p.x * p.x + p.y * p.y);
  if (IMAG) {
    df64 e;
    if (fabsf(a.hi) < 0.125f) {
      const df64 m = -a;
      const float mf = m.hi;
      const float te = 1.0f / 720 + mf * (1.0f / 5040 + mf * (1.0f / 40320 + mf * (1.0f / 362880 + mf * (1.0f / 3628800))));
      constexpr df64 c5(1.0 / 120), c4(1.0 / 24), c3(1.0 / 6), c2(0.5), c1(1.0);
      e = df_mulf(m, te) + c5;
      e = m * e + c4;
      e = m * e + c3;
      e = m * e + c2;
      e = m * e + c1;
      e = m * e + c1;
    } else {
      e = df64(::exp(-(double)a));
    }
    p = df64x2{e * p.x, e * p.y};
    if (A.tfV) {
      const tf3c F = A.tfV[gidx];
      p = df64x2{tf_mul(F.re, p.x), tf_mul(F.re, p.y)};
    } else {
      const tf3c Fx = A.tfx[k], Fl = A.tfyz[L];
      p = df64x2{tf_mul(Fx.re, p.x), tf_mul(Fx.re, p.y)};
      p = df64x2{tf_mul(Fl.re, p.x), tf_mul(Fl.re, p.y)};
    }
    return p;
  } else {
    df64 sn, cs;
    if (fabsf(a.hi) < 0.125f) {
      const df64 a2 = a * a;
      const float q = a2.hi;
      const float ts = -1.0f / 5040 + q * (1.0f / 362880 + q * (-1.0f / 39916800));
      const float tc = -1.0f / 720 + q * (1.0f / 40320 + q * (-1.0f / 3628800 + q * (1.0f / 479001600)));
      constexpr df64 s2(1.0 / 120), s1(-1.0 / 6), c2(1.0 / 24), c1(-0.5), one(1.0);
      df64 S = df_mulf(a2, ts) + s2;
      S = a2 * S + s1;
      S = a2 * S + one;
      sn = a * S;
      df64 C = df_mulf(a2, tc) + c2;
      C = a2 * C + c1;
      cs = a2 * C + one;
    } else {
      double sd, cd;
      ::sincos((double)a, &sd, &cd);
      sn = df64(sd);
      cs = df64(cd);
    }
    // exp(-i a) p = (cs px + sn py) + i (cs py - sn px)
    p = df64x2{cs * p.x + sn * p.y, cs * p.y - sn * p.x};
    auto cmul_tf = [](const tf3c& F, df64x2 v) {
      // (Fr + i Fi)(vx + i vy) = (Fr vx - Fi vy) + i (Fr vy - Fi (-vx))
      return df64x2{tf_dot2(F.re, v.x, F.im, v.y), tf_dot2(F.re, v.y, F.im, -v.x)};
    };
    if (A.tfV) {
      p = cmul_tf(A.tfV[gidx], p);
    } else {
      p = cmul_tf(A.tfx[k], p);
      p = cmul_tf(A.tfyz[L], p);
    }
    return p;
  }
}

// product of two potential factors (real in imaginary time)
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> fac_mul(c2_t<T> a, c2_t<T> b) {
  if (IMAG) return mk<T>(a.x * b.x, T(0));
  return cmul<T>(a, b);
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
  return mk<T>(shfl_up_t(v.x, o), shfl_up_t(v.y, o));
}
template <typename T>
__device__ __forceinline__ c2_t<T> shfl_down2(c2_t<T> v, int o) {
  return mk<T>(shfl_down_t(v.x, o), shfl_down_t(v.y, o));
}

// 2 p - (l + r) = -lap, the part of the half-scale forward step that does not
// depend on the recurrence (exactly half of 4 p - 2 (l + r))
template <typename T>
__device__ __forceinline__ T neg_lap(T l, T r, T p) {
  if constexpr (is_df<T>::value) return df_scale(p, 2.f) - (l + r);
  else return fma(T(2), p, -(l + r));
}

// u = p - 2 z~ (one rounding, the same as p - z at full scale)
template <typename T>
__device__ __forceinline__ c2_t<T> sub2(c2_t<T> p, c2_t<T> zh) {
  if constexpr (is_df<T>::value) return mk<T>(p.x - df_scale(zh.x, 2.f), p.y - df_scale(zh.y, 2.f));
  else return mk<T>(fma(T(-2), zh.x, p.x), fma(T(-2), zh.y, p.y));
}

// 2 p - hl l - hr r, the stencil of a rho row (VAR)
template <typename T>
__device__ __forceinline__ T lapv(T l, T r, T p, T hl, T hr) {
  if constexpr (is_df<T>::value) return df_scale(p, 2.f) - (hl * l + hr * r);
  else return fma(T(2), p, -fma(hl, l, hr * r));
}

// One forward step of the VAR recurrence at interior point k.
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> var_forward(c2_t<T> prev, c2_t<T> left, c2_t<T> mid, c2_t<T> right,
                                               const c2_t<T>* alpha, const c2_t<T>* vbf, const c2_t<T>* vh, int k) {
  const c2_t<T> h = vh[k];
  const c2_t<T> lv = mk<T>(lapv(left.x, right.x, mid.x, h.x, h.y), lapv(left.y, right.y, mid.y, h.x, h.y));
  return cf_fma<T, IMAG>(alpha[k], prev, cf_mul<T, IMAG>(vbf[k], lv));
}

// Segment-local passes over SEG registers.  k0 = first interior index of the
// segment; points with k > M are padding (p = 0 there).
template <typename T, bool IMAG, int SEG, bool VAR = false>
__device__ __forceinline__ void local_forward(const c2_t<T> (&p)[SEG], c2_t<T> (&e)[SEG], c2_t<T> pl, c2_t<T> pr,
                                              const c2_t<T>* alpha, int k0, int M, const c2_t<T>* vbf = nullptr,
                                              const c2_t<T>* vh = nullptr) {
  c2_t<T> prev = mk<T>(0, 0);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    const c2_t<T> left = j == 0 ? pl : p[j - 1];
    const c2_t<T> right = j == SEG - 1 ? pr : p[j + 1];
    c2_t<T> v = mk<T>(0, 0);
    if constexpr (VAR) {
      if (k <= M) v = var_forward<T, IMAG>(prev, left, p[j], right, alpha, vbf, vh, k);
    } else {
      // t = e~_{k-1} - lap_k,  lap_k = left - 2 p_k + right
      const c2_t<T> t = mk<T>(prev.x + neg_lap(left.x, right.x, p[j].x), prev.y + neg_lap(left.y, right.y, p[j].y));
      if (k <= M) v = cf_mul<T, IMAG>(alpha[k], t);
    }
    e[j] = v;
    prev = v;
  }
}

template <typename T, bool IMAG, int SEG>
__device__ __forceinline__ void local_backward(c2_t<T> (&e)[SEG], const c2_t<T>* alpha, int k0, int M) {
  c2_t<T> next = mk<T>(0, 0);
#pragma unroll
  for (int j = SEG - 1; j >= 0; --j) {
    const int k = k0 + j;
    if (k <= M) next = cf_fma<T, IMAG>(alpha[k], next, e[j]);
    else next = mk<T>(0, 0);
    e[j] = next;
  }
}

// Shared-memory coefficient copy: alpha, gf, gb [n each] then Pf, Pb [512].
template <typename T>
__device__ __forceinline__ void load_coefs(const Sweep2Args<T>& A, c2_t<T>* sc, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    sc[k] = A.alpha[k];
    sc[n + k] = A.gf[k];
    sc[2 * n + k] = A.gb[k];
  }
  for (int q = threadIdx.x; q < 512; q += blockDim.x) sc[3 * n + q] = A.ptab[q];
}

// Forward pass over a segment whose points are fetched one at a time by
// getp(k) (0 outside 1..M), so the input segment need not sit in registers.
template <typename T, bool IMAG, int SEG, bool VAR = false, typename GetP>
__device__ __forceinline__ void stream_forward(GetP getp, c2_t<T> (&e)[SEG], const c2_t<T>* alpha, int k0, int M,
                                               const c2_t<T>* vbf = nullptr, const c2_t<T>* vh = nullptr) {
  using c2 = c2_t<T>;
  c2 pm = getp(k0 - 1), pc = getp(k0), prev = mk<T>(0, 0);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    const c2 pn = getp(k + 1);
    c2 v = mk<T>(0, 0);
    if constexpr (VAR) {
      if (k <= M) v = var_forward<T, IMAG>(prev, pm, pc, pn, alpha, vbf, vh, k);
    } else {
      const c2 t = mk<T>(prev.x + neg_lap(pm.x, pn.x, pc.x), prev.y + neg_lap(pm.y, pn.y, pc.y));
      if (k <= M) v = cf_mul<T, IMAG>(alpha[k], t);
    }
    e[j] = v;
    prev = v;
    pm = pc;
    pc = pn;
  }
}

// Completes the segment of thread (lane, warp s) of a block whose lines run
// one per lane and whose segments run one per warp: on entry z holds the
// segment-local forward values e^ (zero carry-in); on exit the increment z_k.
// Two block barriers; every thread of the block must call it.  vab: the
// backward coefficients of a rho axis (VAR), else those of sc.  cdepth, cpts
// (Sweep2Args): the carries' reach; the terms left out are products of the
// recurrence coefficients below the host's threshold (2^-48 for an FP32
// state, 2^-64 otherwise), far below a rounding of the carried value.
template <typename T, bool IMAG, int SEG>
__device__ __forceinline__ void seg_carries(c2_t<T> (&z)[SEG], const c2_t<T>* sc, int n, c2_t<T> (*cf)[33],
                                            c2_t<T> (*cb)[33], int s, int nseg, int lane,
                                            const c2_t<T>* vab = nullptr, int cdepth = 0, int cpts = 0) {
  using c2 = c2_t<T>;
  const int M = n - 2, k0 = 1 + s * SEG;
  const int dep = cdepth > 0 ? cdepth : 16;
  // cpts is 4, 8, 12 or 0 (every point): the carry loops below are unrolled for
  // each class, so that no per-point test is added; a partial last segment
  // takes every point
  const bool whole = k0 + SEG - 1 <= M;
  const c2* al = sc;
  const c2* gf = sc + n;
  const c2* gb = sc + 2 * n;
  const c2* Pf = sc + 3 * n;
  const c2* Pb = Pf + 256;
  {
    c2 Bend = z[SEG - 1];
#pragma unroll
    for (int j = 0; j < SEG; ++j) if (k0 + j == M) Bend = z[j];
    cf[s][lane] = Bend;
  }
  __syncthreads();
  c2 Ein = mk<T>(0, 0);
  for (int q = max(0, s - dep); q < s; ++q) Ein = cf_fma<T, IMAG>(Pf[q * 16 + s - 1], cf[q][lane], Ein);
  auto fwd = [&](auto nj) {
#pragma unroll
    for (int j = 0; j < decltype(nj)::value; ++j) {
      const int k = k0 + j;
      if (k <= M) z[j] = cf_fma<T, IMAG>(gf[k], Ein, z[j]);
    }
  };
  if (SEG > 4 && cpts == 4) fwd(std::integral_constant<int, (SEG > 4 ? 4 : SEG)>());
  else if (SEG > 8 && cpts == 8) fwd(std::integral_constant<int, (SEG > 8 ? 8 : SEG)>());
  else if (SEG > 12 && cpts == 12) fwd(std::integral_constant<int, (SEG > 12 ? 12 : SEG)>());
  else fwd(std::integral_constant<int, SEG>());
  local_backward<T, IMAG, SEG>(z, vab ? vab : al, k0, M);
  cb[s][lane] = z[0];
  __syncthreads();
  c2 Zin = mk<T>(0, 0);
  const int qe = min(nseg, s + 1 + dep);
  for (int q = s + 1; q < qe; ++q) Zin = cf_fma<T, IMAG>(Pb[q * 16 + s + 1], cb[q][lane], Zin);
  auto bwd = [&](auto nj) {
#pragma unroll
    for (int j = SEG - decltype(nj)::value; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) z[j] = cf_fma<T, IMAG>(gb[k], Zin, z[j]);
    }
  };
  if (SEG > 4 && whole && cpts == 4) bwd(std::integral_constant<int, (SEG > 4 ? 4 : SEG)>());
  else if (SEG > 8 && whole && cpts == 8) bwd(std::integral_constant<int, (SEG > 8 ? 8 : SEG)>());
  else if (SEG > 12 && whole && cpts == 12) bwd(std::integral_constant<int, (SEG > 12 ? 12 : SEG)>());
  else bwd(std::integral_constant<int, SEG>());
}

__device__ __forceinline__ int line_base32(const LineGeom& g, int L) {
  if (g.axis == 0) return L * g.nx;
  if (g.axis == 1) return (L % g.nx) + (L / g.nx) * g.nx * g.ny;
  return L;
}

// The closing half sub-step N(dt/2) of a Strang step at grid point q = (i, j,
// kz) (A's sub-step fields hold the dt/2 factors; no weight on the nonlinear
// term: 2d/3d grids).  The arithmetic of strang_phase_kernel.
template <typename T, bool IMAG>
__device__ __forceinline__ c2_t<T> half_phase(const Sweep2Args<T>& A, c2_t<T> w, long q, int i, int j, int kz) {
  if constexpr (is_df<T>::value) {
    return phase_df<IMAG>(w, A, q, i, j + A.geom.ny * kz, A.dtg);
  } else if constexpr (std::is_same<T, double>::value) {
    const c2_t<T> F = A.fV ? A.fV[q] : fac_mul<T, IMAG>(A.fx[i], fac_mul<T, IMAG>(A.fy[j], A.fz[kz]));
    return phase_N<T, IMAG>(w, F, A.dtg);
  } else {
    return phase_direct<T, IMAG>(w, A.V ? A.V[q] : A.vx[i] + (A.vy[j] + A.vz[kz]), A.dt, A.g);
  }
}

// Norm of the block's output: the per-thread values (in the state
// precision) are summed over the block in the state precision -- a tree of at
// most log2(blockDim) levels -- and stored as the block's FP64 sum; the next
// step's first sweep (or the final scaling) sums the blocks' values in FP64 in
// a fixed order (pending_scale).  No atomics, fences or last-block tail here.
template <typename T, bool LAST>
__device__ __forceinline__ void finish_norm(T tval, double* parts_out) {
  if (LAST) {
    __shared__ T tred[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tval += shfl_xor_t(tval, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) tred[warp] = tval;
    __syncthreads();
    if (warp == 0) {
      T b = lane < nw ? tred[lane] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) b += shfl_xor_t(b, o);
      if (lane == 0) parts_out[blockIdx.x] = (double)b;  // FP64 from here on
    }
  }
}

// ---------------------------------------------------------------- y/z sweep
// blockDim.x >= 32 * nseg, nseg = ceil((n-2)/SEG) <= 16, blockDim.x <= 512;
// dynamic shared memory holds the coefficients (3n + 512 complex values).
// Body shared with the batched kernels: lines L0 .. L0+31 of the grid
// described by A; nseg = ceil((n-2)/SEG) warps take part, the other warps of
// the block (if any) only join the barriers.
// RP (a real imaginary-time state viewed as complex): the complex point i' of
// a line holds the real values at x = 2i' (re) and 2i' + 1 (im); with real
// coefficients one complex sweep is the two real sweeps, and only the norm
// (LAST) needs the two x weights w_a[2i'], w_a[2i' + 1] apart.
// CLOSE (the last sweep of a Strang step): the closing sub-step N(dt/2) --
// A's sub-step fields hold the dt/2 factors -- is applied to every output
// point before it is stored and enters the norm, the same arithmetic as
// strang_phase_kernel's, so the step needs no extra pass over the state.
template <typename T, bool IMAG, bool LAST, int SEG, bool KEEP = (SEG * sizeof(T) <= 64), bool RP = false,
          bool CLOSE = false>
__device__ __forceinline__ void colsweep_body(const Sweep2Args<T>& A, int L0, c2_t<T>* sc, c2_t<T> (*cf)[33],
                                              c2_t<T> (*cb)[33], double* red_smem) {
  using c2 = c2_t<T>;
  const LineGeom& G = A.geom;
  const int n = G.n, M = n - 2;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
  const int nseg = (M + SEG - 1) / SEG;
  const bool seg_ok = s < nseg;
  const int L = L0 + lane;
  const bool active = L < G.nlines && seg_ok;
  const int st = (int)G.stride;
  const int k0 = 1 + s * SEG;
  load_coefs<T>(A, sc, n);
  pdl_wait();  // the state is the previous kernel's output
  pdl_release();
  c2* line = A.psi + (active ? line_base32(G, L) : 0);
  const long lim = G.points() - (line - A.psi);  // elements from the line's start to the array's end
  // KEEP: the input segment stays in registers; otherwise it is streamed in
  // the forward pass and read again (from L2) for u = p - z, which halves the
  // registers per thread and doubles the blocks an SM can hold
  c2 p[KEEP ? SEG : 1];
  if constexpr (KEEP) {
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      p[j] = (active && k <= M && GPE_CHECK((long)k * st < lim, 201)) ? line[k * st] : mk<T>(0, 0);
    }
  }
  __syncthreads();  // coefficients
  c2 z[SEG];
  if constexpr (KEEP) {
    const c2 pl = (active && k0 - 1 >= 1 && GPE_CHECK((long)(k0 - 1) * st < lim, 202)) ? line[(k0 - 1) * st]
                                                                                         : mk<T>(0, 0);
    const c2 pr = (active && k0 + SEG <= M && GPE_CHECK((long)(k0 + SEG) * st < lim, 203)) ? line[(k0 + SEG) * st]
                                                                                           : mk<T>(0, 0);
    local_forward<T, IMAG, SEG>(p, z, pl, pr, sc, k0, M);
  } else {
    stream_forward<T, IMAG, SEG>(
        [&](int k) {
          return (active && k >= 1 && k <= M && GPE_CHECK((long)k * st < lim, 204)) ? line[k * st] : mk<T>(0, 0);
        },
        z, sc, k0, M);
  }
  seg_carries<T, IMAG, SEG>(z, sc, n, cf, cb, s, nseg, lane, nullptr, A.cdepth, A.cpts);
  T nval = T(0);
  if (active) {
    const T* w = A.w_axis;
    T tacc = T(0), tim = T(0);
    // CLOSE: the line's x index and its other fixed index (z for y lines, y for z lines)
    const int ci = L % G.nx, cf2 = L / G.nx;
    const long qb = line - A.psi;
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) {
        c2 pk;
        if constexpr (KEEP) pk = p[j];
        else pk = GPE_CHECK((long)k * st < lim, 205) ? __ldcg(&line[k * st]) : mk<T>(0, 0);
        c2 u = sub2<T>(pk, z[j]);
        if constexpr (CLOSE) {
          const int jy = G.axis == 2 ? cf2 : k, kz = G.axis == 2 ? k : cf2;
          u = half_phase<T, IMAG>(A, u, qb + (long)k * st, ci, jy, kz);
        }
        if (GPE_CHECK((long)k * st < lim, 206)) line[k * st] = u;
        if constexpr (LAST && RP) {
          tacc += w[k] * (u.x * u.x);
          tim += w[k] * (u.y * u.y);
        } else if (LAST) {
          tacc += w[k] * (u.x * u.x + u.y * u.y);
        }
      }
    }
    if (s == 0 && GPE_CHECK((long)(n - 1) * st < lim, 207)) {
      line[0] = mk<T>(0, 0);
      line[(n - 1) * st] = mk<T>(0, 0);
    }
    if constexpr (LAST && RP) {
      const int i2 = 2 * (L % G.nx);
      nval = (tacc * A.w_a[i2] + tim * A.w_a[i2 + 1]) * A.w_b[L / G.nx];
    } else if (LAST) {
      nval = tacc * (A.w_a[L % G.nx] * A.w_b[L / G.nx]);
    }
  }
  finish_norm<T, LAST>(nval, A.parts_out);
}

template <typename T, bool IMAG, bool LAST, int SEG, bool KEEP, bool RP = false, bool CLOSE = false>
__global__ void __launch_bounds__(512) colsweep_kernel(Sweep2Args<T> A) {
  extern __shared__ __align__(16) unsigned char csmem_raw[];
  __shared__ c2_t<T> cf[16][33], cb[16][33];
  __shared__ double red_smem[32];
  colsweep_body<T, IMAG, LAST, SEG, KEEP, RP, CLOSE>(A, blockIdx.x * 32, reinterpret_cast<c2_t<T>*>(csmem_raw), cf,
                                                     cb, red_smem);
}

// ---------------------------------------------------------------- x sweep (2d/3d)
// Tile of 32 x lines in shared memory, transposed ([point][line], pitch 33).
// blockDim.x >= 32 * nseg (<= 512); dynamic shared memory: coefficients
// (3n + 512) then the tile (33 n) complex values.
constexpr int kTilePitch = 33;

// Body shared with the batched kernels: x lines L0 .. L0+31; sc points to
// 3n + 512 + 33n complex values of shared memory.
// RL (a real imaginary-time state, 2d/3d): tile column c holds the real x
// lines 2(L0+c) (re) and 2(L0+c) + 1 (im), so a tile covers 64 real lines
// and G.nlines counts real lines; N is applied to each real line with its own
// density and potential, and with real coefficients the complex solve of a
// column is the two real solves.
// VAR: the rho axis of an axial trap (see Sweep2Args::vab).
template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool RL = false, bool VAR = false>
__device__ __forceinline__ void tsweep_body(const Sweep2Args<T>& A, int L0, c2_t<T>* sc, c2_t<T> (*cf)[33],
                                            c2_t<T> (*cb)[33], double* red_smem) {
  static_assert(!(RL && (LAST || is_df<T>::value || !IMAG)), "packed real lines: imaginary-time x sweeps of 2d/3d");
  using c2 = c2_t<T>;
  const LineGeom& G = A.geom;
  const int n = G.n, M = n - 2;
  c2* tile = sc + 3 * n + 512;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nseg = (M + SEG - 1) / SEG;
  const int ncols = RL ? (int)((G.nlines + 1) / 2) : (int)G.nlines;  // tile columns in the grid
  const int nl = min(32, ncols - L0);
  load_coefs<T>(A, sc, n);
  pdl_wait();  // the state and the norm sums are the previous kernels' output
  pdl_release();
  constexpr bool kFactors = std::is_same<T, double>::value;  // FP64: precomputed potential factors
  const int per_line = (n + 31) >> 5;  // n <= 512: at most 16 chunks
  const c2* in = A.src ? A.src : A.psi;
  const T* rin = reinterpret_cast<const T*>(in);  // RL
  const long lim = G.points();  // complex values (RL: reals) of the array
  // per-line part of the sub-step N (FIRST) of grid line Lg
  auto line_factors = [&](int Lg, c2& fline, T& vline) {
    fline = mk<T>(1, 0);
    vline = T(0);
    if (FIRST && Lg < G.nlines && !is_df<T>::value) {
      if (kFactors && !A.fV) fline = fac_mul<T, IMAG>(A.fy[Lg % G.ny], A.fz[Lg / G.ny]);
      if (!kFactors && !A.V) vline = A.vy[Lg % G.ny] + A.vz[Lg / G.ny];
    }
  };
  // the factor scl and the sub-step N at interior point k of grid line Lg
  auto apply_N = [&](c2 w, int Lg, int k, const c2& fline, T vline, T scl) -> c2 {
    const int gbase = Lg * G.nx;
    if constexpr (is_df<T>::value) {
      if (IMAG) { w.x *= scl; w.y *= scl; }
      return phase_df<IMAG>(w, A, gbase + k, k, Lg, A.dtg);
    } else {
      w.x *= scl; w.y *= scl;
      if (kFactors) {
        const c2 F = A.fV ? A.fV[gbase + k] : fac_mul<T, IMAG>(A.fx[k], fline);
        return phase_N<T, IMAG>(w, F, A.dtg);
      } else {
        return phase_direct<T, IMAG>(w, A.V ? A.V[gbase + k] : A.vx[k] + vline, A.dt, A.g);
      }
    }
  };
  // RL: N on one real value (as the complex path does on (x, 0))
  auto apply_R = [&](T x, int Lg, int k, const c2& fline, T vline, T scl) -> T {
    return apply_N(mk<T>(x, T(0)), Lg, k, fline, vline, scl).x;
  };
  // A pending renormalisation factor (imaginary time, after the first step)
  // is summed by warp 0 from the previous step's per-block norms while the
  // other warps bring the tile in unchanged; the factor and N are then
  // applied in a second pass over the tile.  Otherwise N is applied on the
  // way in.  Either way: warp w takes columns w, w + nwarps, ...; lane takes
  // points lane, lane + 32, ... (coalesced rows; tile pitch 33, no conflicts).
  const bool pend = FIRST && A.parts_in != nullptr;
  if (pend && s == 0) {
    const double f = pending_factor_warp(A.parts_in, A.nparts_in, A.parts_wscale);
    if (lane == 0) red_smem[0] = f;
  }
  const int w0 = (pend && nwarps > 1) ? 1 : 0;  // first loading warp
  if (s >= w0) {
    for (int c = s - w0; c < 32; c += nwarps - w0) {
      const bool line_ok = c < nl;
      if constexpr (RL) {
        const int La = 2 * (L0 + c), Lb = La + 1;
        const bool oka = line_ok, okb = line_ok && Lb < G.nlines;
        c2 fa, fb;
        T va, vb;
        if (!pend) {
          line_factors(La, fa, va);
          line_factors(Lb, fb, vb);
        }
        for (int q0 = 0; q0 < per_line; q0 += 4) {
          c2 v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = (q0 + i) * 32 + lane;
            const bool in_k = k >= 1 && k <= M;
            v[i] = mk<T>((oka && in_k && GPE_CHECK((long)La * G.nx + k < lim, 211)) ? rin[La * G.nx + k] : T(0),
                         (okb && in_k && GPE_CHECK((long)Lb * G.nx + k < lim, 212)) ? rin[Lb * G.nx + k] : T(0));
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = (q0 + i) * 32 + lane;
            if (k >= n) break;
            c2 w = v[i];
            if (FIRST && !pend && k >= 1 && k <= M) {
              if (oka) w.x = apply_R(w.x, La, k, fa, va, T(1));
              if (okb) w.y = apply_R(w.y, Lb, k, fb, vb, T(1));
            }
            if (GPE_CHECK(k < n && c < 32, 213)) tile[k * kTilePitch + c] = w;
          }
        }
      } else {
        const int gbase = (L0 + c) * G.nx;
        c2 fline;
        T vline;
        if (!pend) line_factors(L0 + c, fline, vline);
        for (int q0 = 0; q0 < per_line; q0 += 4) {
          c2 v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = (q0 + i) * 32 + lane;
            v[i] = (line_ok && k >= 1 && k <= M && GPE_CHECK((long)gbase + k < lim, 214)) ? in[gbase + k]
                                                                                          : mk<T>(0, 0);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = (q0 + i) * 32 + lane;
            if (k >= n) break;
            c2 w = v[i];
            if (FIRST && !pend && line_ok && k >= 1 && k <= M) w = apply_N(w, L0 + c, k, fline, vline, T(1));
            if (GPE_CHECK(k < n && c < 32, 215)) tile[k * kTilePitch + c] = w;
          }
        }
      }
    }
  }
  if (pend) {
    __syncthreads();
    const T scl = (T)red_smem[0];
    for (int c = s; c < nl; c += nwarps) {
      if constexpr (RL) {
        const int La = 2 * (L0 + c), Lb = La + 1;
        const bool okb = Lb < G.nlines;
        c2 fa, fb;
        T va, vb;
        line_factors(La, fa, va);
        line_factors(Lb, fb, vb);
        for (int k = lane; k < n; k += 32)
          if (k >= 1 && k <= M) {
            c2 w = tile[k * kTilePitch + c];
            w.x = apply_R(w.x, La, k, fa, va, scl);
            if (okb) w.y = apply_R(w.y, Lb, k, fb, vb, scl);
            tile[k * kTilePitch + c] = w;
          }
      } else {
        c2 fline;
        T vline;
        line_factors(L0 + c, fline, vline);
        for (int k = lane; k < n; k += 32)
          if (k >= 1 && k <= M)
            tile[k * kTilePitch + c] = apply_N(tile[k * kTilePitch + c], L0 + c, k, fline, vline, scl);
      }
    }
  }
  __syncthreads();
  // ---- segments: lane = line, warp = segment; the input stays in the tile
  const int k0 = 1 + s * SEG;
  c2 z[SEG];
  stream_forward<T, IMAG, SEG, VAR>(
      [&](int k) { return (k >= 1 && k <= M) ? tile[k * kTilePitch + lane] : mk<T>(0, 0); }, z, sc, k0, M, A.vbf,
      A.vh);
  seg_carries<T, IMAG, SEG>(z, sc, n, cf, cb, s, nseg, lane, VAR ? A.vab : nullptr, A.cdepth, A.cpts);
  T tacc = T(0);
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int k = k0 + j;
    if (k <= M) {
      const c2 pk = tile[k * kTilePitch + lane];
      const c2 u = sub2<T>(pk, z[j]);
      tile[k * kTilePitch + lane] = u;
      if (LAST) tacc += A.w_axis[k] * (u.x * u.x + u.y * u.y);
    }
  }
  T nval = T(0);
  if (LAST && lane < nl) {
    const int L = L0 + lane;
    nval = tacc * (A.w_a[L % G.ny] * A.w_b[L / G.ny]);
  }
  __syncthreads();
  // ---- store (tile end points are zero)
  for (int c = s; c < nl; c += nwarps) {
    if constexpr (RL) {
      T* rout = reinterpret_cast<T*>(A.psi);
      const int La = 2 * (L0 + c), Lb = La + 1;
      for (int k = lane; k < n; k += 32)
        if (GPE_CHECK((long)La * G.nx + k < lim, 216)) rout[La * G.nx + k] = tile[k * kTilePitch + c].x;
      if (Lb < G.nlines)
        for (int k = lane; k < n; k += 32)
          if (GPE_CHECK((long)Lb * G.nx + k < lim, 217)) rout[Lb * G.nx + k] = tile[k * kTilePitch + c].y;
    } else {
      const int gbase = (L0 + c) * G.nx;
      for (int k = lane; k < n; k += 32)
        if (GPE_CHECK((long)gbase + k < lim, 218)) A.psi[gbase + k] = tile[k * kTilePitch + c];
    }
  }
  finish_norm<T, LAST>(nval, A.parts_out);
}

template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool RL = false, bool VAR = false>
__global__ void __launch_bounds__(512) tsweep_kernel(Sweep2Args<T> A) {
  extern __shared__ __align__(16) unsigned char tsmem_raw[];
  __shared__ c2_t<T> cf[16][33], cb[16][33];
  __shared__ double red_smem[32];
  tsweep_body<T, IMAG, FIRST, LAST, SEG, RL, VAR>(A, blockIdx.x * 32, reinterpret_cast<c2_t<T>*>(tsmem_raw), cf, cb,
                                         red_smem);
}

// ---------------------------------------------------------------- fused x + y sweeps (3d, FP32)
// One block per xy plane (fixed z index): the plane is loaded once into
// shared memory (rows along x, pitch nx + 1), the pending renormalisation
// factor and the sub-step N are applied as in the tile x sweep, then the x
// sweep runs on its rows (lane = row, warp = segment, up to four 32-row groups
// at once) and the y sweep on its columns (lane = column), both in place, and
// the plane is stored once: one read and one write of the state instead of
// two each, and one launch instead of two.  The per-line arithmetic is that
// of tsweep_body (x) and colsweep_body (y) with the same segment length.
// Ax: the x sweep's arguments (FIRST: sub-step fields, pending factor); Ay:
// the y axis' coefficients.  Needs nx, ny <= 128 so that the groups fit, and
// the plane in shared memory (checked by plane_fits on the host).
constexpr int kPlaneGroups = 4;

template <bool IMAG, int SEG>
__global__ void __launch_bounds__(1024) xyplane_kernel(Sweep2Args<float> Ax, Sweep2Args<float> Ay) {
  using T = float;
  using c2 = float2;
  extern __shared__ __align__(16) unsigned char plane_smem_raw[];
  __shared__ c2 cf[kPlaneGroups + 1][16][33], cb[kPlaneGroups + 1][16][33];
  __shared__ double red_smem[32];
  const int nx = Ax.geom.nx, ny = Ax.geom.ny;
  const int PX = nx + 1;
  c2* scx = reinterpret_cast<c2*>(plane_smem_raw);
  c2* scy = scx + 3 * nx + 512;
  c2* P = scy + 3 * ny + 512;
  const int kz = blockIdx.x;
  const long base = (long)kz * nx * ny;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  load_coefs<T>(Ax, scx, nx);
  load_coefs<T>(Ay, scy, ny);
  pdl_wait();  // the state and the norm sums are the previous kernels' output
  pdl_release();
  const int Mx = nx - 2, My = ny - 2;
  const c2* in = Ax.psi + base;
  const long lim = Ax.geom.points() - base;  // complex values from the plane's start to the array's end
  // per-row part of N (row j of plane kz is x line j + ny kz)
  auto row_v = [&](int j) -> T { return Ax.V ? T(0) : Ax.vy[j] + Ax.vz[kz]; };
  auto apply = [&](c2 w, int j, int i, T vline, T scl) -> c2 {
    w.x *= scl;
    w.y *= scl;
    return phase_direct<T, IMAG>(w, Ax.V ? Ax.V[base + (long)j * nx + i] : Ax.vx[i] + vline, Ax.dt, Ax.g);
  };
  const bool pend = Ax.parts_in != nullptr;
  if (pend && warp == 0) {
    const double f = pending_factor_warp(Ax.parts_in, Ax.nparts_in, Ax.parts_wscale);
    if (lane == 0) red_smem[0] = f;
  }
  // ---- load (N on the way in, or raw while warp 0 forms the pending factor);
  // four points of a row per lane at a time, their loads issued first
  const int w0 = (pend && nwarps > 1) ? 1 : 0;
  const int per_row = (nx + 31) >> 5;
  if (warp >= w0) {
    for (int j = warp - w0; j < ny; j += nwarps - w0) {
      const T vline = pend ? T(0) : row_v(j);
      for (int q0 = 0; q0 < per_row; q0 += 4) {
        c2 v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = (q0 + t) * 32 + lane;
          v[t] = (i >= 1 && i <= Mx && GPE_CHECK((long)j * nx + i < lim, 221)) ? in[(long)j * nx + i] : mk<T>(0, 0);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = (q0 + t) * 32 + lane;
          if (i >= nx) break;
          if (GPE_CHECK(j < ny && i < PX, 222))
            P[j * PX + i] = (!pend && i >= 1 && i <= Mx) ? apply(v[t], j, i, vline, T(1)) : v[t];
        }
      }
    }
  }
  if (pend) {
    __syncthreads();
    const T scl = (T)red_smem[0];
    for (int j = warp; j < ny; j += nwarps) {
      const T vline = row_v(j);
      for (int q0 = 0; q0 < per_row; q0 += 4) {
        c2 v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = (q0 + t) * 32 + lane;
          if (i >= 1 && i <= Mx) v[t] = P[j * PX + i];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = (q0 + t) * 32 + lane;
          if (i >= 1 && i <= Mx) P[j * PX + i] = apply(v[t], j, i, vline, scl);
        }
      }
    }
  }
  __syncthreads();
  // ---- x sweep: row j = 32 g + lane, segment s of x
  {
    const int nseg = (Mx + SEG - 1) / SEG, ng = (ny + 31) >> 5;
    int g = warp / nseg, s = warp % nseg;
    if (g > ng) g = ng;  // spare warps: a zero group, they only join the barriers
    const int j = 32 * g + lane;
    const bool row_ok = g < ng && j < ny;
    const int k0 = 1 + s * SEG;
    c2 z[SEG];
    stream_forward<T, IMAG, SEG>(
        [&](int k) { return (row_ok && k >= 1 && k <= Mx) ? P[j * PX + k] : mk<T>(0, 0); }, z, scx, k0, Mx);
    seg_carries<T, IMAG, SEG>(z, scx, nx, cf[g], cb[g], s, nseg, lane, nullptr, Ax.cdepth, Ax.cpts);
    if (row_ok) {
#pragma unroll
      for (int q = 0; q < SEG; ++q) {
        const int k = k0 + q;
        if (k <= Mx) P[j * PX + k] = sub2<T>(P[j * PX + k], z[q]);
      }
    }
  }
  __syncthreads();
  // ---- y sweep: column i = 32 g + lane, segment s of y
  {
    const int nseg = (My + SEG - 1) / SEG, ng = (nx + 31) >> 5;
    int g = warp / nseg, s = warp % nseg;
    if (g > ng) g = ng;
    const int i = 32 * g + lane;
    const bool col_ok = g < ng && i < nx;
    const int k0 = 1 + s * SEG;
    c2 z[SEG];
    stream_forward<T, IMAG, SEG>(
        [&](int k) { return (col_ok && k >= 1 && k <= My) ? P[k * PX + i] : mk<T>(0, 0); }, z, scy, k0, My);
    seg_carries<T, IMAG, SEG>(z, scy, ny, cf[g], cb[g], s, nseg, lane, nullptr, Ay.cdepth, Ay.cpts);
    if (col_ok) {
#pragma unroll
      for (int q = 0; q < SEG; ++q) {
        const int k = k0 + q;
        if (k <= My) P[k * PX + i] = sub2<T>(P[k * PX + i], z[q]);
      }
      if (s == 0) {  // the y ends are held at zero
        P[i] = mk<T>(0, 0);
        P[(ny - 1) * PX + i] = mk<T>(0, 0);
      }
    }
  }
  __syncthreads();
  // ---- store (x ends are zero), four points of a row per lane at a time
  c2* out = Ax.psi + base;
  for (int j = warp; j < ny; j += nwarps)
    for (int q0 = 0; q0 < per_row; q0 += 4) {
      c2 v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = (q0 + t) * 32 + lane;
        if (i < nx) v[t] = P[j * PX + i];
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = (q0 + t) * 32 + lane;
        if (i < nx && GPE_CHECK((long)j * nx + i < lim, 223)) out[(long)j * nx + i] = v[t];
      }
    }
}

// ---------------------------------------------------------------- x sweep (1d)
// One warp per line; lane j owns interior points k = 1 + j*SEG .. (j+1)*SEG;
// carries by a Kogge-Stone affine scan over shuffles.
// Body shared with the batched kernels: each warp takes line L.
// VAR: the rho axis of a circular or axial trap (see Sweep2Args::vab).
template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool VAR = false>
__device__ __forceinline__ void xsweep_body(const Sweep2Args<T>& A, int L, double* red_smem) {
  using c2 = c2_t<T>;
  const LineGeom& G = A.geom;
  const int lane = threadIdx.x & 31;
  const bool active = L < G.nlines;  // warp-uniform
  pdl_wait();
  pdl_release();
  // (every thread of the block takes part in the pending-scale reduction)
  const double pend = FIRST ? pending_scale(A.parts_in, A.nparts_in, A.parts_wscale, red_smem) : 1.0;
  T nval = T(0);
  if (active) {
    const int M = G.n - 2;
    const int base = L * G.nx;
    c2* line = A.psi + base;
    const int k0 = 1 + lane * SEG;
    const int ta = L % G.ny, tb = L / G.ny;
    constexpr bool kFactors = std::is_same<T, double>::value;  // FP64: precomputed potential factors
    c2 fline = mk<T>(1, 0);
    T vline = T(0);
    const T scl = (T)pend;
    if (FIRST && !is_df<T>::value) {
      if (kFactors && A.fV == nullptr) fline = fac_mul<T, IMAG>(A.fy[ta], A.fz[tb]);
      if (!kFactors && A.V == nullptr) vline = A.vy[ta] + A.vz[tb];
    }
    const c2* in = (A.src ? A.src : A.psi) + base;
    const long lim = G.points() - base;
    c2 p[SEG], e[SEG];
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      c2 v = mk<T>(0, 0);
      if (k <= M && GPE_CHECK(k < lim, 231)) {
        v = in[k];
        if constexpr (FIRST && is_df<T>::value) {
          if (IMAG) { v.x *= scl; v.y *= scl; }
          v = phase_df<IMAG>(v, A, base + k, k, L, A.gw ? A.dtg * A.gw[k] : A.dtg);
        } else if constexpr (FIRST) {
          v.x *= scl; v.y *= scl;
          if (kFactors) {
            const c2 F = A.fV ? A.fV[base + k] : fac_mul<T, IMAG>(A.fx[k], fline);
            v = phase_N<T, IMAG>(v, F, A.gw ? A.dtg * A.gw[k] : A.dtg);
          } else {
            v = phase_direct<T, IMAG>(v, A.V ? A.V[base + k] : A.vx[k] + vline, A.dt, A.gw ? A.g * A.gw[k] : A.g);
          }
        }
      }
      p[j] = v;
    }
    c2 pl = shfl_up2<T>(p[SEG - 1], 1);
    c2 pr = shfl_down2<T>(p[0], 1);
    if (lane == 0) pl = mk<T>(0, 0);
    if (lane == 31) pr = mk<T>(0, 0);
    local_forward<T, IMAG, SEG, VAR>(p, e, pl, pr, A.alpha, k0, M, A.vbf, A.vh);
    const int kend = k0 + SEG - 1;
    c2 Pm = (k0 <= M) ? __ldg(&A.gf[min(kend, M)]) : mk<T>(1, 0);
    c2 Bc = e[SEG - 1];
#pragma unroll
    for (int j = 0; j < SEG; ++j) if (k0 + j == M) Bc = e[j];
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
    // (the carries are applied to every point here: cutting them to A.cpts
    // points, as the block-wide sweeps do, made this latency-bound warp-per-line
    // sweep slower -- 1d FP32 10.4 -> 12.0 us per step at 513 points)
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) e[j] = cf_fma<T, IMAG>(__ldg(&A.gf[k]), Ein, e[j]);
    }
    local_backward<T, IMAG, SEG>(e, VAR ? A.vab : A.alpha, k0, M);
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
    T tacc = T(0);
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int k = k0 + j;
      if (k <= M) {
        const c2 z = cf_fma<T, IMAG>(__ldg(&A.gb[k]), Zin, e[j]);
        const c2 u = sub2<T>(p[j], z);
        if (GPE_CHECK(k < lim, 232)) line[k] = u;
        if (LAST) tacc += A.w_axis[k] * (u.x * u.x + u.y * u.y);
      }
    }
    if (lane == 0) line[0] = mk<T>(0, 0);
    if (lane == 31 && GPE_CHECK(G.n - 1 < lim, 233)) line[G.n - 1] = mk<T>(0, 0);
    if (LAST) nval = tacc * (A.w_a[ta] * A.w_b[tb]);
  }
  finish_norm<T, LAST>(nval, A.parts_out);
}

template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool VAR = false>
__global__ void __launch_bounds__(128) xsweep_kernel(Sweep2Args<T> A) {
  __shared__ double red_smem[32];
  xsweep_body<T, IMAG, FIRST, LAST, SEG, VAR>(A, blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), red_smem);
}

}  // namespace gpe

namespace gpe {

// ---------------------------------------------------------------- pipelined sweep
// Persistent blocks, each taking 32-line tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...; while one tile is solved the next is already on its way
// into the second shared-memory stage (cp.async, zero-filled outside the
// interior), so the memory system never waits for a block to finish its
// arithmetic.  Tile layout per stage: y/z lines [point][line] with pitch 33,
// x lines [line][point] with pitch n + 1 -- both conflict-free for the
// lane = line reads of the solve.  The coefficient tables are loaded once per
// block, the norm (LAST) is reduced once per block.  blockDim.x = 32 * nseg.

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// async copy of one complex value (8 or 16 bytes); src_bytes = 0 zero-fills
template <typename T>
__device__ __forceinline__ void cp_async_c2(c2_t<T>* dst, const c2_t<T>* src, bool valid) {
  const unsigned d = smem_u32(dst);
  if constexpr (sizeof(c2_t<T>) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0));
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Issues the copies of tile `tile` into stage buffer `buf` (every thread its share).
template <typename T, bool AXIS0>
__device__ __forceinline__ void psweep_issue(const Sweep2Args<T>& A, int tile, c2_t<T>* buf, int pitch) {
  const LineGeom& G = A.geom;
  const int n = G.n, M = n - 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int L0 = tile * 32;
  const int nl = min(32, (int)G.nlines - L0);
  const c2_t<T>* in = A.src ? A.src : A.psi;
  if (AXIS0) {
    for (int c = w; c < 32; c += nwarps) {
      const bool lok = c < nl;
      const int gbase = lok ? (L0 + c) * G.nx : 0;
      for (int k = lane; k < n; k += 32)
        if (GPE_CHECK((long)gbase + k < G.points() && c * pitch + k < 32 * pitch, 241))
          cp_async_c2<T>(buf + c * pitch + k, in + gbase + k, lok && k >= 1 && k <= M);
    }
  } else {
    const bool lok = lane < nl;
    const int base = lok ? line_base32(G, L0 + lane) : 0;
    const int st = (int)G.stride;
    for (int k = w; k < n; k += nwarps)
      if (GPE_CHECK((long)base + (long)k * st < G.points(), 242))
        cp_async_c2<T>(buf + k * kTilePitch + lane, in + base + k * st, lok && k >= 1 && k <= M);
  }
}

template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool AXIS0>
__global__ void __launch_bounds__(512) psweep_kernel(Sweep2Args<T> A) {
  using c2 = c2_t<T>;
  extern __shared__ __align__(16) unsigned char psmem_raw[];
  __shared__ c2 cf[16][33], cb[16][33];
  __shared__ double red_smem[32];
  const LineGeom& G = A.geom;
  const int n = G.n, M = n - 2;
  const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
  const int nseg = blockDim.x >> 5;
  const int k0 = 1 + s * SEG;
  const int pitch = AXIS0 ? n + 1 : kTilePitch;
  const int stage_elems = AXIS0 ? 32 * (n + 1) : n * kTilePitch;
  c2* sc = reinterpret_cast<c2*>(psmem_raw);
  c2* stage[2] = {sc + 3 * n + 512, sc + 3 * n + 512 + stage_elems};
  const int ntiles = (int)((G.nlines + 31) / 32);
  load_coefs<T>(A, sc, n);
  pdl_wait();
  pdl_release();
  T scl = T(1);
  if (FIRST) scl = (T)pending_scale(A.parts_in, A.nparts_in, A.parts_wscale, red_smem);
  constexpr bool kFactors = std::is_same<T, double>::value;
  static_assert(!is_df<T>::value, "the pipelined sweeps take FP32 and FP64 states");
  T tval = T(0);
  int it = 0;
  if (blockIdx.x < ntiles) psweep_issue<T, AXIS0>(A, blockIdx.x, stage[0], pitch);
  cp_async_commit();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    c2* buf = stage[it & 1];
    const int next = tile + gridDim.x;
    if (next < ntiles) psweep_issue<T, AXIS0>(A, next, stage[(it + 1) & 1], pitch);
    cp_async_commit();
    cp_async_wait<1>();  // this tile's group has landed (the newest may still be in flight)
    __syncthreads();
    const int L0 = tile * 32;
    const int nl = min(32, (int)G.nlines - L0);
    auto at = [&](int k) -> c2& { return AXIS0 ? buf[lane * pitch + k] : buf[k * kTilePitch + lane]; };
    if (FIRST) {
      // sub-step N (and the pending renormalisation) on this thread's own points
      if (lane < nl) {
        const int L = L0 + lane;
        c2 fline = mk<T>(1, 0);
        T vline = T(0);
        if (kFactors && !A.fV) fline = fac_mul<T, IMAG>(A.fy[L % G.ny], A.fz[L / G.ny]);
        if (!kFactors && !A.V) vline = A.vy[L % G.ny] + A.vz[L / G.ny];
        const int gb = L * G.nx;
#pragma unroll
        for (int j = 0; j < SEG; ++j) {
          const int k = k0 + j;
          if (k <= M) {
            c2 w = at(k);
            w.x *= scl; w.y *= scl;
            if (kFactors) {
              const c2 F = A.fV ? A.fV[gb + k] : fac_mul<T, IMAG>(A.fx[k], fline);
              w = phase_N<T, IMAG>(w, F, A.dtg);
            } else {
              w = phase_direct<T, IMAG>(w, A.V ? A.V[gb + k] : A.vx[k] + vline, A.dt, A.g);
            }
            at(k) = w;
          }
        }
      }
      __syncthreads();
    }
    c2 z[SEG];
    stream_forward<T, IMAG, SEG>([&](int k) { return (k >= 1 && k <= M) ? at(k) : mk<T>(0, 0); }, z, sc, k0, M);
    seg_carries<T, IMAG, SEG>(z, sc, n, cf, cb, s, nseg, lane, nullptr, A.cdepth, A.cpts);
    T tacc = T(0);
    if (AXIS0) {
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        const int k = k0 + j;
        if (k <= M) {
          const c2 p = at(k);
          const c2 u = sub2<T>(p, z[j]);
          at(k) = u;
          if (LAST) tacc += A.w_axis[k] * (u.x * u.x + u.y * u.y);
        }
      }
      __syncthreads();
      // coalesced store of the tile: warp w takes lines w, w + nseg, ...
      for (int c = s; c < nl; c += nseg) {
        const int gbase = (L0 + c) * G.nx;
        for (int k = lane; k < n; k += 32)
          if (GPE_CHECK((long)gbase + k < G.points(), 243)) A.psi[gbase + k] = buf[c * pitch + k];
      }
    } else if (lane < nl) {
      c2* line = A.psi + line_base32(G, L0 + lane);
      const int st = (int)G.stride;
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        const int k = k0 + j;
        if (k <= M) {
          const c2 p = at(k);
          const c2 u = sub2<T>(p, z[j]);
          if (GPE_CHECK((line - A.psi) + (long)k * st < G.points(), 244)) line[k * st] = u;
          if (LAST) tacc += A.w_axis[k] * (u.x * u.x + u.y * u.y);
        }
      }
      if (s == 0 && GPE_CHECK((line - A.psi) + (long)(n - 1) * st < G.points(), 245)) {
        line[0] = mk<T>(0, 0);
        line[(n - 1) * st] = mk<T>(0, 0);
      }
    }
    if (LAST && lane < nl) {
      const int L = L0 + lane;
      tval += AXIS0 ? tacc * (A.w_a[L % G.ny] * A.w_b[L / G.ny]) : tacc * (A.w_a[L % G.nx] * A.w_b[L / G.nx]);
    }
    __syncthreads();  // the stage is refilled by the prefetch of the next iteration
  }
  cp_async_wait<0>();
  finish_norm<T, LAST>(tval, A.parts_out);
}

// ------------------------------------------------------- closing N of Strang
// The symmetric splitting's second half sub-step N(dt/2), on the output of
// the last sweep, with the Simpson-weighted norm of its result (imaginary
// time, LAST) left per block as the sweeps' LAST does.  A's sub-step fields
// hold the dt/2 factors and dtg = dt g/2 (FP32: dt/2); w_axis, w_a, w_b are
// the Simpson coefficients of x, y and z.  A warp takes chunks of 32
// consecutive points of one x line (coalesced), kStrangUnroll chunks at a
// time with all their loads issued first (a read and a write per point:
// enough bytes in flight per SM to stream at HBM rate); grid-stride over all
// chunks.  The chunk count is below 2^26 (np < 2^31), so the index
// arithmetic is 32-bit.
constexpr int kStrangUnroll = 4;

template <typename T, bool IMAG, bool LAST>
__global__ void __launch_bounds__(256) strang_phase_kernel(Sweep2Args<T> A) {
  using c2 = c2_t<T>;
  const LineGeom& G = A.geom;
  pdl_wait();
  pdl_release();
  const int lane = threadIdx.x & 31;
  const unsigned cpl = (unsigned)(G.nx + 31) >> 5;  // chunks per x line
  const unsigned nchunks = cpl * (unsigned)G.nlines;
  const unsigned nwarps = gridDim.x * (blockDim.x >> 5);
  constexpr bool kFactors = std::is_same<T, double>::value;
  T tacc = T(0);
  for (unsigned u0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kStrangUnroll; u0 < nchunks;
       u0 += nwarps * kStrangUnroll) {
    c2 v[kStrangUnroll];
    long q[kStrangUnroll];
    int ii[kStrangUnroll], ll[kStrangUnroll];
    bool ok[kStrangUnroll];
#pragma unroll
    for (int r = 0; r < kStrangUnroll; ++r) {
      const unsigned u = u0 + r, L = u / cpl;
      ii[r] = (int)(u - L * cpl) * 32 + lane;
      ll[r] = (int)L;
      ok[r] = u < nchunks && ii[r] < G.nx;
      q[r] = (long)L * G.nx + ii[r];
      ok[r] = ok[r] && GPE_CHECK(q[r] < G.points(), 251);
      if (ok[r]) v[r] = A.psi[q[r]];
    }
#pragma unroll
    for (int r = 0; r < kStrangUnroll; ++r) {
      if (!ok[r]) continue;
      const int i = ii[r], L = ll[r], j = L % G.ny, k = L / G.ny;
      c2 w = v[r];
      if constexpr (is_df<T>::value) {
        w = phase_df<IMAG>(w, A, q[r], i, L, A.gw ? A.dtg * A.gw[i] : A.dtg);
      } else if constexpr (kFactors) {
        const c2 F = A.fV ? A.fV[q[r]] : fac_mul<T, IMAG>(A.fx[i], fac_mul<T, IMAG>(A.fy[j], A.fz[k]));
        w = phase_N<T, IMAG>(w, F, A.gw ? A.dtg * A.gw[i] : A.dtg);
      } else {
        w = phase_direct<T, IMAG>(w, A.V ? A.V[q[r]] : A.vx[i] + (A.vy[j] + A.vz[k]), A.dt,
                                  A.gw ? A.g * A.gw[i] : A.g);
      }
      A.psi[q[r]] = w;
      if (LAST) tacc += (A.w_axis[i] * (A.w_a[j] * A.w_b[k])) * (w.x * w.x + w.y * w.y);
    }
  }
  finish_norm<T, LAST>(tacc, A.parts_out);
}
}  // namespace gpe
