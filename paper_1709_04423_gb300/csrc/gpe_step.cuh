// gpe_step.cuh -- per-step launch sequence of the split-step propagator,
// instantiated once per state precision (gpe_step_f32.cu, gpe_step_f64.cu).
//
// One step = N fused into the x sweep, then the y sweep, then the z sweep; in
// imaginary time the last sweep also produces the next renormalisation factor
// from the Simpson norm, consumed by the next step's x sweep (two device
// slots, alternating with the step parity), and a final kernel applies the
// last factor.  Step blocks of kGraphSteps steps are captured once into a CUDA
// graph and replayed.
#pragma once
#include <algorithm>
#include <cstring>

#include "gpe_adjoint.cuh"
#include "gpe_internal.h"
#include "gpe_obs.cuh"
#include "gpe_sweep.cuh"
#include "gpe_sweep2.cuh"
#include "gpe_tma.cuh"

#include <cudaTypedefs.h>

namespace gpe {

constexpr int kLegacyThreads = 128;
constexpr int kXWarps = 4;
constexpr int kGraphSteps = 16;  // even: keeps the renormalisation-slot parity

inline LineGeom geom_of(const gp_handle* h, int axis) {
  LineGeom g;
  g.axis = axis;
  g.nx = axis_len(h, 0);
  g.ny = axis_len(h, 1);
  g.nz = axis_len(h, 2);
  g.n = axis_len(h, axis);
  g.stride = axis == 0 ? 1 : axis == 1 ? g.nx : (long)g.nx * g.ny;
  g.nlines = h->np / g.n;
  return g;
}

template <typename T>
inline const c2_t<T>* coef_ptr(const gp_handle* h, int mode, int axis, int slot) {
  return (const c2_t<T>*)h->coef[mode][axis] + (size_t)slot * h->n[axis];
}

// ---- segmented x sweep
// Every launcher returns its number of blocks (a LAST sweep leaves one norm
// sum per block for the next step's reader).
template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool VAR = false>
unsigned launch_x(const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  const unsigned blocks = (unsigned)((a.geom.nlines + kXWarps - 1) / kXWarps);
  launch_k(pdl, xsweep_kernel<T, IMAG, FIRST, LAST, SEG, VAR>, dim3(blocks), dim3(32 * kXWarps), 0, s, a);
  count_launch();
  return blocks;
}

template <typename T, bool IMAG, bool FIRST, bool LAST, bool VAR = false>
unsigned launch_x_seg(int seg, const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  switch (seg) {
    case 1: return launch_x<T, IMAG, FIRST, LAST, 1, VAR>(a, s, pdl);
    case 2: return launch_x<T, IMAG, FIRST, LAST, 2, VAR>(a, s, pdl);
    case 4: return launch_x<T, IMAG, FIRST, LAST, 4, VAR>(a, s, pdl);
    case 8: return launch_x<T, IMAG, FIRST, LAST, 8, VAR>(a, s, pdl);
    default: return launch_x<T, IMAG, FIRST, LAST, 16, VAR>(a, s, pdl);
  }
}

// ---- segmented y/z sweep (registers, coefficients in shared memory)
template <typename T, bool IMAG, bool LAST, int SEG, bool KEEP, bool RP = false, bool CLOSE = false>
unsigned launch_c(const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  const int M = a.geom.n - 2;
  const int nseg = (M + SEG - 1) / SEG;
  const unsigned blocks = (unsigned)((a.geom.nlines + 31) / 32);
  const size_t smem = (size_t)(3 * a.geom.n + 512) * sizeof(c2_t<T>);
  // static + dynamic shared memory can pass 48 KB
  opt_in_smem((const void*)colsweep_kernel<T, IMAG, LAST, SEG, KEEP, RP, CLOSE>, 64 * 1024);
  launch_k(pdl, colsweep_kernel<T, IMAG, LAST, SEG, KEEP, RP, CLOSE>, dim3(blocks), dim3(32 * nseg), smem, s, a);
  count_launch();
  return blocks;
}

// keep = 1: input segment in registers (only for short segments); 0: streamed
template <typename T, bool IMAG, bool LAST, bool RP = false, bool CLOSE = false>
unsigned launch_c_seg(int seg, int keep, const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  const bool k = keep && seg * (int)sizeof(T) <= 64;
  switch (seg) {
    case 4:
      return k ? launch_c<T, IMAG, LAST, 4, true, RP, CLOSE>(a, s, pdl)
               : launch_c<T, IMAG, LAST, 4, false, RP, CLOSE>(a, s, pdl);
    case 8:
      return k ? launch_c<T, IMAG, LAST, 8, true, RP, CLOSE>(a, s, pdl)
               : launch_c<T, IMAG, LAST, 8, false, RP, CLOSE>(a, s, pdl);
    case 16:
      return k ? launch_c<T, IMAG, LAST, 16, true, RP, CLOSE>(a, s, pdl)
               : launch_c<T, IMAG, LAST, 16, false, RP, CLOSE>(a, s, pdl);
    default: return launch_c<T, IMAG, LAST, 32, false, RP, CLOSE>(a, s, pdl);
  }
}

// ---- fused x + y sweeps of a 3d FP32 grid (one block per xy plane)
template <bool IMAG, int SEG>
unsigned launch_xy(const Sweep2Args<float>& ax, const Sweep2Args<float>& ay, cudaStream_t s, bool pdl) {
  const int nx = ax.geom.nx, ny = ax.geom.ny;
  const int wx = ((nx - 2 + SEG - 1) / SEG) * ((ny + 31) / 32), wy = ((ny - 2 + SEG - 1) / SEG) * ((nx + 31) / 32);
  const int threads = 32 * std::max(wx, wy);
  const size_t smem = (size_t)(3 * nx + 512 + 3 * ny + 512 + ny * (nx + 1)) * sizeof(float2);
  opt_in_smem((const void*)xyplane_kernel<IMAG, SEG>, 180 * 1024);
  launch_k(pdl, xyplane_kernel<IMAG, SEG>, dim3(ax.geom.nz), dim3(threads), smem, s, ax, ay);
  count_launch();
  return (unsigned)ax.geom.nz;
}

template <bool IMAG>
unsigned launch_xy_seg(int seg, const Sweep2Args<float>& ax, const Sweep2Args<float>& ay, cudaStream_t s, bool pdl) {
  switch (seg) {
    case 8: return launch_xy<IMAG, 8>(ax, ay, s, pdl);
    case 16: return launch_xy<IMAG, 16>(ax, ay, s, pdl);
    default: return launch_xy<IMAG, 32>(ax, ay, s, pdl);
  }
}

// Whether the x and y sweeps of this handle run as one kernel (the complex
// state of a 3d FP32 grid whose planes fit; the adjoint's sweeps, which read
// the step's input from another buffer, run apart).
inline bool xy_fused(const gp_handle* h) {
  return h->xyfuse && h->prec == GP_F32 && h->dim == 3 && !h->real_mode;
}

// ---- shared-memory tile x sweep
// (RL: a.geom.nlines real lines, two per tile column; VAR: a rho axis)
template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool RL = false, bool VAR = false>
unsigned launch_t(const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  const int M = a.geom.n - 2;
  const int nseg = (M + SEG - 1) / SEG;
  const long ncols = RL ? (a.geom.nlines + 1) / 2 : a.geom.nlines;
  const unsigned blocks = (unsigned)((ncols + 31) / 32);
  const size_t smem = (size_t)a.geom.n * (kTilePitch + 3) * sizeof(c2_t<T>) + 512 * sizeof(c2_t<T>);
  opt_in_smem((const void*)tsweep_kernel<T, IMAG, FIRST, LAST, SEG, RL, VAR>, 200 * 1024);
  launch_k(pdl, tsweep_kernel<T, IMAG, FIRST, LAST, SEG, RL, VAR>, dim3(blocks), dim3(32 * nseg), smem, s, a);
  count_launch();
  return blocks;
}

template <typename T, bool IMAG, bool FIRST, bool LAST, bool RL = false, bool VAR = false>
unsigned launch_t_seg(int seg, const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  switch (seg) {
    case 4: return launch_t<T, IMAG, FIRST, LAST, 4, RL, VAR>(a, s, pdl);
    case 8: return launch_t<T, IMAG, FIRST, LAST, 8, RL, VAR>(a, s, pdl);
    case 16: return launch_t<T, IMAG, FIRST, LAST, 16, RL, VAR>(a, s, pdl);
    default: return launch_t<T, IMAG, FIRST, LAST, 32, RL, VAR>(a, s, pdl);
  }
}

// ---- pipelined (persistent, double-buffered) sweeps
template <typename T>
inline size_t psweep_smem(int n, bool axis0) {
  const size_t stage = axis0 ? 32 * (size_t)(n + 1) : (size_t)n * kTilePitch;
  return (3 * (size_t)n + 512 + 2 * stage) * sizeof(c2_t<T>);
}

template <typename T, bool IMAG, bool FIRST, bool LAST, int SEG, bool AXIS0>
unsigned launch_p(const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  const int M = a.geom.n - 2;
  const int nseg = (M + SEG - 1) / SEG;
  const int ntiles = (int)((a.geom.nlines + 31) / 32);
  const size_t smem = psweep_smem<T>(a.geom.n, AXIS0);
  opt_in_smem((const void*)psweep_kernel<T, IMAG, FIRST, LAST, SEG, AXIS0>, smem);  // static + dynamic <= 227 KB
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, psweep_kernel<T, IMAG, FIRST, LAST, SEG, AXIS0>, 32 * nseg,
                                                smem);
  const int blocks = std::max(1, std::min(ntiles, std::max(1, per_sm) * std::max(1, sms)));
  launch_k(pdl, psweep_kernel<T, IMAG, FIRST, LAST, SEG, AXIS0>, dim3(blocks), dim3(32 * nseg), smem, s, a);
  count_launch();
  return (unsigned)blocks;
}

template <typename T, bool IMAG, bool FIRST, bool LAST, bool AXIS0>
unsigned launch_p_seg(int seg, const Sweep2Args<T>& a, cudaStream_t s, bool pdl) {
  switch (seg) {
    case 4: return launch_p<T, IMAG, FIRST, LAST, 4, AXIS0>(a, s, pdl);
    case 8: return launch_p<T, IMAG, FIRST, LAST, 8, AXIS0>(a, s, pdl);
    case 16: return launch_p<T, IMAG, FIRST, LAST, 16, AXIS0>(a, s, pdl);
    default: return launch_p<T, IMAG, FIRST, LAST, 32, AXIS0>(a, s, pdl);
  }
}

// ---- TMA-pipelined persistent y/z sweeps (FP32 state; gpe_tma.cuh)
// The tensor-map encoder is a driver entry point, looked up through the
// runtime (no link against the driver library).
inline PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The FP32 state (nx, ny, nz complex values of 8 bytes, x fastest) as a 3d
// tensor whose box is 32 x positions times a whole y line (axis 1) or z line
// (axis 2).  Needs nx even (row strides a multiple of 16 bytes) and the line
// length <= 256 (a box dimension's limit); false if the driver refuses.
inline bool encode_line_map(CUtensorMap* m, void* psi, const LineGeom& g) {
  auto enc = tmap_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 8, (cuuint64_t)g.nx * g.ny * 8};
  const cuuint32_t box[3] = {32u, g.axis == 1 ? (cuuint32_t)g.ny : 1u, g.axis == 2 ? (cuuint32_t)g.nz : 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, psi, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t tmacol_smem(int n) {
  const size_t coef = (size_t)(3 * n + 512) * 8;
  return ((coef + 1023) / 1024) * 1024 + 1024 + (size_t)kTmaStages * 32 * n * 8;
}

template <bool IMAG, bool LAST, int SEG, bool CLOSE>
unsigned launch_tc(gp_handle* h, const Sweep2Args<float>& a, cudaStream_t s, bool pdl) {
  const LineGeom& g = a.geom;
  const int nseg = (g.n - 2 + SEG - 1) / SEG;
  const size_t smem = tmacol_smem(g.n);
  auto kern = tmacol_kernel<IMAG, LAST, SEG, CLOSE>;
  opt_in_smem((const void*)kern, smem);
  CUtensorMap map;
  if (!encode_line_map(&map, a.psi, g)) {
    g_err = "cuTensorMapEncodeTiled refused the state's tensor map";
    return 0;
  }
  TmaTiles T;
  T.nxt = (g.nx + 31) / 32;
  T.ntiles = T.nxt * (g.axis == 1 ? g.nz : g.ny);
  T.limit_ns = h->tma_limit_ns;
  T.expect_extra = h->tma_expect_extra;
  T.err = h->dev_err;
  T.depth = 0;  // (x sweep only)
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * (nseg + 1), smem);
  const int blocks = std::max(1, std::min(T.ntiles, std::max(1, per_sm) * std::max(1, sms)));
  launch_k(pdl, kern, dim3(blocks), dim3(32 * (nseg + 1)), smem, s, map, a, T);
  count_launch();
  return (unsigned)blocks;
}

// The FP32 state as (16, nx/16, nlines) 8-byte elements -- 16-point chunks of
// the x lines -- with the box (16, 1, 32) and the 128-byte swizzle (the TMA x
// sweep's tiles).  Needs nx a multiple of 16.
inline bool encode_row_map(CUtensorMap* m, void* psi, const LineGeom& g) {
  auto enc = tmap_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {16u, (cuuint64_t)(g.nx / 16), (cuuint64_t)g.nlines};
  const cuuint64_t strides[2] = {128u, (cuuint64_t)g.nx * 8};
  const cuuint32_t box[3] = {16u, 1u, 32u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, psi, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t tmarow_smem(int n) {
  const size_t coef = (size_t)(3 * n + 512) * 8 + (size_t)n * 4;
  return ((coef + 1023) / 1024) * 1024 + 1024 + (size_t)kTmaStages * 32 * n * 8;
}

template <bool IMAG, int SEG>
unsigned launch_tx(gp_handle* h, Sweep2Args<float> a, int mode, cudaStream_t s, bool pdl) {
  const LineGeom& g = a.geom;
  const int nseg = g.n / SEG;
  const size_t smem = tmarow_smem(g.n);
  const int si = SEG == 8 ? 0 : 1;
  // the points of a segment that take a carry (the host's bound on the tables)
  const int nj = h->even_nj[mode][si];
  auto kern = nj <= 4 ? tmarow_kernel<IMAG, SEG, 4> : (nj <= 8 ? tmarow_kernel<IMAG, SEG, 8> : tmarow_kernel<IMAG, SEG, SEG>);
  opt_in_smem((const void*)kern, smem);
  // the tables of segments aligned to even points
  const float2* ev = (const float2*)h->coef_even[mode];
  a.gf = ev + (size_t)(2 * si) * g.n;
  a.gb = ev + (size_t)(2 * si + 1) * g.n;
  a.ptab = ev + (size_t)4 * g.n + 512 * si;
  CUtensorMap map;
  if (!encode_row_map(&map, a.psi, g)) {
    g_err = "cuTensorMapEncodeTiled refused the state's tensor map";
    return 0;
  }
  TmaTiles T;
  T.nxt = 1;
  T.ntiles = (int)((g.nlines + 31) / 32);
  T.limit_ns = h->tma_limit_ns;
  T.expect_extra = h->tma_expect_extra;
  T.err = h->dev_err;
  T.depth = std::max(1, h->even_depth[mode][si]);
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * (nseg + 1), smem);
  const int blocks = std::max(1, std::min(T.ntiles, std::max(1, per_sm) * std::max(1, sms)));
  // nseg consumer warps (one per segment) and one producer warp
  launch_k(pdl, kern, dim3(blocks), dim3(32 * (nseg + 1)), smem, s, map, a, T);
  count_launch();
  return (unsigned)blocks;
}

template <bool IMAG, bool LAST, bool CLOSE = false>
unsigned launch_tc_seg(gp_handle* h, int seg, const Sweep2Args<float>& a, cudaStream_t s, bool pdl) {
  switch (seg) {
    case 8: return launch_tc<IMAG, LAST, 8, CLOSE>(h, a, s, pdl);
    case 16: return launch_tc<IMAG, LAST, 16, CLOSE>(h, a, s, pdl);
    default: return launch_tc<IMAG, LAST, 32, CLOSE>(h, a, s, pdl);
  }
}

// ---- thread-per-line fallback (lines longer than the segmented kernels take)
template <typename T, bool IMAG, bool FIRST, bool LAST>
unsigned launch_legacy(const SweepArgs<T>& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.geom.nlines + kLegacyThreads - 1) / kLegacyThreads);
  cn_sweep_kernel<T, IMAG, FIRST, LAST><<<blocks, kLegacyThreads, 0, s>>>(a);
  count_launch();
  return blocks;
}

// Slots of the imaginary-time renormalisation: step t > 0 of a call reads the
// per-block norm sums left by step t-1 in slot (t-1) & 1 and its last sweep
// writes slot t & 1; step 0 reads nothing (the state is taken as given).
struct NormSlots {
  int rd = -1, wr = -1;
};

// The sub-step N fields of the sweep arguments: step dt, or dt/2 for the
// halves of the Strang splitting.
template <typename T, typename A>
void set_phase_args(const gp_handle* h, bool imag, bool half, A& a) {
  const int fm = imag ? 1 : 0;
  const double dt = half ? 0.5 * h->dt : h->dt;
  void* const* fac = half ? h->fac_h[fm] : h->fac[fm];
  if constexpr (std::is_same<A, Sweep2Args<T>>::value) {
    a.fV = h->Vd ? (const c2_t<T>*)(half ? h->fV_h : h->fV)[fm] : nullptr;
    a.fx = (const c2_t<T>*)fac[0];
    a.fy = (const c2_t<T>*)fac[1];
    a.fz = (const c2_t<T>*)fac[2];
    a.dtg = (T)(dt * h->g);
    if constexpr (is_df<T>::value) {
      a.tfV = h->Vd ? (const tf3c*)(half ? h->tfV_h : h->tfV)[fm] : nullptr;
      a.tfx = (const tf3c*)(half ? h->tfx_h : h->tfx)[fm];
      a.tfyz = (const tf3c*)(half ? h->tfyz_h : h->tfyz)[fm];
    }
  }
  a.V = (const T*)h->Vt;
  a.vx = (const T*)h->vt[0];
  a.vy = (const T*)h->vt[1];
  a.vz = (const T*)h->vt[2];
  a.dt = (T)dt;
  a.g = (T)h->g;
  a.gw = (const T*)h->gw_t;
}

// How a step's sub-step N is split under the Strang splitting.  Imaginary-time
// steps run N(dt/2), the sweeps, N(dt/2).  In a run of real-time steps the
// closing half of one step and the opening half of the next make one N(dt)
// (in real time N keeps |phi|, so the two halves compose exactly, up to
// rounding), so the run is N(dt/2) and the sweeps, then N(dt) and the sweeps
// per further step, then N(dt/2): the cost of the Lie steps plus one pass.
struct StepForm {
  bool half_open = true;  // the x sweep applies N(dt/2) (else N(dt))
  bool close = true;      // N(dt/2) after the last sweep
};

// Whether an imaginary-time Strang step applies its closing N(dt/2) inside
// its last sweep (a segmented y/z sweep of a 2d/3d grid) rather than in
// strang_phase_kernel.
inline bool strang_close_fused(const gp_handle* h, bool imag) {
  return imag && h->strang && h->dim > 1 && h->seg_c > 0 && !h->pipe_c;
}

// Returns whether the sweep applied the step's closing N(dt/2).
template <typename T>
bool enqueue_sweep(gp_handle* h, bool imag, NormSlots ns, int d, const void* src = nullptr, bool half_open = true) {
  const bool first = d == 0, last = d == h->dim - 1;
  const int mode = imag ? MODE_IMAG : MODE_REAL;
  const int seg = d == 0 ? h->seg_x : h->seg_c;
  const bool fuse_close = last && d > 0 && strang_close_fused(h, imag);
  // with the Strang splitting the norm is taken after the closing N(dt/2)
  const bool read = imag && first && ns.rd >= 0, write = imag && last && (!h->strang || fuse_close);
  const double* parts_in = read ? h->parts[ns.rd] : nullptr;
  double* parts_out = write ? h->parts[ns.wr] : nullptr;
  unsigned blocks = 0;
  const bool fuse_xy = xy_fused(h) && src == nullptr && (d == 0 || d == 1);
  if (fuse_xy && d == 1) return false;  // done by the fused x + y kernel
  if (seg > 0) {
    Sweep2Args<T> a;
    std::memset(&a, 0, sizeof(a));
    a.psi = (c2_t<T>*)h->psi;
    a.src = d == 0 ? (const c2_t<T>*)src : nullptr;
    a.geom = geom_of(h, d);
    const int si = seg_index(seg);
    a.alpha = coef_ptr<T>(h, mode, d, 0);
    a.gf = coef_ptr<T>(h, mode, d, 1 + 2 * si);
    a.gb = coef_ptr<T>(h, mode, d, 2 + 2 * si);
    a.ptab = (const c2_t<T>*)h->ctab[mode][d] + (size_t)si * 512;
    a.cdepth = h->cdepth[mode][d][si];
    a.cpts = h->cpts[mode][d][si];
    set_phase_args<T>(h, imag, (h->strang && half_open) || fuse_close, a);
    a.parts_in = parts_in;
    a.nparts_in = h->parts_n;
    a.parts_wscale = h->parts_ws;
    a.w_axis = (const T*)h->wt[d];
    a.w_a = (const T*)(d == 0 ? h->wt[1] : h->wt[0]);
    a.w_b = (const T*)(d == 2 ? h->wt[1] : h->wt[2]);
    a.parts_out = parts_out;
    // the rho axis of a circular or axial trap: non-symmetric coefficients
    const bool var = h->geom == 2 && d == 0;
    if (var) {
      const c2_t<T>* cv = (const c2_t<T>*)h->cvar[mode];
      a.vab = cv;
      a.vbf = cv + h->n[0];
      a.vh = cv + 2 * h->n[0];
    }
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (fuse_xy) {  // d == 0: the y axis' coefficients beside the x sweep's arguments
        Sweep2Args<float> ay;
        std::memset(&ay, 0, sizeof(ay));
        ay.geom = geom_of(h, 1);
        ay.alpha = coef_ptr<float>(h, mode, 1, 0);
        ay.gf = coef_ptr<float>(h, mode, 1, 1 + 2 * si);
        ay.gb = coef_ptr<float>(h, mode, 1, 2 + 2 * si);
        ay.ptab = (const float2*)h->ctab[mode][1] + (size_t)si * 512;
        ay.cdepth = h->cdepth[mode][1][si];
        ay.cpts = h->cpts[mode][1][si];
        blocks = imag ? launch_xy_seg<true>(seg, a, ay, h->work, h->pdl_now)
                      : launch_xy_seg<false>(seg, a, ay, h->work, h->pdl_now);
        done = true;
      }
    }
    if (var) {
      if (h->tile_x) {  // axial trap: x is not the last axis
        blocks = imag ? launch_t_seg<T, true, true, false, false, true>(seg, a, h->work, h->pdl_now)
                      : launch_t_seg<T, false, true, false, false, true>(seg, a, h->work, h->pdl_now);
      } else if (imag) {
        blocks = write ? launch_x_seg<T, true, true, true, true>(seg, a, h->work, h->pdl_now)
                       : launch_x_seg<T, true, true, false, true>(seg, a, h->work, h->pdl_now);
      } else {
        blocks = launch_x_seg<T, false, true, false, true>(seg, a, h->work, h->pdl_now);
      }
      done = true;
    }
    if constexpr (std::is_same<T, float>::value) {
      if (!done && d == 0 && h->tma_x && src == nullptr && !var) {
        blocks = seg == 8 ? (imag ? launch_tx<true, 8>(h, a, mode, h->work, h->pdl_now)
                                  : launch_tx<false, 8>(h, a, mode, h->work, h->pdl_now))
                          : (imag ? launch_tx<true, 16>(h, a, mode, h->work, h->pdl_now)
                                  : launch_tx<false, 16>(h, a, mode, h->work, h->pdl_now));
        done = true;
      }
      if (!done && d > 0 && h->tma_c) {
        if (fuse_close) blocks = launch_tc_seg<true, true, true>(h, seg, a, h->work, h->pdl_now);
        else if (imag) blocks = write ? launch_tc_seg<true, true>(h, seg, a, h->work, h->pdl_now)
                                      : launch_tc_seg<true, false>(h, seg, a, h->work, h->pdl_now);
        else blocks = launch_tc_seg<false, false>(h, seg, a, h->work, h->pdl_now);
        done = true;
      }
    }
    if constexpr (!is_df<T>::value) {  // pipelined shapes: FP32 and FP64 states only
      if (done) {
      } else if (d == 0 && h->tile_x && h->pipe_x) {
        if (imag) {
          blocks = write ? launch_p_seg<T, true, true, true, true>(seg, a, h->work, h->pdl_now)
                        : launch_p_seg<T, true, true, false, true>(seg, a, h->work, h->pdl_now);
        } else {
          blocks = launch_p_seg<T, false, true, false, true>(seg, a, h->work, h->pdl_now);
        }
        done = true;
      } else if (d > 0 && h->pipe_c) {
        if (imag) {
          blocks = write ? launch_p_seg<T, true, false, true, false>(seg, a, h->work, h->pdl_now)
                        : launch_p_seg<T, true, false, false, false>(seg, a, h->work, h->pdl_now);
        } else {
          blocks = launch_p_seg<T, false, false, false, false>(seg, a, h->work, h->pdl_now);
        }
        done = true;
      }
    }
    if (done) {
    } else if (d == 0 && h->tile_x) {
      if (imag) {
        blocks = write ? launch_t_seg<T, true, true, true>(seg, a, h->work, h->pdl_now)
                      : launch_t_seg<T, true, true, false>(seg, a, h->work, h->pdl_now);
      } else {
        blocks = launch_t_seg<T, false, true, false>(seg, a, h->work, h->pdl_now);
      }
    } else if (d == 0) {
      if (imag) {
        blocks = write ? launch_x_seg<T, true, true, true>(seg, a, h->work, h->pdl_now)
                      : launch_x_seg<T, true, true, false>(seg, a, h->work, h->pdl_now);
      } else {
        blocks = launch_x_seg<T, false, true, false>(seg, a, h->work, h->pdl_now);
      }
    } else {
      if (fuse_close) {
        blocks = launch_c_seg<T, true, true, false, true>(seg, h->keep_c, a, h->work, h->pdl_now);
      } else if (imag) {
        blocks = write ? launch_c_seg<T, true, true>(seg, h->keep_c, a, h->work, h->pdl_now)
                      : launch_c_seg<T, true, false>(seg, h->keep_c, a, h->work, h->pdl_now);
      } else {
        blocks = launch_c_seg<T, false, false>(seg, h->keep_c, a, h->work, h->pdl_now);
      }
    }
    if (write) {
      h->parts_n = (int)blocks;
      h->parts_ws = h->wscale;  // Simpson coefficients: the factor prod dx/3 is still to come
    }
    return fuse_close;
  }
  if constexpr (is_df<T>::value) {
    return false;  // the double-float form needs the segmented kernels (checked at gp_init)
  } else {
  SweepArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.psi = (c2_t<T>*)h->psi;
  a.geom = geom_of(h, d);
  a.m = (const c2_t<T>*)h->cm[imag][d];
  a.cp = (const c2_t<T>*)h->ccp[imag][d];
  a.beta = (T)(h->dt / (4.0 * h->dx[d] * h->dx[d]));
  set_phase_args<T>(h, imag, h->strang && half_open, a);
  a.parts_in = parts_in;
  a.nparts_in = h->parts_n;
  a.parts_wscale = h->parts_ws;
  a.w_axis = h->wd[d];
  a.w_a = d == 0 ? h->wd[1] : h->wd[0];
  a.w_b = d == 2 ? h->wd[1] : h->wd[2];
  a.parts_out = parts_out;
  if (imag) {
    if (first && write) blocks = launch_legacy<T, true, true, true>(a, h->work);
    else if (first) blocks = launch_legacy<T, true, true, false>(a, h->work);
    else if (write) blocks = launch_legacy<T, true, false, true>(a, h->work);
    else blocks = launch_legacy<T, true, false, false>(a, h->work);
  } else {
    if (first) blocks = launch_legacy<T, false, true, false>(a, h->work);
    else blocks = launch_legacy<T, false, false, false>(a, h->work);
  }
  if (write) {
    h->parts_n = (int)blocks;
    h->parts_ws = 1.0;  // FP64 Simpson weights: the sums are complete
  }
  return false;
  }
}

// A real imaginary-time state (h->rpsi, np values of T; imaginary-time maps
// keep a real state real): the x sweep packs two real lines per tile column,
// the y/z sweeps view the array as complex with nx/2 points per row (x = 2i'
// as re, 2i' + 1 as im).  Half the bytes and half the arithmetic of the
// complex state, the same operations on the real parts.
template <typename T>
void enqueue_sweep_real(gp_handle* h, NormSlots ns, int d) {
  if constexpr (!is_df<T>::value) {
    const bool first = d == 0, last = d == h->dim - 1;
    const int seg = d == 0 ? h->seg_x : h->seg_c;
    const bool read = first && ns.rd >= 0, write = last;
    Sweep2Args<T> a;
    std::memset(&a, 0, sizeof(a));
    a.psi = (c2_t<T>*)h->rpsi;
    LineGeom g = geom_of(h, d);
    if (d > 0) {
      g.nx /= 2;
      g.stride = d == 1 ? g.nx : (long)g.nx * g.ny;
      g.nlines = h->np / 2 / g.n;
    }
    a.geom = g;
    const int si = seg_index(seg);
    a.alpha = coef_ptr<T>(h, MODE_IMAG, d, 0);
    a.gf = coef_ptr<T>(h, MODE_IMAG, d, 1 + 2 * si);
    a.gb = coef_ptr<T>(h, MODE_IMAG, d, 2 + 2 * si);
    a.ptab = (const c2_t<T>*)h->ctab[MODE_IMAG][d] + (size_t)si * 512;
    a.cdepth = h->cdepth[MODE_IMAG][d][si];
    a.cpts = h->cpts[MODE_IMAG][d][si];
    set_phase_args<T>(h, true, false, a);
    a.parts_in = read ? h->parts[ns.rd] : nullptr;
    a.nparts_in = h->parts_n;
    a.parts_wscale = h->parts_ws;
    a.w_axis = (const T*)h->wt[d];
    a.w_a = (const T*)(d == 0 ? h->wt[1] : h->wt[0]);
    a.w_b = (const T*)(d == 2 ? h->wt[1] : h->wt[2]);
    a.parts_out = write ? h->parts[ns.wr] : nullptr;
    unsigned blocks;
    if (d == 0)
      blocks = launch_t_seg<T, true, true, false, true>(seg, a, h->work, h->pdl_now);
    else if (write)
      blocks = launch_c_seg<T, true, true, true>(seg, h->keep_c, a, h->work, h->pdl_now);
    else
      blocks = launch_c_seg<T, true, false>(seg, h->keep_c, a, h->work, h->pdl_now);
    if (write) {
      h->parts_n = (int)blocks;
      h->parts_ws = h->wscale;
    }
  }
}

// The closing N(dt/2) of a Strang step (and, imaginary time, the norm sums of
// its result into slot ns.wr).
template <typename T>
void enqueue_strang_close(gp_handle* h, bool imag, NormSlots ns) {
  Sweep2Args<T> a;
  std::memset(&a, 0, sizeof(a));
  a.psi = (c2_t<T>*)h->psi;
  a.geom = geom_of(h, 0);
  set_phase_args<T>(h, imag, true, a);
  a.w_axis = (const T*)h->wt[0];
  a.w_a = (const T*)h->wt[1];
  a.w_b = (const T*)h->wt[2];
  const long chunks = (long)((a.geom.nx + 31) / 32) * a.geom.nlines;
  const long per_block = 8L * kStrangUnroll;  // 8 warps
  const unsigned blocks = (unsigned)std::min<long>((chunks + per_block - 1) / per_block, 152L * 8);
  if (imag) {
    a.parts_out = h->parts[ns.wr];
    launch_k(h->pdl_now, strang_phase_kernel<T, true, true>, dim3(blocks), dim3(256), 0, h->work, a);
    h->parts_n = (int)blocks;
    h->parts_ws = h->wscale;
  } else {
    launch_k(h->pdl_now, strang_phase_kernel<T, false, false>, dim3(blocks), dim3(256), 0, h->work, a);
  }
  count_launch();
}

// One step; with src != nullptr the x sweep reads the step's input from src
// (segmented kernels only) and every sweep writes h->psi.
template <typename T>
void enqueue_step(gp_handle* h, bool imag, NormSlots ns, cudaEvent_t* ev = nullptr, const void* src = nullptr,
                  StepForm f = StepForm{}) {
  bool closed = false;
  for (int d = 0; d < h->dim; ++d) {
    if (ev) cudaEventRecord(ev[2 * d], h->work);
    if (h->real_mode)
      enqueue_sweep_real<T>(h, ns, d);  // imaginary time only
    else
      closed = enqueue_sweep<T>(h, imag, ns, d, src, f.half_open) || closed;
    if (ev) cudaEventRecord(ev[2 * d + 1], h->work);
  }
  if (h->strang && f.close && !closed) enqueue_strang_close<T>(h, imag, ns);
}

inline NormSlots slots_of_step(bool imag, long t) {
  NormSlots ns;
  if (imag) {
    ns.rd = t > 0 ? (int)((t - 1) & 1) : -1;
    ns.wr = (int)(t & 1);
  }
  return ns;
}

// The renormalisation left pending after the last of nsteps imaginary-time steps.
template <typename T>
void enqueue_finish_imag(gp_handle* h, long nsteps) {
  const int blocks = (int)std::min<long>((h->np + 255) / 256, 152L * 8);
  // (a real state: its np values scaled as np/2 complex ones)
  c2_t<T>* psi = (c2_t<T>*)(h->real_mode ? h->rpsi : h->psi);
  launch_k(h->pdl_now, scale_kernel<T>, dim3(blocks), dim3(256), 0, h->work, psi, h->real_mode ? h->np / 2 : h->np,
           (const double*)h->parts[(nsteps - 1) & 1], h->parts_n, h->parts_ws);
  count_launch();
}

// Step 0 eagerly (imaginary time: it has no pending factor; real-time Strang:
// it opens with N(dt/2)), then blocks of kGraphSteps steps replayed from one
// captured graph (a block starts at an odd step in imaginary time, so its
// slot pattern is always the same), then the rest.
template <typename T>
int run_steps_t(gp_handle* h, bool imag, long nsteps) {
  if (nsteps == 0) return GP_OK;
  int rc = join_in(h);
  if (rc) return rc;
  // consecutive sweeps overlap their launch and prologue (FP32 and
  // double-float; the FP64 form, bound by its FP64 pipe, was measured 10 %
  // slower with it)
  struct PdlScope {
    gp_handle* h;
    explicit PdlScope(gp_handle* hh) : h(hh) { h->pdl_now = pdl_enabled() && h->prec != GP_F64; }
    ~PdlScope() { h->pdl_now = false; }
  } pdl_scope(h);
  // real-time Strang: the halves between steps merged (StepForm)
  const bool merged = h->strang && !imag;
  const StepForm first_f{true, !merged}, next_f{!merged, !merged};
  long t = 0;
  if (imag || merged) enqueue_step<T>(h, imag, slots_of_step(imag, t++), nullptr, nullptr, first_f);
  if (nsteps - t >= 2 * kGraphSteps) {
    cudaGraphExec_t& ge = h->graph[imag ? 1 : 0];
    if (!ge) {
      cudaGraph_t graph;
      GP_CUDA(cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal));
      const unsigned long long before = g_launches.load();
      for (int s = 0; s < kGraphSteps; ++s)
        enqueue_step<T>(h, imag, slots_of_step(imag, t + s), nullptr, nullptr, next_f);
      g_launches.store(before);  // capturing launches nothing
      GP_CUDA(cudaStreamEndCapture(h->work, &graph));
      cudaError_t e = cudaGraphInstantiate(&ge, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        ge = nullptr;
        return fail(GP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
    }
    for (; nsteps - t >= kGraphSteps; t += kGraphSteps) {
      GP_CUDA(cudaGraphLaunch(ge, h->work));
      count_launch((unsigned long long)kGraphSteps * (h->dim - (xy_fused(h) ? 1 : 0) +
                                                      (next_f.close && h->strang && !strang_close_fused(h, imag) ? 1 : 0)));
    }
  }
  for (; t < nsteps; ++t) enqueue_step<T>(h, imag, slots_of_step(imag, t), nullptr, nullptr, next_f);
  if (merged) enqueue_strang_close<T>(h, false, NormSlots{});
  if (imag) enqueue_finish_imag<T>(h, nsteps);
  GP_CUDA(cudaGetLastError());
  return join_out(h);
}

// Eager steps with an event pair around every sweep launch (recorded on the
// library's stream, read once at the end); returns the mean duration of each
// axis' sweep kernel in ms_out[axis].
template <typename T>
int time_steps_t(gp_handle* h, bool imag, long nsteps, double* ms_out) {
  std::vector<cudaEvent_t> ev((size_t)nsteps * 2 * h->dim);
  for (auto& e : ev) GP_CUDA(cudaEventCreate(&e));
  int rc = join_in(h);
  for (long t = 0; t < nsteps && !rc; ++t)
    enqueue_step<T>(h, imag, slots_of_step(imag, t), ev.data() + (size_t)t * 2 * h->dim);
  if (imag && !rc && nsteps > 0) enqueue_finish_imag<T>(h, nsteps);
  cudaError_t e = cudaStreamSynchronize(h->work);
  if (!rc && e != cudaSuccess) rc = fail(GP_ERR_CUDA, std::string("gp_time_sweeps: ") + cudaGetErrorString(e));
  double acc[3] = {0, 0, 0};
  for (long t = 0; t < nsteps && !rc; ++t)
    for (int d = 0; d < h->dim; ++d) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[(size_t)t * 2 * h->dim + 2 * d], ev[(size_t)t * 2 * h->dim + 2 * d + 1]);
      acc[d] += ms;
    }
  for (auto& ee : ev) cudaEventDestroy(ee);
  if (rc) return rc;
  for (int d = 0; d < 3; ++d) ms_out[d] = (d < h->dim && nsteps > 0) ? acc[d] / nsteps : 0.0;
  GP_CUDA(cudaGetLastError());
  return join_out(h);
}

// Each axis' sweep (the x sweep with N, or the fused x + y kernel; the y/z
// sweeps, the last with its norm) launched reps times back to back inside a
// captured graph -- programmatic edges as in the step graph -- and the
// replay timed with events on the library's stream: ms_out[d] = mean
// duration per launch as the kernel runs inside a step's graph (0 for an axis
// that has no launch of its own).  Two eager steps first give the norm slots
// valid contents; the caller restores the state.
template <typename T>
int time_sweeps_graph_t(gp_handle* h, bool imag, int reps, double* ms_out) {
  int rc = join_in(h);
  if (rc) return rc;
  for (int d = 0; d < 3; ++d) ms_out[d] = 0.0;
  struct PdlScope {
    gp_handle* h;
    explicit PdlScope(gp_handle* hh) : h(hh) { h->pdl_now = pdl_enabled() && h->prec != GP_F64; }
    ~PdlScope() { h->pdl_now = false; }
  } pdl_scope(h);
  for (long t = 0; t < 2; ++t) enqueue_step<T>(h, imag, slots_of_step(imag, t));
  NormSlots ns;
  if (imag) {
    ns.rd = 1;  // written by step 1 above
    ns.wr = 0;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  for (int d = 0; d < h->dim && !rc; ++d) {
    if (xy_fused(h) && d == 1) continue;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t ge = nullptr;
    const int nparts = h->parts_n;
    const double pws = h->parts_ws;
    cudaError_t e = cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal);
    const unsigned long long before = g_launches.load();
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      if (h->real_mode) enqueue_sweep_real<T>(h, ns, d);
      else enqueue_sweep<T>(h, imag, ns, d);
      h->parts_n = nparts;  // every x launch reads the slot step 1 wrote
      h->parts_ws = pws;
    }
    g_launches.store(before);
    if (e == cudaSuccess) e = cudaStreamEndCapture(h->work, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->work);  // warm-up replay
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->work);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, h->work);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->work);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (ge) cudaGraphExecDestroy(ge);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) rc = fail(GP_ERR_CUDA, std::string("gp_time_sweeps_graph: ") + cudaGetErrorString(e));
    else ms_out[d] = ms / reps;
    count_launch(2ull * reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  GP_CUDA(cudaGetLastError());
  return join_out(h);
}

template <typename T>
int run_observables_t(gp_handle* h, double* dens_dev, double* sums_out = nullptr) {
  ObsArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.psi = (const c2_t<T>*)h->psi;
  a.dim = h->dim;
  a.nx = axis_len(h, 0);
  a.ny = axis_len(h, 1);
  a.nz = axis_len(h, 2);
  a.hx = h->dx[0];
  a.hy = h->dx[1];
  a.hz = h->dx[2];
  a.V = h->Vd;
  if constexpr (std::is_same<T, float>::value) {  // tables in the state precision
    for (int d = 0; d < 3; ++d) {
      (d == 0 ? a.vx : d == 1 ? a.vy : a.vz) = (const float*)h->vt[d];
      (d == 0 ? a.cx : d == 1 ? a.cy : a.cz) = (const float*)h->ct[d];
      (d == 0 ? a.wx : d == 1 ? a.wy : a.wz) = (const float*)h->wt[d];  // Simpson coefficients
    }
    a.wscale = h->wscale;
  } else {
    a.vx = h->vd[0]; a.vy = h->vd[1]; a.vz = h->vd[2];
    a.cx = h->cdx[0]; a.cy = h->cdx[1]; a.cz = h->cdx[2];
    a.wx = h->wd[0]; a.wy = h->wd[1]; a.wz = h->wd[2];
    a.wscale = 1.0;
  }
  if (h->geom == 1) {
    a.gx = (const obs_r<T>*)h->gw_o;
    a.x0 = 1;
  }
  if (h->geom == 2) a.x0 = 2;
  a.density = dens_dev;
  a.partials = h->partials;
  a.counter = h->counter;
  a.out = sums_out ? sums_out : h->obs_out;
  launch_observables<T>(a, h->work, pdl_enabled() && h->prec != GP_F64);
  count_launch();
  GP_CUDA(cudaGetLastError());
  return GP_OK;
}

// ---------------------------------------------------------------- adjoint
// Sweep of the adjoint state along axis d with the dt -> -dt coefficients
// (the conjugate-transposed Crank-Nicolson map).
template <typename T>
void enqueue_adj_sweep(gp_handle* h, int d) {
  Sweep2Args<T> a;
  std::memset(&a, 0, sizeof(a));
  a.psi = (c2_t<T>*)h->adj_lam;
  a.geom = geom_of(h, d);
  const int seg = d == 0 ? h->seg_x : h->seg_c;
  const int si = seg_index(seg);
  a.alpha = coef_ptr<T>(h, MODE_REAL_ADJ, d, 0);
  a.gf = coef_ptr<T>(h, MODE_REAL_ADJ, d, 1 + 2 * si);
  a.gb = coef_ptr<T>(h, MODE_REAL_ADJ, d, 2 + 2 * si);
  a.ptab = (const c2_t<T>*)h->ctab[MODE_REAL_ADJ][d] + (size_t)si * 512;
  a.cdepth = h->cdepth[MODE_REAL_ADJ][d][si];
  a.cpts = h->cpts[MODE_REAL_ADJ][d][si];
  if (d == 0 && h->tile_x && h->pipe_x) launch_p_seg<T, false, false, false, true>(seg, a, h->work, h->pdl_now);
  else if (d == 0 && h->tile_x) launch_t_seg<T, false, false, false>(seg, a, h->work, h->pdl_now);
  else if (d == 0) launch_x_seg<T, false, false, false>(seg, a, h->work, h->pdl_now);
  else if (h->pipe_c) launch_p_seg<T, false, false, false, false>(seg, a, h->work, h->pdl_now);
  else launch_c_seg<T, false, false>(seg, h->keep_c, a, h->work, h->pdl_now);
}

template <typename T>
void enqueue_adj_phase(gp_handle* h, const void* phi) {
  AdjPhaseArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.phi = (const c2_t<T>*)phi;
  a.lam = (c2_t<T>*)h->adj_lam;
  a.np = h->np;
  a.nx = axis_len(h, 0);
  a.ny = axis_len(h, 1);
  a.V = (const T*)h->Vt;
  a.vx = (const T*)h->vt[0];
  a.vy = (const T*)h->vt[1];
  a.vz = (const T*)h->vt[2];
  a.dt = (T)h->adj_dt;
  a.g = (T)h->adj_g;
  a.dJdV = h->adj_dJdV;
  a.partials = h->partials;
  a.counter = h->counter;
  a.dJdg = h->adj_dJdg;
  const int blocks = (int)std::min<long>((h->np + 255) / 256, 152L * 16);
  adjoint_phase_kernel<T><<<blocks, 256, 0, h->work>>>(a);
  count_launch();
}

// Forward run of nsteps real-time steps from the current state, keeping the
// state at steps 0, K, 2K, ... (buffers sized by the caller of this function).
template <typename T>
int adjoint_forward_t(gp_handle* h, long nsteps, int K) {
  const long nck = (nsteps + K - 1) / K;
  for (long c = 0; c < nck; ++c) {
    int rc = join_in(h);
    if (rc) return rc;
    GP_CUDA(cudaMemcpyAsync((char*)h->adj_ckpt + (size_t)c * h->np * h->esize, h->psi, (size_t)h->np * h->esize,
                            cudaMemcpyDeviceToDevice, h->work));
    if ((rc = join_out(h))) return rc;
    if ((rc = run_steps_t<T>(h, false, std::min<long>(K, nsteps - c * K)))) return rc;
  }
  return GP_OK;
}

// Reverse pass: h->adj_lam holds lambda(T) on entry and lambda(0) on exit;
// h->adj_dJdV (when dJdV_dev is null) or dJdV_dev receives dJ/dV, h->adj_dJdg
// dJ/dg.  Each checkpoint segment is recomputed forward into the trajectory
// buffer (the x sweep reads step j and writes step j+1), then walked back.
template <typename T>
int adjoint_backward_t(gp_handle* h, double* dJdV_dev, void* lam0_dev) {
  const long nsteps = h->adj_nsteps;
  const int K = h->adj_K;
  const long nck = (nsteps + K - 1) / K;
  const size_t sbytes = (size_t)h->np * h->esize;
  double* dJdV_keep = h->adj_dJdV;
  if (dJdV_dev) h->adj_dJdV = dJdV_dev;
  int rc = join_in(h);
  if (rc) return rc;
  GP_CUDA(cudaMemsetAsync(h->adj_dJdV, 0, (size_t)h->np * sizeof(double), h->work));
  GP_CUDA(cudaMemsetAsync(h->adj_dJdg, 0, sizeof(double), h->work));
  void* psi_saved = h->psi;
  const double g_now = h->g, dt_now = h->dt;
  h->g = h->adj_g;  // the forward's g and dt drive the recomputation
  h->dt = h->adj_dt;
  for (long c = nck - 1; c >= 0; --c) {
    const long t0 = c * K;
    const int len = (int)std::min<long>(K, nsteps - t0);
    char* traj = (char*)h->adj_traj;
    cudaMemcpyAsync(traj, (const char*)h->adj_ckpt + (size_t)c * sbytes, sbytes, cudaMemcpyDeviceToDevice, h->work);
    for (int j = 0; j + 1 < len; ++j) {
      h->psi = traj + (size_t)(j + 1) * sbytes;
      enqueue_step<T>(h, false, NormSlots{}, nullptr, traj + (size_t)j * sbytes);
    }
    for (int j = len - 1; j >= 0; --j) {
      for (int d = h->dim - 1; d >= 0; --d) enqueue_adj_sweep<T>(h, d);
      enqueue_adj_phase<T>(h, traj + (size_t)j * sbytes);
    }
  }
  h->psi = psi_saved;
  h->g = g_now;
  h->dt = dt_now;
  h->adj_dJdV = dJdV_keep;
  if (lam0_dev) cudaMemcpyAsync(lam0_dev, h->adj_lam, sbytes, cudaMemcpyDeviceToDevice, h->work);
  GP_CUDA(cudaGetLastError());
  return join_out(h);
}

}  // namespace gpe
