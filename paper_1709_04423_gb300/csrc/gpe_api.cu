// gpe_api.cu -- C ABI of the GB300 split-step Crank-Nicolson GP propagator
// (declared and documented in include/gpe.h).
//
// Host side of the library: argument validation, device memory owned by the
// handle, the time-invariant elimination coefficients (Thomas factors of the
// Crank-Nicolson systems and the segment products the segmented sweeps use),
// the choice of kernel shapes, and the observables reduction.  The per-step
// launch sequence lives in gpe_step.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gpe_df.cuh"
#include "gpe_internal.h"

using cd = std::complex<double>;

namespace gpe {

thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};

// ---- guarded allocations and the checking build's readers
namespace {
#ifdef GPE_BOUNDS_CHECK
constexpr size_t kGuard = 64 * 1024;  // bytes of 0xFF before and after every buffer
std::mutex g_guard_mutex;
std::map<void*, std::pair<char*, size_t>>& guard_map() {  // user pointer -> (raw pointer, bytes)
  static std::map<void*, std::pair<char*, size_t>> m;
  return m;
}
#endif
std::mutex g_reader_mutex;
std::vector<int (*)()>& check_readers() {
  static std::vector<int (*)()> v;
  return v;
}
}  // namespace

void register_check_reader(int (*reader)()) {
  std::lock_guard<std::mutex> lock(g_reader_mutex);
  check_readers().push_back(reader);
}

cudaError_t guarded_malloc(void** p, size_t bytes) {
#ifdef GPE_BOUNDS_CHECK
  char* raw = nullptr;
  cudaError_t e = cudaMalloc((void**)&raw, bytes + 2 * kGuard);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemset(raw, 0xFF, kGuard)) == cudaSuccess) e = cudaMemset(raw + kGuard + bytes, 0xFF, kGuard);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(raw);
    return e;
  }
  *p = raw + kGuard;
  std::lock_guard<std::mutex> lock(g_guard_mutex);
  guard_map()[*p] = {raw, bytes};
  return cudaSuccess;
#else
  return cudaMalloc(p, bytes);
#endif
}

void guarded_free(void* p) {
  if (!p) return;
#ifdef GPE_BOUNDS_CHECK
  std::lock_guard<std::mutex> lock(g_guard_mutex);
  auto it = guard_map().find(p);
  if (it != guard_map().end()) {
    cudaFree(it->second.first);
    guard_map().erase(it);
    return;
  }
#endif
  cudaFree(p);
}

int dev_alloc(gp_handle* h, void** p, size_t bytes) {
  const size_t b = bytes < 16 ? 16 : bytes;
  GP_CUDA(guarded_malloc(p, b));
  h->allocs.push_back(*p);
  GP_CUDA(cudaMemsetAsync(*p, 0, b, h->work));
  return GP_OK;
}

int join_in(gp_handle* h) {
  GP_CUDA(cudaEventRecord(h->ev_in, h->user));
  GP_CUDA(cudaStreamWaitEvent(h->work, h->ev_in, 0));
  return GP_OK;
}

int join_out(gp_handle* h) {
  GP_CUDA(cudaEventRecord(h->ev_out, h->work));
  GP_CUDA(cudaStreamWaitEvent(h->user, h->ev_out, 0));
  return GP_OK;
}

void drop_graphs(gp_handle* h) {
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
}

// Crank-Nicolson system (1 + A) with A = r T along one axis: a = -r (off
// diagonals), b = 1 + 2r, r = i beta (real time) or beta (imaginary time),
// beta = dt/(4 dx^2).  Thomas factors m_k = 1/(b - a c'_{k-1}), c'_k = a m_k
// for the interior k = 1..n-2, and alpha_k = r m_k (= -c'_k).
AxisFactors thomas_factors(int n, double beta, bool imag) {
  AxisFactors f;
  f.m.assign(n, cd(0, 0));
  f.cp.assign(n, cd(0, 0));
  f.alpha.assign(n, cd(0, 0));
  const cd r = imag ? cd(beta, 0) : cd(0, beta);
  const cd a = -r, b = 1.0 + 2.0 * r;
  cd cprev(0, 0);
  for (int k = 1; k <= n - 2; ++k) {
    const cd den = b - a * cprev;
    f.m[k] = 1.0 / den;
    f.cp[k] = a * f.m[k];
    f.alpha[k] = r * f.m[k];
    cprev = f.cp[k];
  }
  return f;
}

// Grid coordinate i of axis d (n points, spacing dx): Cartesian (R1)
// -n dx/2 + i dx; the spherical trap's r = i dr; the rho axis of a circular
// or axial trap (i - 1/2) drho (point 0 the mirror image of point 1).
double axis_coord(int geom, int d, int n, double dx, int i) {
  if (geom == 1) return i * dx;
  if (geom == 2 && d == 0) return (i - 0.5) * dx;
  return -0.5 * n * dx + i * dx;
}

// The rho axis of a circular or axial trap (geom 2): row k of T is
// (-(1 - h_k), 2, -(1 + h_k)) with h_k = drho/(2 rho_k) = 1/(2k - 1) on
// rho_k = (k - 1/2) drho.  Thomas factors of (1 + rT): m_k = 1/(b - a_k
// c'_{k-1}) with a_k = -r(1 - h_k), c_k = -r(1 + h_k), c'_k = c_k m_k; the
// increment form's forward recurrence e_k = af_k e_{k-1} + 2 r m_k lapv_k and
// backward recurrence z_k = e_k + ab_k z_{k+1} have af_k = r(1 - h_k) m_k,
// ab_k = r(1 + h_k) m_k; the sweeps carry them at half scale, so bf_k =
// r m_k (half of 2 r m_k, exactly); hh_k = (1 - h_k, 1 + h_k).
static void rho_factors(int n, double beta, bool imag, std::vector<cd>& af, std::vector<cd>& ab, std::vector<cd>& bf,
                 std::vector<cd>& hh) {
  af.assign(n, cd(0, 0));
  ab.assign(n, cd(0, 0));
  bf.assign(n, cd(0, 0));
  hh.assign(n, cd(0, 0));
  const cd r = imag ? cd(beta, 0) : cd(0, beta);
  const cd b = 1.0 + 2.0 * r;
  cd cprev(0, 0);
  for (int k = 1; k <= n - 2; ++k) {
    const double h = 1.0 / (2.0 * k - 1.0);
    const cd a = -r * (1.0 - h), c = -r * (1.0 + h);
    const cd m = 1.0 / (b - a * cprev);
    af[k] = r * (1.0 - h) * m;
    ab[k] = r * (1.0 + h) * m;
    bf[k] = r * m;
    hh[k] = cd(1.0 - h, 1.0 + h);
    cprev = c * m;
  }
}

// Segment products for segments of `seg` interior points starting at k = 1:
// gf[k] = prod_{i=start..k} af_i, gb[k] = prod_{i=k..end} ab_i.
void segment_products(const std::vector<cd>& alpha, int n, int seg, std::vector<cd>& gf, std::vector<cd>& gb) {
  segment_products(alpha, alpha, n, seg, gf, gb);
}

void segment_products(const std::vector<cd>& af, const std::vector<cd>& ab, int n, int seg, std::vector<cd>& gf,
                      std::vector<cd>& gb, int first) {
  const int last = first == 0 ? n - 1 : n - 2;  // even-aligned segments also cover the two end points
  gf.assign(n, cd(0, 0));
  gb.assign(n, cd(0, 0));
  for (int k0 = first; k0 <= last; k0 += seg) {
    const int k1 = std::min(last, k0 + seg - 1);
    cd acc(1, 0);
    for (int k = k0; k <= k1; ++k) {
      acc *= af[k];
      gf[k] = acc;
    }
    acc = cd(1, 0);
    for (int k = k1; k >= k0; --k) {
      acc *= ab[k];
      gb[k] = acc;
    }
  }
}

// Carry tables of the segment scans for segment length sg: with A_q (B_q)
// the product of af (ab) over segment q, Pf[q][t] = prod_{q<r<=t} A_r (q <= t)
// and Pb[q][t] = prod_{t<=r<q} B_r (q >= t); 16 x 16 each, Pf then Pb.
void carry_tables(const std::vector<cd>& alpha, int n, int sg, cd* out /* 512 */) {
  carry_tables(alpha, alpha, n, sg, out);
}

void carry_tables(const std::vector<cd>& af, const std::vector<cd>& ab, int n, int sg, cd* out /* 512 */, int first) {
  const int last = first == 0 ? n - 1 : n - 2;
  cd Aseg[16], Bseg[16];
  for (int q = 0; q < 16; ++q) {
    cd acc(1, 0), bcc(1, 0);
    for (int k = first + q * sg; k <= std::min(last, first + (q + 1) * sg - 1); ++k) {
      acc *= af[k];
      bcc *= ab[k];
    }
    Aseg[q] = acc;
    Bseg[q] = bcc;
  }
  cd* Pf = out;
  cd* Pb = out + 256;
  for (int q = 0; q < 16; ++q)
    for (int t = 0; t < 16; ++t) {
      cd acc(1, 0);
      Pf[q * 16 + t] = cd(0, 0);
      Pb[q * 16 + t] = cd(0, 0);
      if (q <= t) {
        for (int r = q + 1; r <= t; ++r) acc *= Aseg[r];
        Pf[q * 16 + t] = acc;
      }
      acc = cd(1, 0);
      if (q >= t) {
        for (int r = t; r < q; ++r) acc *= Bseg[r];
        Pb[q * 16 + t] = acc;
      }
    }
}

int carry_pts_class(int pts) { return pts <= 4 ? 4 : pts <= 8 ? 8 : pts <= 12 ? 12 : 0; }

void carry_reach(const cd* gf, const cd* gb, const cd* tabs, int n, int sg, int first, double tau, int& depth,
                 int& pts) {
  const int last = first == 0 ? n - 1 : n - 2;
  const int nall = (last - first + 1 + sg - 1) / sg;  // every segment (a warp-per-line sweep has up to 32)
  const int nseg = std::min(16, nall);                // those of the 16 x 16 carry tables
  pts = 1;
  for (int q = 0; q < nall; ++q) {
    const int k0 = first + q * sg, kend = std::min(last, k0 + sg - 1), jend = kend - k0 + 1;
    for (int k = k0; k <= kend; ++k) {
      const int j = k - k0;
      if (std::abs(gf[k]) > tau) pts = std::max(pts, j + 1);
      if (std::abs(gb[k]) > tau) pts = std::max(pts, jend - j);
    }
  }
  const cd* Pf = tabs;
  const cd* Pb = tabs + 256;
  depth = 1;
  for (int a = 0; a < nseg; ++a)
    for (int b = 0; b < nseg; ++b) {
      if (b < a && std::abs(Pf[b * 16 + a - 1]) > tau) depth = std::max(depth, a - b);
      if (b > a && a + 1 < 16 && std::abs(Pb[b * 16 + a + 1]) > tau) depth = std::max(depth, b - a);
    }
}

namespace {

template <typename T>
int upload_c2(gp_handle* h, void* dst, const std::vector<cd>& v) {
  std::vector<T> tmp(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    tmp[2 * i] = (T)v[i].real();
    tmp[2 * i + 1] = (T)v[i].imag();
  }
  GP_CUDA(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  return GP_OK;
}

template <typename T>
int upload_real(gp_handle* h, void* dst, const std::vector<double>& v) {
  std::vector<T> tmp(v.begin(), v.end());
  GP_CUDA(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  return GP_OK;
}

template <typename T>
int upload_coefs_t(gp_handle* h) {
  for (int mode = 0; mode < NUM_MODES; ++mode)
    for (int d = 0; d < h->dim; ++d) {
      const int n = h->n[d];
      const double sign = mode == MODE_REAL_ADJ ? -1.0 : 1.0;
      const double beta = sign * h->dt / (4.0 * h->dx[d] * h->dx[d]);
      const AxisFactors f = thomas_factors(n, beta, mode == MODE_IMAG);
      // forward / backward coefficients: alpha for both, or the rho axis' own
      std::vector<cd> af = f.alpha, ab = f.alpha;
      if (h->geom == 2 && d == 0) {
        std::vector<cd> bf, hh;
        rho_factors(n, beta, mode == MODE_IMAG, af, ab, bf, hh);
        std::vector<cd> cv((size_t)3 * n);
        std::copy(ab.begin(), ab.end(), cv.begin());
        std::copy(bf.begin(), bf.end(), cv.begin() + n);
        std::copy(hh.begin(), hh.end(), cv.begin() + 2 * n);
        int rc = upload_c2<T>(h, h->cvar[mode], cv);
        if (rc) return rc;
      }
      std::vector<cd> all((size_t)(1 + 2 * kNumSegs) * n);
      std::copy(af.begin(), af.end(), all.begin());
      std::vector<cd> gf, gb;
      for (int s = 0; s < kNumSegs; ++s) {
        segment_products(af, ab, n, kSegs[s], gf, gb);
        std::copy(gf.begin(), gf.end(), all.begin() + (size_t)(1 + 2 * s) * n);
        std::copy(gb.begin(), gb.end(), all.begin() + (size_t)(2 + 2 * s) * n);
      }
      std::vector<cd> tabs((size_t)kNumSegs * 512, cd(0, 0));
      for (int si = 0; si < kNumSegs; ++si) carry_tables(af, ab, n, kSegs[si], tabs.data() + (size_t)si * 512);
      // how far the carries reach above the state precision's threshold
      const double tau = std::ldexp(1.0, h->prec == GP_F32 ? -48 : -64);
      for (int si = 0; si < kNumSegs; ++si) {
        int pts = 0;
        carry_reach(all.data() + (size_t)(1 + 2 * si) * n, all.data() + (size_t)(2 + 2 * si) * n,
                    tabs.data() + (size_t)si * 512, n, kSegs[si], 1, tau, h->cdepth[mode][d][si], pts);
        h->cpts[mode][d][si] = carry_pts_class(pts);
      }
      int rc = upload_c2<T>(h, h->coef[mode][d], all);
      if (rc) return rc;
      if ((rc = upload_c2<T>(h, h->ctab[mode][d], tabs))) return rc;
      if (d == 0 && h->coef_even[mode]) {
        // segments aligned to even points (q SEG .. q SEG + SEG - 1, alpha = 0 at both
        // ends) for SEG = 8 and 16: gf, gb, then the carry tables of each
        std::vector<cd> ev((size_t)4 * n + 1024, cd(0, 0));
        for (int si = 0; si < 2; ++si) {
          const int sg = si == 0 ? 8 : 16;
          segment_products(af, ab, n, sg, gf, gb, 0);
          std::copy(gf.begin(), gf.end(), ev.begin() + (size_t)(2 * si) * n);
          std::copy(gb.begin(), gb.end(), ev.begin() + (size_t)(2 * si + 1) * n);
          carry_tables(af, ab, n, sg, ev.data() + (size_t)4 * n + 512 * si, 0);
          // how far a carry reaches above 2^-48 (the TMA x sweep truncates the rest)
          int depth = 1, nj = 1;
          carry_reach(gf.data(), gb.data(), ev.data() + (size_t)4 * n + 512 * si, n, sg, 0, std::ldexp(1.0, -48),
                      depth, nj);
          h->even_nj[mode][si] = nj <= 4 ? 4 : (nj <= 8 ? 8 : sg);
          h->even_depth[mode][si] = depth;
        }
        if ((rc = upload_c2<T>(h, h->coef_even[mode], ev))) return rc;
      }
      if (mode < 2) {
        if ((rc = upload_c2<T>(h, h->cm[mode == MODE_IMAG][d], f.m))) return rc;
        if ((rc = upload_c2<T>(h, h->ccp[mode == MODE_IMAG][d], f.cp))) return rc;
      }
    }
  return GP_OK;
}

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : dflt;
}

}  // namespace

// Kernel shapes.  y/z lines: 32 lines per block, one warp per segment, at
// most 16 segments: seg = smallest of 4, 8, 16, 32 with ceil((n-2)/seg) <= 16.
// x lines in 2d/3d: the shared-memory tile kernel with the same rule; the 1d
// line: one warp per line with 32 * seg_x >= n - 2.  Lines longer than 514
// points use the thread-per-line kernel (shape 0).  GPE_SEG_X, GPE_SEG_YZ and
// GPE_TILE_X override the defaults (used by the autotuner and the shape tests).
// two shared-memory stages of a 32-line tile plus the coefficient tables
// (200 KB of dynamic shared memory leaves room for the kernel's static carry
// buffers within the 227 KB a block may hold)
bool pipe_fits(const gp_handle* h, int n, bool axis0) {
  const long stage = axis0 ? 32L * (n + 1) : (long)n * 33;
  return (3L * n + 512 + 2 * stage) * (long)h->esize <= 200L * 1024;
}

// The fused x + y sweeps (one block per xy plane): FP32 3d Cartesian grids
// with nx, ny <= 128 (four 32-line groups), a segment length of 8, 16 or 32
// for both axes, at most 32 warps, and the plane in dynamic shared memory.
bool plane_fits(const gp_handle* h, int seg) {
  if (h->prec != GP_F32 || h->dim != 3 || h->geom != 0) return false;
  const int nx = h->n[0], ny = h->n[1];
  if (nx > 128 || ny > 128 || (seg != 8 && seg != 16 && seg != 32)) return false;
  const int sx = (nx - 2 + seg - 1) / seg, sy = (ny - 2 + seg - 1) / seg;
  if (sx > 16 || sy > 16) return false;
  if (sx * ((ny + 31) / 32) > 32 || sy * ((nx + 31) / 32) > 32) return false;
  return (3L * nx + 512 + 3L * ny + 512 + (long)ny * (nx + 1)) * 8 <= 180L * 1024;
}

// The TMA y/z sweeps (gpe_tma.cuh): FP32 complex states of 2d/3d grids with
// nx even (the tensor map's row strides are multiples of 16 bytes), y/z lines
// of at most 256 points (a box dimension's limit), a segment length of 8, 16
// or 32 with at most 16 segments per line, and three 32-line stages plus the
// coefficients in shared memory.
bool tma_fits(const gp_handle* h, int seg) {
  if (h->prec != GP_F32 || h->dim < 2 || h->real_mode || (h->n[0] & 1)) return false;
  if (seg != 8 && seg != 16 && seg != 32) return false;
  int nmax = 0;
  for (int d = 1; d < h->dim; ++d) {
    if (h->n[d] > 256 || (h->n[d] - 2 + seg - 1) / seg > 16) return false;
    nmax = std::max(nmax, h->n[d]);
  }
  const long coef = (3L * nmax + 512) * 8;
  const long smem = (coef + 1023) / 1024 * 1024 + 1024 + 3L * 32 * nmax * 8;
  return smem + 9 * 1024 <= 227L * 1024;  // + the static carries and barriers
}

// The TMA x sweep: FP32 complex states of 2d/3d Cartesian grids with nx a
// multiple of 16 (whole 16-point chunks per box) and at most 256, segments of
// 8 or 16 points aligned to even points with at most 16 per line.
bool tma_x_fits(const gp_handle* h, int seg) {
  if (h->prec != GP_F32 || h->dim < 2 || h->real_mode || h->geom != 0 || !h->coef_even[0]) return false;
  const int nx = h->n[0];
  if ((nx & 15) || nx > 256 || (seg != 8 && seg != 16) || nx / seg > 16) return false;
  const long coef = (3L * nx + 512) * 8 + 4L * nx;
  const long smem = (coef + 1023) / 1024 * 1024 + 1024 + 3L * 32 * nx * 8;
  return smem + 17 * 1024 <= 227L * 1024;  // + the static carries, edge points and barriers
}

int read_dev_err(gp_handle* h, const char* who) {
  int e = 0;
  GP_CUDA(cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  if (e == 0) return GP_OK;
  GP_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  return fail(GP_ERR_TIMEOUT, std::string(who) + ": a device-side wait gave up (a sweep's tile transfer did not "
                                                  "complete within the wait limit); the state is not valid");
}

int tile_seg(int M) {
  for (int s : {4, 8, 16, 32})
    if ((M + s - 1) / s <= 16) return s;
  return 0;
}

namespace {

void choose_shapes(gp_handle* h) {
  const int M0 = h->n[0] - 2;
  // the x tile needs (36 n + 512) complex values of shared memory (<= 200 KB)
  const bool tile_fits = (36L * h->n[0] + 512) * (long)h->esize <= 200L * 1024;
  h->tile_x = env_int("GPE_TILE_X", h->dim > 1 && tile_fits ? 1 : 0) != 0 && tile_fits;
  int sx = 0;
  if (h->tile_x) {
    sx = tile_seg(M0);
  } else {
    for (int s : {1, 2, 4, 8, 16})
      if (32 * s >= M0) { sx = s; break; }
  }
  sx = env_int("GPE_SEG_X", sx);
  if (h->tile_x) {
    if (sx < 4 || sx > 32 || seg_index(sx) < 0 || (M0 + sx - 1) / sx > 16) sx = 0;
  } else if (sx > 0 && (seg_index(sx) < 0 || sx > 16 || 32 * sx < M0)) {
    sx = 0;
  }
  if (sx == 0) h->tile_x = false;
  h->seg_x = sx;
  int Mc = 0;
  for (int d = 1; d < h->dim; ++d) Mc = std::max(Mc, h->n[d] - 2);
  int sc = env_int("GPE_SEG_YZ", tile_seg(Mc));
  if (sc > 0 && (seg_index(sc) < 0 || sc < 4 || (Mc + sc - 1) / sc > 16)) sc = 0;
  h->seg_c = sc;
  h->keep_c = env_int("GPE_KEEP", 1) != 0;
  int nmax = 0;
  for (int d = 1; d < h->dim; ++d) nmax = std::max(nmax, h->n[d]);
  const bool pipe = env_int("GPE_PIPE", 0) != 0 && h->prec != GP_DF64;
  h->pipe_x = pipe && h->tile_x && h->geom != 2 && pipe_fits(h, h->n[0], true);  // (no rho-axis pipelined sweep)
  h->xyfuse = env_int("GPE_FUSE_XY", 0) != 0 && plane_fits(h, sx);
  h->pipe_c = pipe && h->dim > 1 && sc > 0 && pipe_fits(h, nmax, false);
}

}  // namespace

int upload_coefs(gp_handle* h) {
  if (h->prec == GP_DF64) return upload_coefs_t<df64>(h);
  return h->prec == GP_F64 ? upload_coefs_t<double>(h) : upload_coefs_t<float>(h);
}

// Step launchers of the handle's state precision.
int run_steps_any(gp_handle* h, bool imag, long nsteps) {
  if (h->prec == GP_DF64) return run_steps_df(h, imag, nsteps);
  return h->prec == GP_F64 ? run_steps_f64(h, imag, nsteps) : run_steps_f32(h, imag, nsteps);
}
int time_steps_any(gp_handle* h, bool imag, long nsteps, double* ms) {
  if (h->prec == GP_DF64) return time_steps_df(h, imag, nsteps, ms);
  return h->prec == GP_F64 ? time_steps_f64(h, imag, nsteps, ms) : time_steps_f32(h, imag, nsteps, ms);
}
int run_observables_any(gp_handle* h, double* dens_dev, double* sums_out) {
  materialize_complex(h);
  if (h->prec == GP_DF64) return run_observables_df(h, dens_dev, sums_out);
  return h->prec == GP_F64 ? run_observables_f64(h, dens_dev, sums_out) : run_observables_f32(h, dens_dev, sums_out);
}

namespace {
// Seven Simpson sums per record -> norm, energy, mu, rms_x, rms_y, rms_z, rms_r
// (the same formulas as gp_observables).
__global__ void series_finish_kernel(const double* __restrict__ S, long nrec, double g, double* __restrict__ out) {
  for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += (long)gridDim.x * blockDim.x) {
    const double* s = S + 8 * r;
    const double N = s[0];
    double* o = out + 7 * r;
    o[0] = N;
    o[1] = (s[1] + s[2]) / N + 0.5 * g * s[3] / (N * N);
    o[2] = (s[1] + s[2]) / N + g * s[3] / (N * N);
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      o[3 + d] = sqrt(s[4 + d] / N);
      r2 += s[4 + d] / N;
    }
    o[6] = sqrt(r2);
  }
}
}  // namespace

namespace {
// Host triple-float images of complex factors (exact splits of the doubles).
int upload_tf(gp_handle* h, void* dst, const std::vector<cd>& v) {
  std::vector<tf3c> tmp(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    tf_split(v[i].real(), tmp[i].re);
    tf_split(v[i].imag(), tmp[i].im);
  }
  GP_CUDA(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(tf3c), cudaMemcpyHostToDevice, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  return GP_OK;
}
}  // namespace

// Per-axis potential factors of the sub-step N for the time step dt_eff
// (absent axes: a single factor 1) into fac[mode][axis] (and, for the
// double-float state, their triple-float images per x index and per x line);
// with a user potential, the per-point ones.
static int upload_factor_set(gp_handle* h, double dt_eff, void* (&fac)[2][3], void* (&tfx)[2], void* (&tfyz)[2],
                             void* (&fV)[2], void* (&tfV)[2]) {
  std::vector<cd> per_axis[2][3];
  for (int d = 0; d < 3; ++d) {
    const int nd = axis_len(h, d);
    std::vector<cd> fr(nd, cd(1, 0)), fi(nd, cd(1, 0));
    if (d < h->dim)
      for (int i = 0; i < nd; ++i) {
        const double x = axis_coord(h->geom, d, nd, h->dx[d], i);
        const double v = 0.5 * h->nkl[d] * h->nkl[d] * x * x;
        fr[i] = cd(std::cos(dt_eff * v), -std::sin(dt_eff * v));
        fi[i] = cd(std::exp(-dt_eff * v), 0.0);
      }
    const bool f64 = h->prec != GP_F32;  // the double-float form keeps FP64 factors too
    int rc = f64 ? upload_c2<double>(h, fac[0][d], fr) : upload_c2<float>(h, fac[0][d], fr);
    if (rc) return rc;
    rc = f64 ? upload_c2<double>(h, fac[1][d], fi) : upload_c2<float>(h, fac[1][d], fi);
    if (rc) return rc;
    per_axis[0][d] = fr;
    per_axis[1][d] = fi;
  }
  if (h->prec == GP_DF64) {
    const int ny = axis_len(h, 1), nz = axis_len(h, 2);
    for (int m = 0; m < 2; ++m) {
      std::vector<cd> yz((size_t)ny * nz);
      for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) yz[(size_t)k * ny + j] = per_axis[m][1][j] * per_axis[m][2][k];
      int rc = upload_tf(h, tfx[m], per_axis[m][0]);
      if (rc) return rc;
      if ((rc = upload_tf(h, tfyz[m], yz))) return rc;
    }
  }
  if (h->Vd) {
    potential_factors(h, dt_eff, fV, tfV);
    GP_CUDA(cudaGetLastError());
  }
  return GP_OK;
}

// The buffers of the dt/2 factors of the Strang splitting (those not yet there).
static int ensure_half_tables(gp_handle* h) {
  int rc = GP_OK;
  for (int m = 0; m < 2; ++m) {
    for (int d = 0; d < 3; ++d)
      if (!h->fac_h[m][d] && (rc = dev_alloc(h, &h->fac_h[m][d], (size_t)axis_len(h, d) * h->esize))) return rc;
    if (h->prec == GP_DF64) {
      const long nyz = (long)axis_len(h, 1) * axis_len(h, 2);
      if (!h->tfx_h[m] && (rc = dev_alloc(h, &h->tfx_h[m], (size_t)h->n[0] * sizeof(tf3c)))) return rc;
      if (!h->tfyz_h[m] && (rc = dev_alloc(h, &h->tfyz_h[m], (size_t)nyz * sizeof(tf3c)))) return rc;
    }
    if (h->Vbuf) {
      if (!h->fV_h[m] && (rc = dev_alloc(h, &h->fV_h[m], (size_t)h->np * h->esize))) return rc;
      if (h->prec == GP_DF64 && !h->tfV_h[m] && (rc = dev_alloc(h, &h->tfV_h[m], (size_t)h->np * sizeof(tf3c))))
        return rc;
    }
  }
  return rc;
}

// The factors for dt and, with the Strang splitting, for dt/2.
int upload_factors(gp_handle* h) {
  int rc = upload_factor_set(h, h->dt, h->fac, h->tfx, h->tfyz, h->fV, h->tfV);
  if (!rc && h->strang) rc = upload_factor_set(h, 0.5 * h->dt, h->fac_h, h->tfx_h, h->tfyz_h, h->fV_h, h->tfV_h);
  return rc;
}

}  // namespace gpe

using namespace gpe;

extern "C" {

const char* gp_last_error(void) { return g_err.c_str(); }

unsigned long long gp_kernel_launches(void) { return g_launches.load(); }

long gp_npoints(const gp_handle* h) { return h ? h->np : 0; }

int gp_precision_of(const gp_handle* h) { return h ? h->prec : -1; }

int gp_destroy(gp_handle* h) {
  if (!h) return GP_OK;
  if (h->work) cudaStreamSynchronize(h->work);
  drop_graphs(h);
  for (void* p : h->allocs) guarded_free(p);
  if (h->obs_host) cudaFreeHost(h->obs_host);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->work) cudaStreamDestroy(h->work);
  delete h;
  return GP_OK;
}

namespace {
int init_handle(gp_handle** out, int geom, int dim, const int n[3], const double dx[3], double dt,
                const double nkl[3], double g, gp_precision prec, void* stream) {
  g_err.clear();
  if (!out || !n || !dx || !nkl) return fail(GP_ERR_INVALID, "gp_init: NULL argument");
  *out = nullptr;
  if (dim < 1 || dim > 3) return fail(GP_ERR_INVALID, "gp_init: dim must be 1, 2 or 3");
  if (prec != GP_F64 && prec != GP_F32 && prec != GP_DF64) return fail(GP_ERR_INVALID, "gp_init: unknown precision");
  long np = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 3) return fail(GP_ERR_INVALID, "gp_init: every axis needs n >= 3 points");
    if (!(dx[d] > 0.0) || !std::isfinite(dx[d])) return fail(GP_ERR_INVALID, "gp_init: dx must be finite and > 0");
    if (!std::isfinite(nkl[d])) return fail(GP_ERR_INVALID, "gp_init: trap frequencies must be finite");
    np *= n[d];
    if (np > 2147483647L) return fail(GP_ERR_INVALID, "gp_init: more than 2^31-1 grid points");
  }
  if (!std::isfinite(dt) || dt == 0.0) return fail(GP_ERR_INVALID, "gp_init: dt must be finite and nonzero");
  if (!std::isfinite(g)) return fail(GP_ERR_INVALID, "gp_init: g must be finite");

  gp_handle* h = new gp_handle();
  h->dim = dim;
  h->geom = geom;
  for (int d = 0; d < 3; ++d) {
    h->n[d] = d < dim ? n[d] : 1;
    h->dx[d] = d < dim ? dx[d] : 1.0;
    h->nkl[d] = d < dim ? nkl[d] : 0.0;
  }
  h->dt = dt;
  h->g = g;
  h->prec = prec;
  h->np = np;
  h->esize = prec == GP_F64 ? sizeof(double2) : prec == GP_DF64 ? sizeof(df64x2) : sizeof(float2);
  h->user = (cudaStream_t)stream;
  int rc = GP_OK;
  auto bail = [&](int code) { gp_destroy(h); return code; };
  {
    cudaError_t e = cudaStreamCreateWithFlags(&h->work, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(GP_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->obs_host, 8 * sizeof(double));
    if (e != cudaSuccess) return bail(fail(GP_ERR_CUDA, std::string("gp_init: ") + cudaGetErrorString(e)));
  }
  const size_t tsz = prec == GP_F64 ? sizeof(double) : prec == GP_DF64 ? sizeof(df64) : sizeof(float);
  if ((rc = dev_alloc(h, &h->psi, (size_t)np * h->esize))) return bail(rc);
  for (int d = 0; d < 3; ++d) {
    const int nd = axis_len(h, d);
    std::vector<double> x(nd, 0.0), v(nd, 0.0), w(nd, 1.0), wc(nd, 1.0);
    if (d < dim) {
      for (int i = 0; i < nd; ++i) {
        x[i] = axis_coord(geom, d, nd, dx[d], i);
        v[i] = 0.5 * nkl[d] * nkl[d] * x[i] * x[i];
      }
      if (geom == 2 && d == 0) {
        // rho of a circular / axial trap: midpoint weights 2 pi rho_i drho =
        // (2i - 1) pi drho^2 on i = 1..n-2 (coefficients 2i - 1, exact in FP32)
        for (int i = 0; i < nd; ++i) {
          const double c = (i >= 1 && i <= nd - 2) ? 2.0 * i - 1.0 : 0.0;
          wc[i] = c;
          w[i] = c * M_PI * dx[d] * dx[d];
        }
        h->wscale *= M_PI * dx[d] * dx[d];
      } else {
        // composite Simpson on the first m points (m = n odd, n-1 even)
        const int m = (nd % 2 == 1) ? nd : nd - 1;
        for (int i = 0; i < nd; ++i) {
          double c = 0.0;
          if (i < m) c = (i == 0 || i == m - 1) ? 1.0 : (i % 2 == 1 ? 4.0 : 2.0);
          wc[i] = c;
          w[i] = c * dx[d] / 3.0;
        }
        h->wscale *= dx[d] / 3.0;
      }
    }
    if ((rc = dev_alloc(h, &h->vt[d], nd * tsz))) return bail(rc);
    if ((rc = dev_alloc(h, &h->fac[0][d], nd * h->esize))) return bail(rc);
    if ((rc = dev_alloc(h, &h->fac[1][d], nd * h->esize))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->vd[d], nd * sizeof(double)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->cdx[d], nd * sizeof(double)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->wd[d], nd * sizeof(double)))) return bail(rc);
    if ((rc = dev_alloc(h, &h->wt[d], nd * tsz))) return bail(rc);
    if ((rc = dev_alloc(h, &h->ct[d], nd * tsz))) return bail(rc);
    if (prec == GP_DF64) {
      rc = upload_real<df64>(h, h->vt[d], v);
      if (!rc) rc = upload_real<df64>(h, h->wt[d], wc);
      if (!rc) rc = upload_real<df64>(h, h->ct[d], x);
    } else {
      rc = prec == GP_F64 ? upload_real<double>(h, h->vt[d], v) : upload_real<float>(h, h->vt[d], v);
      if (!rc) rc = prec == GP_F64 ? upload_real<double>(h, h->wt[d], wc) : upload_real<float>(h, h->wt[d], wc);
      if (!rc) rc = prec == GP_F64 ? upload_real<double>(h, h->ct[d], x) : upload_real<float>(h, h->ct[d], x);
    }
    if (rc) return bail(rc);
    if ((rc = upload_real<double>(h, h->vd[d], v))) return bail(rc);
    if ((rc = upload_real<double>(h, h->cdx[d], x))) return bail(rc);
    if ((rc = upload_real<double>(h, h->wd[d], w))) return bail(rc);
  }
  for (int d = 0; d < dim; ++d) {
    for (int mode = 0; mode < NUM_MODES; ++mode) {
      if ((rc = dev_alloc(h, &h->coef[mode][d], (size_t)(1 + 2 * kNumSegs) * h->n[d] * h->esize))) return bail(rc);
      if ((rc = dev_alloc(h, &h->ctab[mode][d], (size_t)kNumSegs * 512 * h->esize))) return bail(rc);
    }
    if (d == 0 && prec == GP_F32 && dim > 1 && geom == 0)
      for (int mode = 0; mode < 2; ++mode)
        if ((rc = dev_alloc(h, &h->coef_even[mode], ((size_t)4 * h->n[0] + 1024) * h->esize))) return bail(rc);
    for (int im = 0; im < 2; ++im) {
      if ((rc = dev_alloc(h, &h->cm[im][d], (size_t)h->n[d] * h->esize))) return bail(rc);
      if ((rc = dev_alloc(h, &h->ccp[im][d], (size_t)h->n[d] * h->esize))) return bail(rc);
    }
  }
  if (prec == GP_DF64) {
    const long nyz = (long)axis_len(h, 1) * axis_len(h, 2);
    for (int m = 0; m < 2; ++m) {
      if ((rc = dev_alloc(h, &h->tfx[m], (size_t)h->n[0] * sizeof(tf3c)))) return bail(rc);
      if ((rc = dev_alloc(h, &h->tfyz[m], (size_t)nyz * sizeof(tf3c)))) return bail(rc);
    }
    if ((rc = dev_alloc(h, &h->df_stage, (size_t)np * sizeof(double2)))) return bail(rc);
  }
  if (geom == 2)
    for (int mode = 0; mode < NUM_MODES; ++mode)
      if ((rc = dev_alloc(h, &h->cvar[mode], (size_t)3 * h->n[0] * h->esize))) return bail(rc);
  if (geom == 1) {
    // weight of the nonlinear term of the radial problem, 1/(4 pi r^2) (0 at r = 0, where u is held at zero)
    std::vector<double> gw(n[0], 0.0);
    for (int i = 1; i < n[0]; ++i) gw[i] = 1.0 / (4.0 * M_PI * (i * dx[0]) * (i * dx[0]));
    if ((rc = dev_alloc(h, &h->gw_t, n[0] * tsz))) return bail(rc);
    if ((rc = dev_alloc(h, &h->gw_o, n[0] * sizeof(double)))) return bail(rc);
    if (prec == GP_DF64) rc = upload_real<df64>(h, h->gw_t, gw);
    else rc = prec == GP_F64 ? upload_real<double>(h, h->gw_t, gw) : upload_real<float>(h, h->gw_t, gw);
    if (!rc) rc = prec == GP_F32 ? upload_real<float>(h, h->gw_o, gw) : upload_real<double>(h, h->gw_o, gw);
    if (rc) return bail(rc);
  }
  if ((rc = upload_coefs(h))) return bail(rc);
  if ((rc = upload_factors(h))) return bail(rc);
  choose_shapes(h);
  if (prec == GP_DF64 && (h->seg_x == 0 || (dim > 1 && h->seg_c == 0)))
    return bail(fail(GP_ERR_INVALID, "gp_init: the double-float form takes at most 514 points per axis"));
  if (geom == 2 && (h->seg_x == 0 || (dim > 1 && h->seg_c == 0)))
    return bail(fail(GP_ERR_INVALID, "gp_init: circular and axial traps take at most 514 points per axis"));
  // reduction scratch: enough partial slots for any sweep or observables grid
  long maxblocks = 152L * 16;
  for (int d = 0; d < dim; ++d) maxblocks = std::max(maxblocks, h->np / h->n[d] / 4 + 1);
  if ((rc = dev_alloc(h, (void**)&h->partials, (size_t)maxblocks * 8 * sizeof(double)))) return bail(rc);
  if ((rc = dev_alloc(h, (void**)&h->counter, 64))) return bail(rc);
  if ((rc = dev_alloc(h, (void**)&h->dev_err, 64))) return bail(rc);
  h->tma_limit_ns = (unsigned long long)env_int("GPE_WAIT_LIMIT_MS", 1000) * 1000000ull;
  {
    // one norm sum per block of any last sweep: 32 lines per block (tiles and
    // y/z sweeps), 4 (one-warp x lines), 128 (long lines), or a persistent grid
    long maxparts = 152L * 32;
    for (int d = 0; d < dim; ++d) maxparts = std::max(maxparts, h->np / h->n[d] / 4 + 1);
    for (int i = 0; i < 2; ++i)
      if ((rc = dev_alloc(h, (void**)&h->parts[i], (size_t)maxparts * sizeof(double)))) return bail(rc);
  }
  if ((rc = dev_alloc(h, (void**)&h->obs_out, 8 * sizeof(double)))) return bail(rc);
  {
    cudaError_t e = cudaStreamSynchronize(h->work);
    if (e != cudaSuccess) return bail(fail(GP_ERR_CUDA, std::string("gp_init: ") + cudaGetErrorString(e)));
  }
  *out = h;
  return GP_OK;
}
}  // namespace

int gp_init(gp_handle** out, int dim, const int n[3], const double dx[3], double dt,
            const double nkl[3], double g, gp_precision prec, void* stream) {
  return init_handle(out, 0, dim, n, dx, dt, nkl, g, prec, stream);
}

int gp_init_spherical(gp_handle** out, int n, double dr, double dt, double nu, double g, gp_precision prec,
                      void* stream) {
  const int n3[3] = {n, 1, 1};
  const double dx3[3] = {dr, 1.0, 1.0}, nkl3[3] = {nu, 0.0, 0.0};
  return init_handle(out, 1, 1, n3, dx3, dt, nkl3, g, prec, stream);
}

int gp_init_circular(gp_handle** out, int n, double drho, double dt, double nu, double g, gp_precision prec,
                     void* stream) {
  const int n3[3] = {n, 1, 1};
  const double dx3[3] = {drho, 1.0, 1.0}, nkl3[3] = {nu, 0.0, 0.0};
  return init_handle(out, 2, 1, n3, dx3, dt, nkl3, g, prec, stream);
}

int gp_init_axial(gp_handle** out, int n_rho, int n_z, double drho, double dz, double dt, double nu, double lambda,
                  double g, gp_precision prec, void* stream) {
  const int n3[3] = {n_rho, n_z, 1};
  const double dx3[3] = {drho, dz, 1.0}, nkl3[3] = {nu, lambda, 0.0};
  return init_handle(out, 2, 2, n3, dx3, dt, nkl3, g, prec, stream);
}

int gp_set_state(gp_handle* h, const void* psi, int on_device) {
  if (!h || !psi) return fail(GP_ERR_INVALID, "gp_set_state: NULL argument");
  int rc = join_in(h);
  if (rc) return rc;
  if (h->prec == GP_DF64) {  // complex128 in, split on the device
    const void* src = psi;
    if (!on_device) {
      GP_CUDA(cudaMemcpyAsync(h->df_stage, psi, (size_t)h->np * sizeof(double2), cudaMemcpyHostToDevice, h->work));
      src = h->df_stage;
    }
    df_from_c128(h, src);
    GP_CUDA(cudaGetLastError());
  } else {
    GP_CUDA(cudaMemcpyAsync(h->psi, psi, (size_t)h->np * h->esize,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->work));
    if (h->real_mode && (rc = real_from_complex(h))) {
      h->real_mode = false;  // the complex state just set stays
      drop_graphs(h);
      join_out(h);
      return rc;
    }
  }
  if (!on_device) GP_CUDA(cudaStreamSynchronize(h->work));
  return join_out(h);
}

int gp_get_state(gp_handle* h, void* psi, int on_device) {
  if (!h || !psi) return fail(GP_ERR_INVALID, "gp_get_state: NULL argument");
  int rc = join_in(h);
  if (rc) return rc;
  if (h->prec == GP_DF64) {  // rounded to complex128
    df_to_c128(h, on_device ? psi : h->df_stage);
    GP_CUDA(cudaGetLastError());
    if (!on_device)
      GP_CUDA(cudaMemcpyAsync(psi, h->df_stage, (size_t)h->np * sizeof(double2), cudaMemcpyDeviceToHost, h->work));
  } else {
    materialize_complex(h);  // a real state: its complex copy
    GP_CUDA(cudaMemcpyAsync(psi, h->psi, (size_t)h->np * h->esize,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->work));
  }
  if (!on_device) GP_CUDA(cudaStreamSynchronize(h->work));
  return join_out(h);
}

int gp_set_potential(gp_handle* h, const double* V, int on_device) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_potential: NULL handle");
  int rc = join_in(h);
  if (rc) return rc;
  drop_graphs(h);
  ++h->pot_version;
  if (!V) {
    h->Vd = nullptr;
    h->Vt = nullptr;
    return join_out(h);
  }
  // persistent buffers, allocated on first use: FP64 copy (observables, FP64
  // sweeps) and, for the FP32 form, an FP32 copy read by the x sweep
  if (!h->Vbuf) {
    void* p = nullptr;
    if ((rc = dev_alloc(h, &p, (size_t)h->np * sizeof(double)))) return rc;
    h->Vbuf = (double*)p;
    if (h->prec == GP_F32) {
      if ((rc = dev_alloc(h, &p, (size_t)h->np * sizeof(float)))) return rc;
      h->Vbuf32 = (float*)p;
    }
    if ((rc = dev_alloc(h, &h->fV[0], (size_t)h->np * h->esize))) return rc;
    if ((rc = dev_alloc(h, &h->fV[1], (size_t)h->np * h->esize))) return rc;
    if (h->prec == GP_DF64) {
      if ((rc = dev_alloc(h, &h->tfV[0], (size_t)h->np * sizeof(tf3c)))) return rc;
      if ((rc = dev_alloc(h, &h->tfV[1], (size_t)h->np * sizeof(tf3c)))) return rc;
    }
  }
  GP_CUDA(cudaMemcpyAsync(h->Vbuf, V, (size_t)h->np * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->work));
  h->Vd = h->Vbuf;
  if (h->prec == GP_F64) {
    h->Vt = h->Vbuf;
  } else if (h->prec == GP_DF64) {
    h->Vt = nullptr;  // the double-float sweeps read only the factors
  } else {
    to_float(h, h->Vbuf32, h->Vbuf, h->np);
    h->Vt = h->Vbuf32;
  }
  potential_factors(h, h->dt, h->fV, h->tfV);
  if (h->strang) {
    if ((rc = ensure_half_tables(h))) return rc;
    potential_factors(h, 0.5 * h->dt, h->fV_h, h->tfV_h);
  }
  GP_CUDA(cudaGetLastError());
  if (!on_device) GP_CUDA(cudaStreamSynchronize(h->work));
  return join_out(h);
}

int gp_set_splitting(gp_handle* h, int strang) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_splitting: NULL handle");
  if (strang != 0 && strang != 1) return fail(GP_ERR_INVALID, "gp_set_splitting: splitting must be 0 (Lie) or 1 (Strang)");
  if ((strang != 0) == h->strang) return GP_OK;
  if (strang && h->real_mode) return fail(GP_ERR_STATE, "gp_set_splitting: the Strang splitting takes the complex state");
  int rc = join_in(h);
  if (rc) return rc;
  drop_graphs(h);
  if (strang && (rc = ensure_half_tables(h))) return rc;
  h->strang = strang != 0;
  if (h->strang && (rc = upload_factor_set(h, 0.5 * h->dt, h->fac_h, h->tfx_h, h->tfyz_h, h->fV_h, h->tfV_h)))
    return rc;
  return join_out(h);
}

int gp_set_g(gp_handle* h, double g) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_g: NULL handle");
  if (!std::isfinite(g)) return fail(GP_ERR_INVALID, "gp_set_g: g must be finite");
  if (g != h->g) drop_graphs(h);
  h->g = g;
  return GP_OK;
}

int gp_set_dt(gp_handle* h, double dt) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_dt: NULL handle");
  if (!std::isfinite(dt) || dt == 0.0) return fail(GP_ERR_INVALID, "gp_set_dt: dt must be finite and nonzero");
  if (dt == h->dt) return GP_OK;
  int rc = join_in(h);
  if (rc) return rc;
  drop_graphs(h);
  h->dt = dt;
  if ((rc = upload_coefs(h))) return rc;
  if ((rc = upload_factors(h))) return rc;
  return join_out(h);
}

int gp_step_imag(gp_handle* h, long nsteps) {
  if (!h) return fail(GP_ERR_INVALID, "gp_step_imag: NULL handle");
  if (nsteps < 0) return fail(GP_ERR_INVALID, "gp_step_imag: nsteps < 0");
  return run_steps_any(h, true, nsteps);
}

int gp_step_real(gp_handle* h, long nsteps) {
  if (!h) return fail(GP_ERR_INVALID, "gp_step_real: NULL handle");
  if (nsteps < 0) return fail(GP_ERR_INVALID, "gp_step_real: nsteps < 0");
  if (h->real_mode) return fail(GP_ERR_STATE, "gp_step_real: real-time steps need the complex state (gp_set_real_state(h, 0))");
  return run_steps_any(h, false, nsteps);
}

int gp_time_sweeps_graph(gp_handle* h, int imag, int reps, double* ms_per_launch) {
  if (!h || !ms_per_launch) return fail(GP_ERR_INVALID, "gp_time_sweeps_graph: NULL argument");
  if (reps < 1 || reps > 1024) return fail(GP_ERR_INVALID, "gp_time_sweeps_graph: reps must be in [1, 1024]");
  if (h->real_mode && !imag) return fail(GP_ERR_STATE, "gp_time_sweeps_graph: a real state takes imaginary time only");
  void* const state = h->real_mode ? h->rpsi : h->psi;
  const size_t sbytes = (size_t)h->np * (h->real_mode ? h->esize / 2 : h->esize);
  void* saved = nullptr;
  GP_CUDA(cudaMalloc(&saved, sbytes));
  int rc = join_in(h);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(saved, state, sbytes, cudaMemcpyDeviceToDevice, h->work);
    if (e != cudaSuccess) rc = fail(GP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (!rc) {
    rc = h->prec == GP_DF64 ? time_graph_df(h, imag != 0, reps, ms_per_launch)
         : h->prec == GP_F64 ? time_graph_f64(h, imag != 0, reps, ms_per_launch)
                             : time_graph_f32(h, imag != 0, reps, ms_per_launch);
  }
  cudaError_t e = cudaMemcpyAsync(state, saved, sbytes, cudaMemcpyDeviceToDevice, h->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->work);
  cudaFree(saved);
  if (!rc && e != cudaSuccess) rc = fail(GP_ERR_CUDA, std::string("gp_time_sweeps_graph: ") + cudaGetErrorString(e));
  if (!rc) rc = read_dev_err(h, "gp_time_sweeps_graph");
  return rc;
}

int gp_time_sweeps(gp_handle* h, int imag, long nsteps, double* ms_per_launch) {
  if (!h || !ms_per_launch) return fail(GP_ERR_INVALID, "gp_time_sweeps: NULL argument");
  if (nsteps < 0 || nsteps > 4096) return fail(GP_ERR_INVALID, "gp_time_sweeps: nsteps must be in [0, 4096]");
  if (h->real_mode && !imag) return fail(GP_ERR_STATE, "gp_time_sweeps: a real state takes imaginary-time steps only");
  return time_steps_any(h, imag != 0, nsteps, ms_per_launch);
}

namespace {

// (Re)allocates a buffer of `count` states when the current one is smaller.
int ensure_states(gp_handle* h, void** buf, long* cap, long count) {
  if (*cap >= count && *buf) return GP_OK;
  if (*buf) {
    cudaStreamSynchronize(h->work);
    guarded_free(*buf);
    for (auto& p : h->allocs)
      if (p == *buf) p = nullptr;
    *buf = nullptr;
    *cap = 0;
  }
  int rc = dev_alloc(h, buf, (size_t)count * h->np * h->esize);
  if (rc) return rc;
  *cap = count;
  return GP_OK;
}

}  // namespace

int gp_adjoint_forward(gp_handle* h, long nsteps, int ckpt_every) {
  if (!h) return fail(GP_ERR_INVALID, "gp_adjoint_forward: NULL handle");
  if (nsteps < 1 || ckpt_every < 1) return fail(GP_ERR_INVALID, "gp_adjoint_forward: need nsteps >= 1, ckpt_every >= 1");
  if (h->seg_x == 0 || (h->dim > 1 && h->seg_c == 0))
    return fail(GP_ERR_INVALID, "gp_adjoint_forward: lines longer than 514 points are not supported");
  if (h->prec == GP_DF64)
    return fail(GP_ERR_INVALID, "gp_adjoint_forward: the adjoint takes GP_F64 or GP_F32 states");
  if (h->geom != 0) return fail(GP_ERR_INVALID, "gp_adjoint_forward: the adjoint is for Cartesian grids");
  if (h->strang) return fail(GP_ERR_INVALID, "gp_adjoint_forward: the adjoint is for the Lie splitting");
  if (h->real_mode) return fail(GP_ERR_STATE, "gp_adjoint_forward: the adjoint takes the complex state");
  const int K = (int)std::min<long>(ckpt_every, nsteps);
  const long nck = (nsteps + K - 1) / K;
  int rc;
  if ((rc = ensure_states(h, &h->adj_ckpt, &h->adj_ckpt_cap, nck))) return rc;
  if ((rc = ensure_states(h, &h->adj_traj, &h->adj_traj_cap, K))) return rc;
  if (!h->adj_lam) {
    if ((rc = dev_alloc(h, &h->adj_lam, (size_t)h->np * h->esize))) return rc;
    void* p = nullptr;
    if ((rc = dev_alloc(h, &p, (size_t)h->np * sizeof(double)))) return rc;
    h->adj_dJdV = (double*)p;
    if ((rc = dev_alloc(h, &p, 16))) return rc;
    h->adj_dJdg = (double*)p;
  }
  h->adj_nsteps = -1;
  rc = h->prec == GP_F64 ? adjoint_forward_f64(h, nsteps, K) : adjoint_forward_f32(h, nsteps, K);
  if (rc) return rc;
  h->adj_nsteps = nsteps;
  h->adj_K = K;
  h->adj_g = h->g;
  h->adj_dt = h->dt;
  h->adj_pot_version = h->pot_version;
  return GP_OK;
}

int gp_adjoint_backward(gp_handle* h, const void* lambda_T, int lambda_on_device, double* dJdV, int dJdV_on_device,
                        double* dJdg, void* lambda_0) {
  if (!h || !lambda_T) return fail(GP_ERR_INVALID, "gp_adjoint_backward: NULL argument");
  if (h->adj_nsteps < 1) return fail(GP_ERR_STATE, "gp_adjoint_backward: no gp_adjoint_forward recorded");
  if (h->strang) return fail(GP_ERR_STATE, "gp_adjoint_backward: the splitting was changed to Strang after the forward run");
  if (h->dt != h->adj_dt || h->pot_version != h->adj_pot_version)
    return fail(GP_ERR_STATE, "gp_adjoint_backward: dt or the potential changed since gp_adjoint_forward");
  int rc = join_in(h);
  if (rc) return rc;
  GP_CUDA(cudaMemcpyAsync(h->adj_lam, lambda_T, (size_t)h->np * h->esize,
                          lambda_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->work));
  if (!lambda_on_device) GP_CUDA(cudaStreamSynchronize(h->work));
  if ((rc = join_out(h))) return rc;
  double* ddev = (dJdV && dJdV_on_device) ? dJdV : nullptr;
  rc = h->prec == GP_F64 ? adjoint_backward_f64(h, ddev, lambda_0) : adjoint_backward_f32(h, ddev, lambda_0);
  if (rc) return rc;
  if ((rc = join_in(h))) return rc;
  if (dJdV && !dJdV_on_device)
    GP_CUDA(cudaMemcpyAsync(dJdV, h->adj_dJdV, (size_t)h->np * sizeof(double), cudaMemcpyDeviceToHost, h->work));
  GP_CUDA(cudaMemcpyAsync(h->obs_host, h->adj_dJdg, sizeof(double), cudaMemcpyDeviceToHost, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  if ((rc = join_out(h))) return rc;
  if (dJdg) *dJdg = h->obs_host[0];
  if (!std::isfinite(h->obs_host[0])) return fail(GP_ERR_NONFINITE, "gp_adjoint_backward: non-finite gradient");
  return GP_OK;
}

namespace {

bool shapes_valid(const gp_handle* h, int tile_x, int seg_x, int seg_c) {
  const int M0 = h->n[0] - 2;
  int Mc = 0;
  for (int d = 1; d < h->dim; ++d) Mc = std::max(Mc, h->n[d] - 2);
  if (seg_x != 0) {
    if (seg_index(seg_x) < 0) return false;
    if (tile_x) {
      if (h->dim < 2 || seg_x < 4 || (M0 + seg_x - 1) / seg_x > 16) return false;
      if ((36L * h->n[0] + 512) * (long)h->esize > 200L * 1024) return false;
    } else if (seg_x > 16 || 32 * seg_x < M0) {
      return false;
    }
  } else if (tile_x) {
    return false;
  }
  if (h->dim > 1 && seg_c != 0 && (seg_index(seg_c) < 0 || seg_c < 4 || (Mc + seg_c - 1) / seg_c > 16)) return false;
  if (h->dim == 1 && seg_c != 0 && (seg_index(seg_c) < 0 || seg_c < 4)) return false;
  return true;
}

struct TuneKey {
  int dim, n0, n1, n2, prec, imag, real;
  bool operator<(const TuneKey& o) const {
    return std::tie(dim, n0, n1, n2, prec, imag, real) < std::tie(o.dim, o.n0, o.n1, o.n2, o.prec, o.imag, o.real);
  }
};
std::map<TuneKey, std::array<int, 4>> g_tuned;  // process-wide results
std::mutex g_tune_mutex;

}  // namespace

int gp_check_status(int* first_failure) {
  if (!first_failure) return fail(GP_ERR_INVALID, "gp_check_status: NULL argument");
  GP_CUDA(cudaDeviceSynchronize());
#ifdef GPE_BOUNDS_CHECK
  int first = 0;
  {
    std::lock_guard<std::mutex> lock(g_reader_mutex);
    for (auto rd : check_readers()) {
      const int v = rd();
      if (v < 0) return fail(GP_ERR_CUDA, "gp_check_status: a check flag could not be read");
      if (v && !first) first = v;
    }
  }
  if (first) {
    *first_failure = first;
    return fail(GP_ERR_STATE, "gp_check_status: index check " + std::to_string(first) + " failed");
  }
  std::lock_guard<std::mutex> lock(g_guard_mutex);
  std::vector<unsigned char> buf(kGuard);
  for (auto& kv : guard_map()) {
    const char* raw = kv.second.first;
    const size_t bytes = kv.second.second;
    for (int side = 0; side < 2; ++side) {
      GP_CUDA(cudaMemcpy(buf.data(), raw + (side ? kGuard + bytes : 0), kGuard, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < kGuard; ++i)
        if (buf[i] != 0xFF) {
          *first_failure = 1;
          return fail(GP_ERR_STATE, std::string("gp_check_status: the guard band ") + (side ? "after" : "before") +
                                        " a buffer of " + std::to_string(bytes) + " bytes was overwritten");
        }
    }
  }
  *first_failure = 0;
  return GP_OK;
#else
  *first_failure = -1;  // a library built without the checks
  return GP_OK;
#endif
}

int gp_test_stall_transfers(gp_handle* h, int extra_bytes) {
  if (!h) return fail(GP_ERR_INVALID, "gp_test_stall_transfers: NULL handle");
  if (extra_bytes < 0 || extra_bytes > 1024)
    return fail(GP_ERR_INVALID, "gp_test_stall_transfers: extra_bytes must be in [0, 1024]");
  drop_graphs(h);  // captured launches carry the old value
  h->tma_expect_extra = extra_bytes;
  return GP_OK;
}

int gp_set_shapes(gp_handle* h, int tile_x, int seg_x, int seg_c, int flags) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_shapes: NULL handle");
  if (!shapes_valid(h, tile_x, seg_x, seg_c)) return fail(GP_ERR_INVALID, "gp_set_shapes: invalid shapes for this grid");
  if (h->real_mode && (!tile_x || seg_x == 0 || seg_c == 0))
    return fail(GP_ERR_STATE, "gp_set_shapes: a real state needs the x tile and segmented y/z sweeps");
  const bool fxy = (flags & GP_SHAPE_FUSE_XY) != 0;
  if (fxy && (!plane_fits(h, seg_x) || (flags & GP_SHAPE_PIPE_X)))
    return fail(GP_ERR_INVALID, "gp_set_shapes: the fused x + y sweeps take 3d FP32 grids with nx, ny <= 128 and "
                                "seg_x 8, 16 or 32 for both axes, without the pipelined x sweep");
  if (h->geom == 2 && (seg_x == 0 || (h->dim > 1 && seg_c == 0) || (flags & GP_SHAPE_PIPE_X)))
    return fail(GP_ERR_INVALID, "gp_set_shapes: the rho axis takes the segmented, non-pipelined x sweeps");
  const bool px = (flags & GP_SHAPE_PIPE_X) != 0, pc = (flags & GP_SHAPE_PIPE_YZ) != 0;
  if ((px || pc) && h->prec == GP_DF64)
    return fail(GP_ERR_INVALID, "gp_set_shapes: the pipelined sweeps take GP_F64 or GP_F32 states");
  if (px && (!tile_x || seg_x == 0 || !pipe_fits(h, h->n[0], true)))
    return fail(GP_ERR_INVALID, "gp_set_shapes: pipelined x sweep needs the x tile and two stages in shared memory");
  int nmax = 0;
  for (int d = 1; d < h->dim; ++d) nmax = std::max(nmax, h->n[d]);
  if (pc && (h->dim < 2 || seg_c == 0 || !pipe_fits(h, nmax, false)))
    return fail(GP_ERR_INVALID, "gp_set_shapes: pipelined y/z sweeps need two stages in shared memory");
  const bool tx = (flags & GP_SHAPE_TMA_X) != 0;
  if (tx && (px || fxy || !tile_x || !tma_x_fits(h, seg_x)))
    return fail(GP_ERR_INVALID, "gp_set_shapes: the TMA x sweep takes GP_F32 complex states of Cartesian 2d/3d grids "
                                "with nx a multiple of 16 and at most 256, the x tile with seg_x 8 or 16, without the "
                                "pipelined or fused x sweeps");
  const bool tc = (flags & GP_SHAPE_TMA_YZ) != 0;
  if (tc && (pc || !tma_fits(h, seg_c)))
    return fail(GP_ERR_INVALID, "gp_set_shapes: the TMA y/z sweeps take GP_F32 complex states with nx even, y/z lines of "
                                "at most 256 points and seg_c 8, 16 or 32 (at most 16 segments), without the "
                                "pipelined y/z sweeps");
  drop_graphs(h);
  h->tma_c = tc;
  h->tma_x = tx;
  h->tile_x = tile_x != 0;
  h->seg_x = seg_x;
  h->seg_c = seg_c;
  h->keep_c = (flags & GP_SHAPE_KEEP_YZ) != 0;
  h->pipe_x = px;
  h->pipe_c = pc;
  h->xyfuse = fxy;
  return GP_OK;
}

int gp_get_shapes(const gp_handle* h, int* tile_x, int* seg_x, int* seg_c, int* flags) {
  if (!h) return fail(GP_ERR_INVALID, "gp_get_shapes: NULL handle");
  if (tile_x) *tile_x = h->tile_x ? 1 : 0;
  if (seg_x) *seg_x = h->seg_x;
  if (seg_c) *seg_c = h->seg_c;
  if (flags)
    *flags = (h->keep_c ? GP_SHAPE_KEEP_YZ : 0) | (h->pipe_x ? GP_SHAPE_PIPE_X : 0) |
             (h->pipe_c ? GP_SHAPE_PIPE_YZ : 0) | (h->xyfuse ? GP_SHAPE_FUSE_XY : 0) |
             (h->tma_c ? GP_SHAPE_TMA_YZ : 0) | (h->tma_x ? GP_SHAPE_TMA_X : 0);
  return GP_OK;
}

int gp_autotune(gp_handle* h, int imag, int nsteps, double* best_ms) {
  if (!h) return fail(GP_ERR_INVALID, "gp_autotune: NULL handle");
  if (nsteps < 1 || nsteps > 256) return fail(GP_ERR_INVALID, "gp_autotune: nsteps must be in [1, 256]");
  if (h->real_mode && !imag) return fail(GP_ERR_STATE, "gp_autotune: a real state takes imaginary-time steps only");
  const bool real = h->real_mode;  // tile x sweep, no pipelined shapes, the real buffer saved
  const TuneKey key{h->dim, h->n[0], h->n[1], h->n[2], h->prec, imag != 0, real ? 1 : 0};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end() && !best_ms) {
      return gp_set_shapes(h, it->second[0], it->second[1], it->second[2], it->second[3]);
    }
  }
  // candidate shapes for the x sweep and for the y/z sweeps (timed separately)
  std::vector<std::array<int, 4>> xs;  // (tile, seg, pipelined, TMA)
  for (int sg : {4, 8, 16, 32})
    if (shapes_valid(h, 1, sg, h->seg_c)) {
      xs.push_back({1, sg, 0, 0});
      if (h->prec != GP_DF64 && !real && h->geom != 2 && pipe_fits(h, h->n[0], true)) xs.push_back({1, sg, 1, 0});
      if (!real && tma_x_fits(h, sg)) xs.push_back({1, sg, 0, 1});
    }
  for (int sg : {1, 2, 4, 8, 16})
    if (!real && shapes_valid(h, 0, sg, h->seg_c)) { xs.push_back({0, sg, 0, 0}); break; }
  std::vector<std::array<int, 4>> cs;  // (seg, keep input in registers, pipelined, TMA)
  int nmax = 0;
  for (int d = 1; d < h->dim; ++d) nmax = std::max(nmax, h->n[d]);
  if (h->dim > 1)
    for (int sg : {4, 8, 16, 32})
      if (shapes_valid(h, h->tile_x, h->seg_x, sg)) {
        if (sg * (int)h->esize / 2 <= 64) cs.push_back({sg, 1, 0, 0});
        cs.push_back({sg, 0, 0, 0});
        if (h->prec != GP_DF64 && !real && pipe_fits(h, nmax, false)) cs.push_back({sg, 0, 1, 0});
        if (!real && tma_fits(h, sg)) cs.push_back({sg, 0, 0, 1});
      }
  const int keep_t = h->tile_x, keep_x = h->seg_x, keep_c = h->seg_c, keep_k = h->keep_c;
  const bool keep_px = h->pipe_x, keep_pc = h->pipe_c, keep_fxy = h->xyfuse, keep_tc = h->tma_c;
  const bool keep_tx = h->tma_x;
  h->xyfuse = false;  // the separate sweeps first
  void* saved = nullptr;
  void* const state = real ? h->rpsi : h->psi;
  const size_t sbytes = (size_t)h->np * (real ? h->esize / 2 : h->esize);
  GP_CUDA(cudaMalloc(&saved, sbytes));
  int rc = join_in(h);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(saved, state, sbytes, cudaMemcpyDeviceToDevice, h->work);
    if (e != cudaSuccess) rc = fail(GP_ERR_CUDA, cudaGetErrorString(e));
  }
  auto time_shape = [&](int t, int sx, int px, int tx, int sc, int kc, int pc, int tc, double* ms3) -> int {
    h->tile_x = t != 0;
    h->seg_x = sx;
    h->pipe_x = px != 0;
    h->tma_x = tx != 0;
    h->seg_c = sc;
    h->keep_c = kc;
    h->pipe_c = pc != 0;
    h->tma_c = tc != 0;
    double warm[3];
    int r = time_steps_any(h, imag != 0, 2, warm);
    if (r) return r;
    return time_steps_any(h, imag != 0, nsteps, ms3);
  };
  double bx = 1e30, bc = 1e30;
  int best_t = keep_t, best_x = keep_x, best_c = keep_c, best_k = keep_k, best_px = keep_px, best_pc = keep_pc;
  int best_tc = keep_tc, best_tx = keep_tx;
  for (const auto& c : xs) {
    if (rc) break;
    double ms[3];
    rc = time_shape(c[0], c[1], c[2], c[3], keep_c, keep_k, keep_pc, keep_tc, ms);
    if (!rc && ms[0] < bx) { bx = ms[0]; best_t = c[0]; best_x = c[1]; best_px = c[2]; best_tx = c[3]; }
  }
  for (const auto& c : cs) {
    if (rc) break;
    double ms[3];
    rc = time_shape(best_t, best_x, best_px, best_tx, c[0], c[1], c[2], c[3], ms);
    const double t = ms[1] + ms[2];
    if (!rc && t < bc) { bc = t; best_c = c[0]; best_k = c[1]; best_pc = c[2]; best_tc = c[3]; }
  }
  // the fused x + y sweeps, with the best z shape, against the best separate ones
  // (8- and 16-point segments: 32-point ones spill under the 64 registers a
  // thread of a 1024-thread block may hold)
  bool best_fxy = false;
  if (!real)
    for (int sg : {8, 16}) {
      if (rc || !plane_fits(h, sg) || !shapes_valid(h, 1, sg, best_c)) continue;
      double ms[3];
      h->xyfuse = true;
      rc = time_shape(1, sg, 0, 0, best_c, best_k, best_pc, best_tc, ms);
      h->xyfuse = false;
      if (!rc && ms[0] + ms[1] + ms[2] < bx + bc) {
        bx = ms[0] + ms[1];
        bc = ms[2];
        best_fxy = true;
        best_t = 1;
        best_x = sg;
        best_px = 0;
        best_tx = 0;
      }
    }
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(state, saved, sbytes, cudaMemcpyDeviceToDevice, h->work);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->work);
    if (e != cudaSuccess) rc = fail(GP_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaFree(saved);
  const int best_flags = (best_k ? GP_SHAPE_KEEP_YZ : 0) | (best_px ? GP_SHAPE_PIPE_X : 0) |
                         (best_pc ? GP_SHAPE_PIPE_YZ : 0) | (best_fxy ? GP_SHAPE_FUSE_XY : 0) |
                         (best_tc ? GP_SHAPE_TMA_YZ : 0) | (best_tx ? GP_SHAPE_TMA_X : 0);
  if (rc) {
    h->tile_x = keep_t; h->seg_x = keep_x; h->seg_c = keep_c; h->keep_c = keep_k;
    h->pipe_x = keep_px; h->pipe_c = keep_pc; h->xyfuse = keep_fxy; h->tma_c = keep_tc; h->tma_x = keep_tx;
    return rc;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = {best_t, best_x, best_c, best_flags};
  }
  if (best_ms) {
    best_ms[0] = xs.empty() ? 0.0 : bx;
    best_ms[1] = cs.empty() ? 0.0 : bc;
  }
  if ((rc = gp_set_shapes(h, best_t, best_x, best_c, best_flags))) return rc;
  return join_out(h);
}

int gp_step_series(gp_handle* h, int imag, long nsteps, int every, double* out, int out_on_device) {
  if (!h || !out) return fail(GP_ERR_INVALID, "gp_step_series: NULL argument");
  if (nsteps < 0 || every < 1) return fail(GP_ERR_INVALID, "gp_step_series: need nsteps >= 0 and every >= 1");
  if (h->real_mode && !imag) return fail(GP_ERR_STATE, "gp_step_series: a real state takes imaginary-time steps only");
  const long nrec = nsteps / every;
  int rc = join_in(h);
  if (rc) return rc;
  const size_t need = 8 * (size_t)nrec + (out_on_device ? 0 : 7 * (size_t)nrec);
  if (need > h->series_cap) {
    if (h->series_buf) {
      cudaStreamSynchronize(h->work);
      guarded_free(h->series_buf);
      for (auto& p : h->allocs)
        if (p == h->series_buf) p = nullptr;
      h->series_buf = nullptr;
      h->series_cap = 0;
    }
    void* p = nullptr;
    if ((rc = dev_alloc(h, &p, need * sizeof(double)))) return rc;
    h->series_buf = (double*)p;
    h->series_cap = need;
  }
  for (long r = 0; r < nrec; ++r) {
    if ((rc = run_steps_any(h, imag != 0, every))) return rc;
    if ((rc = run_observables_any(h, nullptr, h->series_buf + 8 * r))) return rc;
  }
  if ((rc = run_steps_any(h, imag != 0, nsteps - nrec * every))) return rc;
  if (nrec > 0) {
    double* dst = out_on_device ? out : h->series_buf + 8 * nrec;
    const int blocks = (int)std::min<long>((nrec + 127) / 128, 152L * 4);
    series_finish_kernel<<<blocks, 128, 0, h->work>>>(h->series_buf, nrec, h->g, dst);
    count_launch();
    GP_CUDA(cudaGetLastError());
    if (!out_on_device) {
      GP_CUDA(cudaMemcpyAsync(out, dst, 7 * (size_t)nrec * sizeof(double), cudaMemcpyDeviceToHost, h->work));
      GP_CUDA(cudaStreamSynchronize(h->work));
    }
  }
  return join_out(h);
}

int gp_observables(gp_handle* h, gp_obs* out, double* density, int density_on_device) {
  if (!h || !out) return fail(GP_ERR_INVALID, "gp_observables: NULL argument");
  int rc = join_in(h);
  if (rc) return rc;
  double* ddev = nullptr;
  if (density) {
    if (density_on_device) {
      ddev = density;
    } else {
      if (!h->dens_scratch) {
        void* p = nullptr;
        if ((rc = dev_alloc(h, &p, (size_t)h->np * sizeof(double)))) return rc;
        h->dens_scratch = (double*)p;
      }
      ddev = h->dens_scratch;
    }
  }
  rc = run_observables_any(h, ddev);
  if (rc) return rc;
  if ((rc = read_dev_err(h, "gp_observables"))) return rc;
  GP_CUDA(cudaMemcpyAsync(h->obs_host, h->obs_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, h->work));
  if (density && !density_on_device)
    GP_CUDA(cudaMemcpyAsync(density, ddev, (size_t)h->np * sizeof(double), cudaMemcpyDeviceToHost, h->work));
  GP_CUDA(cudaStreamSynchronize(h->work));
  rc = join_out(h);
  if (rc) return rc;
  const double* S = h->obs_host;
  const double N = S[0];
  out->norm = N;
  out->energy = (S[1] + S[2]) / N + 0.5 * h->g * S[3] / (N * N);
  out->mu = (S[1] + S[2]) / N + h->g * S[3] / (N * N);
  double r2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    out->rms[d] = std::sqrt(S[4 + d] / N);
    r2 += S[4 + d] / N;
  }
  out->rms_r = std::sqrt(r2);
  for (int q = 0; q < 7; ++q)
    if (!std::isfinite(S[q])) return fail(GP_ERR_NONFINITE, "gp_observables: the state holds NaN or Inf");
  return GP_OK;
}

}  // extern "C"
