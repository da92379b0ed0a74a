// gpe_batch.cu -- many independent 2d real-time runs of uneven size stepped
// together (the batched form; declared in include/gpe.h).
//
// Every run is its own split-step Crank-Nicolson problem ("Solution method" of
// the paper) with its own grid, trap and nonlinearity; they share dt.  One
// time step of the whole batch is one launch of the x sweep (sub-step N fused
// into the load) and one launch of the y sweep per segment-length class --
// runs are grouped by the segment length their line length needs (n <= 66,
// <= 130, <= 258, <= 514 points, plus FP64 x lines too long for the shared
// tile) -- and each block takes one (run, tile) work item from a table, so
// uneven runs share the launch without padding.  The
// kernels are the single-grid bodies of gpe_sweep2.cuh driven by a per-run
// descriptor table, so a run in a batch takes exactly the same arithmetic as
// the same run alone.  Step blocks are captured once into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "gpe_internal.h"
#include "gpe_obs.cuh"
#include "gpe_sweep2.cuh"

using cd = std::complex<double>;

namespace gpe {

template <typename T>
struct BatchRun {
  c2_t<T>* psi;
  int nx, ny;
  const c2_t<T>* coef[2];  // per axis: alpha | gf | gb (3 n values) for the run's segment length
  const c2_t<T>* ptab[2];  // per axis: carry tables (512 values)
  const c2_t<T>* fx; const c2_t<T>* fy; const c2_t<T>* fz1;  // exp(-i dt v(x)), exp(-i dt v(y)), a single 1 (FP64)
  T dtg;                                                   // dt g (FP64)
  const T* vx; const T* vy; const T* vz0;                  // nu^2 x^2/2, kappa^2 y^2/2, a single 0 (FP32)
  T g;
  const tf3c* tfx; const tf3c* tfy;  // the factors fx, fy as exact triple-floats (double-float state)
  int cdepth[2], cpts[2];            // per axis: the segment carries' reach (as the single-grid handle's)
};

struct BatchItem {
  int run, L0;
};

template <typename T, int SEG>
__global__ void __launch_bounds__(512) batch_x_kernel(const BatchRun<T>* __restrict__ runs,
                                                      const BatchItem* __restrict__ items, T dt) {
  extern __shared__ __align__(16) unsigned char bsmem_raw[];
  __shared__ c2_t<T> cf[16][33], cb[16][33];
  __shared__ double red_smem[32];
  const BatchItem it = items[blockIdx.x];
  const BatchRun<T>& R = runs[it.run];
  Sweep2Args<T> A;
  memset(&A, 0, sizeof(A));
  A.psi = R.psi;
  A.geom.axis = 0;
  A.geom.n = R.nx;
  A.geom.stride = 1;
  A.geom.nlines = R.ny;
  A.geom.nx = R.nx;
  A.geom.ny = R.ny;
  A.geom.nz = 1;
  A.alpha = R.coef[0];
  A.gf = R.coef[0] + R.nx;
  A.gb = R.coef[0] + 2 * R.nx;
  A.ptab = R.ptab[0];
  A.cdepth = R.cdepth[0];
  A.cpts = R.cpts[0];
  A.fx = R.fx;
  A.fy = R.fy;
  A.fz = R.fz1;
  A.dtg = R.dtg;
  A.vx = R.vx;
  A.vy = R.vy;
  A.vz = R.vz0;
  A.dt = dt;
  A.g = R.g;
  A.tfx = R.tfx;
  A.tfyz = R.tfy;  // fz = 1 in 2d: the line factor is fy
  tsweep_body<T, false, true, false, SEG>(A, it.L0, reinterpret_cast<c2_t<T>*>(bsmem_raw), cf, cb, red_smem);
}

// x lines whose shared-memory tile would not fit (FP64 and double-float,
// n > 333): one warp per line, 4 lines per block; the item's L0 is the
// block's first line.  The double-float body is held to 128 registers (four
// blocks per SM): with the 234 it would take, 8 warps per SM left it
// latency-bound (604 us per launch on the 64-run workload, ncu; the whole
// double-float batch 7.29e9 -> 9.24e9 point-steps/s with the cap, 8.96e9 at
// 80 registers).
template <typename T, int SEG>
__global__ void __launch_bounds__(128, std::is_same<T, df64>::value ? 4 : 1)
    batch_xw_kernel(const BatchRun<T>* __restrict__ runs, const BatchItem* __restrict__ items, T dt) {
  __shared__ double red_smem[32];
  const BatchItem it = items[blockIdx.x];
  const BatchRun<T>& R = runs[it.run];
  Sweep2Args<T> A;
  memset(&A, 0, sizeof(A));
  A.psi = R.psi;
  A.geom.axis = 0;
  A.geom.n = R.nx;
  A.geom.stride = 1;
  A.geom.nlines = R.ny;
  A.geom.nx = R.nx;
  A.geom.ny = R.ny;
  A.geom.nz = 1;
  A.alpha = R.coef[0];
  A.gf = R.coef[0] + R.nx;
  A.gb = R.coef[0] + 2 * R.nx;
  A.cdepth = R.cdepth[0];
  A.cpts = R.cpts[0];
  A.fx = R.fx;
  A.fy = R.fy;
  A.fz = R.fz1;
  A.dtg = R.dtg;
  A.vx = R.vx;
  A.vy = R.vy;
  A.vz = R.vz0;
  A.dt = dt;
  A.g = R.g;
  A.tfx = R.tfx;
  A.tfyz = R.tfy;
  xsweep_body<T, false, true, false, SEG>(A, it.L0 + (threadIdx.x >> 5), red_smem);
}

template <typename T, int SEG>
__global__ void __launch_bounds__(512) batch_y_kernel(const BatchRun<T>* __restrict__ runs,
                                                      const BatchItem* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char bsmem_raw[];
  __shared__ c2_t<T> cf[16][33], cb[16][33];
  __shared__ double red_smem[32];
  const BatchItem it = items[blockIdx.x];
  const BatchRun<T>& R = runs[it.run];
  Sweep2Args<T> A;
  memset(&A, 0, sizeof(A));
  A.psi = R.psi;
  A.geom.axis = 1;
  A.geom.n = R.ny;
  A.geom.stride = R.nx;
  A.geom.nlines = R.nx;
  A.geom.nx = R.nx;
  A.geom.ny = R.ny;
  A.geom.nz = 1;
  A.alpha = R.coef[1];
  A.gf = R.coef[1] + R.ny;
  A.gb = R.coef[1] + 2 * R.ny;
  A.ptab = R.ptab[1];
  A.cdepth = R.cdepth[1];
  A.cpts = R.cpts[1];
  colsweep_body<T, false, false, SEG, (SEG * sizeof(T) <= 64)>(A, it.L0, reinterpret_cast<c2_t<T>*>(bsmem_raw), cf, cb, red_smem);
}

// ---------------------------------------------------------------- one persistent launch
// Every x and y sweep of every run over nsteps steps in one launch (FP32
// states).  Work items (step t, axis, run, 32-line tile) are numbered step by
// step -- the x items of all runs, then the y items of all runs -- and claimed
// in that order from one counter by persistent CTAs.  An x item of run r at
// step t needs every y item of run r at step t - 1 to have finished, a y item
// every x item of run r at step t (per-run completion counters, counted over
// the whole launch): a run's sweeps follow each other while different runs'
// sweeps overlap, with no grid-wide barrier.  Because items are claimed in
// order and every dependency has a lower number, the lowest unfinished item
// always has its inputs ready, so the waits end.  Each wait is bounded by the
// global timer: past the limit the CTA records the error and every CTA stops
// claiming; the host returns GP_ERR_TIMEOUT at the next gp_batch_observables.
// The per-line arithmetic is that of the per-class launches (the same bodies
// and segment lengths), so the states are bit for bit the same.
struct PersistArgs {
  const BatchRun<float>* runs;
  const BatchItem* items;  // the x items of one step, then its y items
  int nx_items, ny_items;
  const int* per_run;      // [2 run]: x items, y items of the run per step
  const int* seg;          // [2 run]: segment length of the run's x, y lines
  unsigned* next;          // claim counter
  unsigned* done;          // [2 run]: x, y items of the run finished in this launch
  long nsteps;
  int stall;               // added to every dependency target (0; a test makes the waits run out)
  unsigned long long limit_ns;
  int* err;                // device error flag: 1 = a wait ran out
  float dt;
};

__device__ __forceinline__ unsigned long long batch_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until *c >= target, for at most limit_ns of global time; gives up at
// once when another CTA has recorded an error.
__device__ __forceinline__ bool wait_count(const unsigned* c, unsigned target, unsigned long long limit_ns,
                                           const int* err) {
  if (ld_acquire(c) >= target) return true;
  const unsigned long long t0 = batch_ns();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire(c) >= target) return true;
    if (*(const volatile int*)err != 0 || batch_ns() - t0 > limit_ns) return false;
  }
}

__global__ void __launch_bounds__(512) batch_persist_kernel(PersistArgs P) {
  extern __shared__ __align__(16) unsigned char bsmem_raw[];
  __shared__ float2 cf[16][33], cb[16][33];
  __shared__ double red_smem[32];
  __shared__ long s_item;
  __shared__ int s_stop;
  const long per_step = (long)P.nx_items + P.ny_items;
  const long total = per_step * P.nsteps;
  for (;;) {
    if (threadIdx.x == 0) {
      long i = -1;
      if (*(volatile int*)P.err == 0) i = (long)atomicAdd(P.next, 1u);
      s_item = i;
    }
    __syncthreads();
    const long i = s_item;
    if (i < 0 || i >= total) break;
    const long t = i / per_step;
    const int j = (int)(i - t * per_step);
    const bool xs = j < P.nx_items;
    const BatchItem it = P.items[j];
    const int r = it.run;
    if (threadIdx.x == 0) {
      // x items of step t wait for the run's y items of step t - 1, y items
      // for the run's x items of step t
      const unsigned target = xs ? (unsigned)(t * P.per_run[2 * r + 1]) : (unsigned)((t + 1) * P.per_run[2 * r]);
      int stop = 0;
      if (target > 0 && !wait_count(P.done + 2 * r + (xs ? 1 : 0), target + (unsigned)P.stall, P.limit_ns, P.err)) {
        atomicExch(P.err, 1);
        stop = 1;
      }
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    __threadfence();  // the inputs other CTAs wrote are seen by every thread
    const BatchRun<float>& R = P.runs[r];
    Sweep2Args<float> A;
    memset(&A, 0, sizeof(A));
    A.psi = R.psi;
    A.geom.nx = R.nx;
    A.geom.ny = R.ny;
    A.geom.nz = 1;
    float2* sm = reinterpret_cast<float2*>(bsmem_raw);
    const int seg = P.seg[2 * r + (xs ? 0 : 1)];
    if (xs) {
      A.geom.axis = 0;
      A.geom.n = R.nx;
      A.geom.stride = 1;
      A.geom.nlines = R.ny;
      A.alpha = R.coef[0];
      A.gf = R.coef[0] + R.nx;
      A.gb = R.coef[0] + 2 * R.nx;
      A.ptab = R.ptab[0];
      A.cdepth = R.cdepth[0];
      A.cpts = R.cpts[0];
      A.fx = R.fx;
      A.fy = R.fy;
      A.fz = R.fz1;
      A.dtg = R.dtg;
      A.vx = R.vx;
      A.vy = R.vy;
      A.vz = R.vz0;
      A.dt = P.dt;
      A.g = R.g;
      switch (seg) {
        case 4: tsweep_body<float, false, true, false, 4>(A, it.L0, sm, cf, cb, red_smem); break;
        case 8: tsweep_body<float, false, true, false, 8>(A, it.L0, sm, cf, cb, red_smem); break;
        case 16: tsweep_body<float, false, true, false, 16>(A, it.L0, sm, cf, cb, red_smem); break;
        default: tsweep_body<float, false, true, false, 32>(A, it.L0, sm, cf, cb, red_smem); break;
      }
    } else {
      A.geom.axis = 1;
      A.geom.n = R.ny;
      A.geom.stride = R.nx;
      A.geom.nlines = R.nx;
      A.alpha = R.coef[1];
      A.gf = R.coef[1] + R.ny;
      A.gb = R.coef[1] + 2 * R.ny;
      A.ptab = R.ptab[1];
      A.cdepth = R.cdepth[1];
      A.cpts = R.cpts[1];
      switch (seg) {  // registers kept for the segment as the per-class launches do (8 floats or fewer)
        case 4: colsweep_body<float, false, false, 4, true>(A, it.L0, sm, cf, cb, red_smem); break;
        case 8: colsweep_body<float, false, false, 8, true>(A, it.L0, sm, cf, cb, red_smem); break;
        case 16: colsweep_body<float, false, false, 16, true>(A, it.L0, sm, cf, cb, red_smem); break;
        default: colsweep_body<float, false, false, 32, false>(A, it.L0, sm, cf, cb, red_smem); break;
      }
    }
    __syncthreads();  // every thread's writes of the item are done ...
    if (threadIdx.x == 0) {
      __threadfence();  // ... and visible before the item is counted
      atomicAdd(P.done + 2 * r + (xs ? 0 : 1), 1u);
    }
  }
}

// Segment-length classes: a line of n points goes to the first class whose
// segment length gives at most 16 segments (the rule the single-grid handle
// uses), so a run in a batch takes the same arithmetic as alone.  x lines
// whose tile does not fit in shared memory form a fifth class, run one warp
// per line (segment length = the smallest power of two >= (n-2)/32).
constexpr int kNumClasses = 5;
constexpr int kClassSegs[4] = {4, 8, 16, 32};
constexpr int kBatchGraphSteps = 16;

}  // namespace gpe

struct gp_batch {
  int nruns = 0, prec = GP_F64;
  size_t esize = 0;
  double dt = 0;
  std::vector<int> n;        // [nruns][2]
  std::vector<double> dx;    // [nruns][2]
  std::vector<double> nk;    // [nruns][2]
  std::vector<double> g;     // [nruns]
  std::vector<long> off;     // element offset of each run's state
  long total = 0;
  cudaStream_t user = nullptr, work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void* psi = nullptr;
  void* runs_d = nullptr;
  void* items_d[2][5] = {{nullptr}};  // [axis][class]
  int nitems[2][5] = {{0}};
  int class_n[2][5] = {{0}};          // longest line of the class
  int warp_seg = 16;                  // segment length of the warp-per-line class
  std::string launch_err;             // first failed launch of the current call
  // FP64 observables: per-run tables
  std::vector<void*> vd, cdx, wd;     // [nruns][2] device arrays, observables' arithmetic type
  void* ztab = nullptr;               // the absent z axis: v = c = 0 (slot 0), w = 1 (slot 1)
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  // one reduction launch for every run: per-run arguments, (run, block,
  // blocks, tx_log2) items, each run's first item, weight factors, per-item sums
  void* obs_runs_d = nullptr;
  void* obs_items_d = nullptr;
  int* obs_first_d = nullptr;
  double* obs_ws_d = nullptr;
  double* obs_parts = nullptr;
  int nobs_items = 0;
  double* obs_out = nullptr;
  double* obs_host = nullptr;
  void* stage = nullptr;  // double-float state: the states as complex128 (exchange, observables)
  cudaGraphExec_t graph = nullptr;
  // the one-launch form (FP32): items of one step, per-run item counts and
  // segment lengths, the claim counter and per-run completion counters
  bool persistent = false;
  void* p_items = nullptr;
  int p_nx = 0, p_ny = 0;
  int* p_per_run = nullptr;
  int* p_seg = nullptr;
  unsigned* p_count = nullptr;  // [1 + 2 nruns]: next, done
  size_t p_smem = 0;
  int p_threads = 32;           // 32 x the most segments of any line
  int p_stall = 0;
  unsigned long long limit_ns = 1000000000ull;
  int* dev_err = nullptr;
  std::vector<void*> allocs;
};

namespace gpe {
namespace {

int b_alloc(gp_batch* b, void** p, size_t bytes) {
  const size_t sz = bytes < 16 ? 16 : bytes;
  GP_CUDA(guarded_malloc(p, sz));
  b->allocs.push_back(*p);
  GP_CUDA(cudaMemsetAsync(*p, 0, sz, b->work));
  return GP_OK;
}

template <typename T>
int b_upload(gp_batch* b, void* dst, const std::vector<T>& v) {
  GP_CUDA(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->work));
  GP_CUDA(cudaStreamSynchronize(b->work));
  return GP_OK;
}

bool x_tile_fits(int n, size_t esize) { return (36L * n + 512) * (long)esize <= 200L * 1024; }

// class of a line of n points along axis a; class 4 = warp-per-line x lines
int class_of(int n, int a, size_t esize) {
  if (a == 0 && !x_tile_fits(n, esize)) return 4;
  const int M = n - 2;
  for (int c = 0; c < 4; ++c)
    if ((M + kClassSegs[c] - 1) / kClassSegs[c] <= 16) return c;
  return -1;
}

int warp_seg_of(int n) {
  for (int s : {1, 2, 4, 8, 16})
    if (32 * s >= n - 2) return s;
  return 16;
}

template <typename T>
int build_tables(gp_batch* b) {
  const int R = b->nruns;
  // one segment length for every warp-per-line x line: enough for the longest
  int nwarp = 0;
  for (int r = 0; r < R; ++r)
    if (class_of(b->n[2 * r], 0, b->esize) == 4) nwarp = std::max(nwarp, b->n[2 * r]);
  b->warp_seg = nwarp ? warp_seg_of(nwarp) : 16;
  // coefficients: per run per axis 3n (alpha | gf | gb) + 512 carry tables
  std::vector<size_t> coff(2 * R), poff(2 * R);
  size_t ctot = 0;
  for (int r = 0; r < R; ++r)
    for (int a = 0; a < 2; ++a) {
      coff[2 * r + a] = ctot;
      ctot += 3 * (size_t)b->n[2 * r + a];
      poff[2 * r + a] = ctot;
      ctot += 512;
    }
  std::vector<T> cbuf(2 * ctot, T(0));
  size_t vtot = 0;
  std::vector<size_t> voff(2 * R);
  for (int r = 0; r < R; ++r)
    for (int a = 0; a < 2; ++a) {
      voff[2 * r + a] = vtot;
      vtot += b->n[2 * r + a];
    }
  std::vector<T> vbuf(2 * (vtot + 1), T(0));  // complex factors; last entry: the shared 1 for the absent z axis
  vbuf[2 * vtot] = T(1);
  std::vector<T> pbuf(vtot + 1, T(0));        // potentials; last entry: the shared 0 for the absent z axis
  std::vector<int> reach_d(2 * R, 0), reach_p(2 * R, 0);
  for (int r = 0; r < R; ++r)
    for (int a = 0; a < 2; ++a) {
      const int n = b->n[2 * r + a];
      const double h = b->dx[2 * r + a];
      const AxisFactors f = thomas_factors(n, b->dt / (4.0 * h * h), false);
      const int cls = class_of(n, a, b->esize);
      const int seg = cls == 4 ? b->warp_seg : kClassSegs[cls];
      std::vector<cd> gf, gb;
      segment_products(f.alpha, n, seg, gf, gb);
      cd tabs[512];
      carry_tables(f.alpha, n, seg, tabs);
      carry_reach(gf.data(), gb.data(), tabs, n, seg, 1, std::ldexp(1.0, std::is_same<T, float>::value ? -48 : -64),
                  reach_d[2 * r + a], reach_p[2 * r + a]);
      T* c = cbuf.data() + 2 * coff[2 * r + a];
      for (int k = 0; k < n; ++k) {
        c[2 * k] = (T)f.alpha[k].real(); c[2 * k + 1] = (T)f.alpha[k].imag();
        c[2 * (n + k)] = (T)gf[k].real(); c[2 * (n + k) + 1] = (T)gf[k].imag();
        c[2 * (2 * n + k)] = (T)gb[k].real(); c[2 * (2 * n + k) + 1] = (T)gb[k].imag();
      }
      T* pt = cbuf.data() + 2 * poff[2 * r + a];
      for (int q = 0; q < 512; ++q) { pt[2 * q] = (T)tabs[q].real(); pt[2 * q + 1] = (T)tabs[q].imag(); }
      const double w = b->nk[2 * r + a];
      for (int i = 0; i < n; ++i) {
        const double x = axis_coord(0, a, n, h, i);  // the single-grid handle's coordinates, bit for bit
        const double v = 0.5 * w * w * x * x;
        vbuf[2 * (voff[2 * r + a] + i)] = (T)std::cos(b->dt * v);
        vbuf[2 * (voff[2 * r + a] + i) + 1] = (T)(-std::sin(b->dt * v));
        pbuf[voff[2 * r + a] + i] = (T)v;
      }
    }
  void *cdev = nullptr, *vdev = nullptr, *pdev = nullptr, *tdev = nullptr;
  int rc;
  if constexpr (std::is_same<T, df64>::value) {
    // the double-float state takes the FP64 factors as exact triple-floats,
    // split from the same doubles as the single-grid handle's
    std::vector<tf3c> tbuf(vtot);
    for (int r = 0; r < R; ++r)
      for (int a = 0; a < 2; ++a) {
        const int n = b->n[2 * r + a];
        const double h = b->dx[2 * r + a], w = b->nk[2 * r + a];
        for (int i = 0; i < n; ++i) {
          const double x = axis_coord(0, a, n, h, i);
          const double v = 0.5 * w * w * x * x;
          tf3c& f = tbuf[voff[2 * r + a] + i];
          tf_split(std::cos(b->dt * v), f.re);
          tf_split(-std::sin(b->dt * v), f.im);
        }
      }
    if ((rc = b_alloc(b, &tdev, tbuf.size() * sizeof(tf3c))) || (rc = b_upload<tf3c>(b, tdev, tbuf))) return rc;
  }
  if ((rc = b_alloc(b, &pdev, pbuf.size() * sizeof(T)))) return rc;
  if ((rc = b_upload<T>(b, pdev, pbuf))) return rc;
  if ((rc = b_alloc(b, &cdev, cbuf.size() * sizeof(T)))) return rc;
  if ((rc = b_upload<T>(b, cdev, cbuf))) return rc;
  if ((rc = b_alloc(b, &vdev, vbuf.size() * sizeof(T)))) return rc;
  if ((rc = b_upload<T>(b, vdev, vbuf))) return rc;
  std::vector<BatchRun<T>> runs(R);
  for (int r = 0; r < R; ++r) {
    BatchRun<T>& q = runs[r];
    q.psi = (c2_t<T>*)b->psi + b->off[r];
    q.nx = b->n[2 * r];
    q.ny = b->n[2 * r + 1];
    for (int a = 0; a < 2; ++a) {
      q.coef[a] = (const c2_t<T>*)cdev + coff[2 * r + a];
      q.ptab[a] = (const c2_t<T>*)cdev + poff[2 * r + a];
    }
    q.fx = (const c2_t<T>*)vdev + voff[2 * r];
    q.fy = (const c2_t<T>*)vdev + voff[2 * r + 1];
    q.fz1 = (const c2_t<T>*)vdev + vtot;
    q.dtg = (T)(b->dt * b->g[r]);
    q.vx = (const T*)pdev + voff[2 * r];
    q.vy = (const T*)pdev + voff[2 * r + 1];
    q.vz0 = (const T*)pdev + vtot;
    q.g = (T)b->g[r];
    q.tfx = tdev ? (const tf3c*)tdev + voff[2 * r] : nullptr;
    q.tfy = tdev ? (const tf3c*)tdev + voff[2 * r + 1] : nullptr;
    for (int a = 0; a < 2; ++a) {
      q.cdepth[a] = reach_d[2 * r + a];
      q.cpts[a] = carry_pts_class(reach_p[2 * r + a]);
    }
  }
  if ((rc = b_alloc(b, &b->runs_d, R * sizeof(BatchRun<T>)))) return rc;
  GP_CUDA(cudaMemcpyAsync(b->runs_d, runs.data(), R * sizeof(BatchRun<T>), cudaMemcpyHostToDevice, b->work));
  GP_CUDA(cudaStreamSynchronize(b->work));
  // work items per axis and class: (run, first line of a 32-line tile)
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < kNumClasses; ++c) {
      std::vector<BatchItem> items;
      int nmax = 0;
      const int step = c == 4 ? 4 : 32;         // lines per block
      for (int r = 0; r < R; ++r) {
        const int n = b->n[2 * r + a];          // line length along axis a
        const int nl = b->n[2 * r + (1 - a)];   // number of lines
        if (class_of(n, a, b->esize) != c) continue;
        nmax = std::max(nmax, n);
        for (int L0 = 0; L0 < nl; L0 += step) items.push_back({r, L0});
      }
      b->nitems[a][c] = (int)items.size();
      b->class_n[a][c] = nmax;
      if (items.empty()) continue;
      if ((rc = b_alloc(b, &b->items_d[a][c], items.size() * sizeof(BatchItem)))) return rc;
      GP_CUDA(cudaMemcpyAsync(b->items_d[a][c], items.data(), items.size() * sizeof(BatchItem),
                              cudaMemcpyHostToDevice, b->work));
      GP_CUDA(cudaStreamSynchronize(b->work));
    }
  if constexpr (std::is_same<T, float>::value) {
    // the one-launch form: the x tiles of every run, then the y tiles (the
    // largest runs first, so that the launch does not end on a large item)
    std::vector<int> order(R);
    for (int r = 0; r < R; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int a_, int b_) {
      return (long)b->n[2 * a_] * b->n[2 * a_ + 1] > (long)b->n[2 * b_] * b->n[2 * b_ + 1];
    });
    std::vector<BatchItem> items;
    std::vector<int> per_run(2 * R, 0), segs(2 * R, 0);
    size_t smem = 0;
    for (int a = 0; a < 2; ++a)
      for (int r : order) {
        const int n = b->n[2 * r + a], nl = b->n[2 * r + (1 - a)];
        segs[2 * r + a] = kClassSegs[class_of(n, a, b->esize)];
        for (int L0 = 0; L0 < nl; L0 += 32) items.push_back({r, L0});
        per_run[2 * r + a] = (nl + 31) / 32;
        b->p_threads = std::max(b->p_threads, 32 * ((n - 2 + segs[2 * r + a] - 1) / segs[2 * r + a]));
        smem = std::max(smem, (a == 0 ? (size_t)(36 * n + 512) : (size_t)(3 * n + 512)) * sizeof(float2));
        (a == 0 ? b->p_nx : b->p_ny) += (nl + 31) / 32;
      }
    b->p_smem = smem;
    if ((rc = b_alloc(b, &b->p_items, items.size() * sizeof(BatchItem))) ||
        (rc = b_upload<BatchItem>(b, b->p_items, items)))
      return rc;
    void* q = nullptr;
    if ((rc = b_alloc(b, &q, per_run.size() * sizeof(int))) || (rc = b_upload<int>(b, q, per_run))) return rc;
    b->p_per_run = (int*)q;
    if ((rc = b_alloc(b, &q, segs.size() * sizeof(int))) || (rc = b_upload<int>(b, q, segs))) return rc;
    b->p_seg = (int*)q;
    if ((rc = b_alloc(b, &q, (1 + 2 * (size_t)R) * sizeof(unsigned)))) return rc;
    b->p_count = (unsigned*)q;
  }
  return GP_OK;
}

// The one-launch form over nsteps steps: counters cleared, one launch.
void enqueue_persistent(gp_batch* b, long nsteps) {
  cudaMemsetAsync(b->p_count, 0, (1 + 2 * (size_t)b->nruns) * sizeof(unsigned), b->work);
  opt_in_smem((const void*)batch_persist_kernel, b->p_smem);
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persist_kernel, b->p_threads, b->p_smem);
  PersistArgs P;
  P.runs = (const BatchRun<float>*)b->runs_d;
  P.items = (const BatchItem*)b->p_items;
  P.nx_items = b->p_nx;
  P.ny_items = b->p_ny;
  P.per_run = b->p_per_run;
  P.seg = b->p_seg;
  P.next = b->p_count;
  P.done = b->p_count + 1;
  P.nsteps = nsteps;
  P.stall = b->p_stall;
  P.limit_ns = b->limit_ns;
  P.err = b->dev_err;
  P.dt = (float)b->dt;
  const long items = ((long)b->p_nx + b->p_ny) * nsteps;
  const int blocks = (int)std::max(1L, std::min<long>(items, (long)std::max(1, per_sm) * std::max(1, sms)));
  batch_persist_kernel<<<blocks, b->p_threads, b->p_smem, b->work>>>(P);
  count_launch();
}

template <typename T, int SEG>
void launch_batch_warp(gp_batch* b) {
  const auto* runs = (const BatchRun<T>*)b->runs_d;
  const auto* items = (const BatchItem*)b->items_d[0][4];
  batch_xw_kernel<T, SEG><<<b->nitems[0][4], 128, 0, b->work>>>(runs, items, (T)b->dt);
  count_launch();
}

template <typename T, int SEG>
void launch_batch_class(gp_batch* b, int a, int c) {
  const int n = b->class_n[a][c];
  const int threads = 32 * ((n - 2 + SEG - 1) / SEG);
  const auto* runs = (const BatchRun<T>*)b->runs_d;
  const auto* items = (const BatchItem*)b->items_d[a][c];
  if (a == 0) {
    const size_t smem = (size_t)(36 * n + 512) * sizeof(c2_t<T>);
    opt_in_smem((const void*)batch_x_kernel<T, SEG>, 200 * 1024);
    batch_x_kernel<T, SEG><<<b->nitems[a][c], threads, smem, b->work>>>(runs, items, (T)b->dt);
  } else {
    const size_t smem = (size_t)(3 * n + 512) * sizeof(c2_t<T>);
    opt_in_smem((const void*)batch_y_kernel<T, SEG>, 64 * 1024);  // static + dynamic can pass 48 KB
    batch_y_kernel<T, SEG><<<b->nitems[a][c], threads, smem, b->work>>>(runs, items);
  }
  count_launch();
}

void note_launch(gp_batch* b, int a, int c) {
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess && b->launch_err.empty())
    b->launch_err = std::string("batch sweep axis ") + std::to_string(a) + " class " + std::to_string(c) +
                    " (longest line " + std::to_string(b->class_n[a][c]) + ", " + std::to_string(b->nitems[a][c]) +
                    " blocks): " + cudaGetErrorString(e);
}

template <typename T>
void enqueue_batch_step(gp_batch* b) {
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < kNumClasses; ++c) {
      if (!b->nitems[a][c]) continue;
      struct Note {
        gp_batch* b; int a, c;
        ~Note() { note_launch(b, a, c); }
      } note{b, a, c};
      switch (c) {
        case 0: launch_batch_class<T, 4>(b, a, c); break;
        case 1: launch_batch_class<T, 8>(b, a, c); break;
        case 2: launch_batch_class<T, 16>(b, a, c); break;
        case 3: launch_batch_class<T, 32>(b, a, c); break;
        default:
          switch (b->warp_seg) {
            case 1: launch_batch_warp<T, 1>(b); break;
            case 2: launch_batch_warp<T, 2>(b); break;
            case 4: launch_batch_warp<T, 4>(b); break;
            case 8: launch_batch_warp<T, 8>(b); break;
            default: launch_batch_warp<T, 16>(b); break;
          }
      }
    }
}

int launches_per_step(const gp_batch* b) {
  int k = 0;
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < kNumClasses; ++c) k += b->nitems[a][c] > 0;
  return k;
}

int b_join_in(gp_batch* b) {
  GP_CUDA(cudaEventRecord(b->ev_in, b->user));
  GP_CUDA(cudaStreamWaitEvent(b->work, b->ev_in, 0));
  return GP_OK;
}

int b_join_out(gp_batch* b) {
  GP_CUDA(cudaEventRecord(b->ev_out, b->work));
  GP_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  return GP_OK;
}

template <typename T>
int batch_steps(gp_batch* b, long nsteps) {
  if (nsteps == 0) return GP_OK;
  int rc = b_join_in(b);
  if (rc) return rc;
  b->launch_err.clear();
  long t = 0;
  if (nsteps >= 2 * kBatchGraphSteps) {
    if (!b->graph) {
      cudaGraph_t graph;
      GP_CUDA(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal));
      const unsigned long long before = g_launches.load();
      if (b->persistent) enqueue_persistent(b, kBatchGraphSteps);
      else
        for (int s = 0; s < kBatchGraphSteps; ++s) enqueue_batch_step<T>(b);
      g_launches.store(before);
      const cudaError_t ce = cudaStreamEndCapture(b->work, &graph);
      if (ce != cudaSuccess)
        return fail(GP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce) +
                                     (b->launch_err.empty() ? "" : "; " + b->launch_err));
      cudaError_t e = cudaGraphInstantiate(&b->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return fail(GP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
    }
    for (; nsteps - t >= kBatchGraphSteps; t += kBatchGraphSteps) {
      GP_CUDA(cudaGraphLaunch(b->graph, b->work));
      count_launch(b->persistent ? 1ull : (unsigned long long)kBatchGraphSteps * launches_per_step(b));
    }
  }
  if (b->persistent && nsteps > t) enqueue_persistent(b, nsteps - t);
  else
    for (; t < nsteps; ++t) enqueue_batch_step<T>(b);
  if (!b->launch_err.empty()) return fail(GP_ERR_CUDA, b->launch_err);
  GP_CUDA(cudaGetLastError());
  return b_join_out(b);
}

// Arguments and items of the one-launch reduction over all runs (built once).
template <typename T>
int build_obs(gp_batch* b) {
  std::vector<ObsArgs<T>> runs(b->nruns);
  std::vector<int4> items;
  std::vector<int> first(b->nruns + 1, 0);
  std::vector<double> ws(b->nruns);
  for (int r = 0; r < b->nruns; ++r) {
    ObsArgs<T>& a = runs[r];
    std::memset(&a, 0, sizeof(a));
    a.psi = (const c2_t<T>*)(b->stage ? b->stage : b->psi) + b->off[r];  // double-float: its complex128 copy
    a.dim = 2;
    a.nx = b->n[2 * r];
    a.ny = b->n[2 * r + 1];
    a.nz = 1;
    a.hx = b->dx[2 * r];
    a.hy = b->dx[2 * r + 1];
    a.hz = 1.0;
    using R = obs_r<T>;
    a.vx = (const R*)b->vd[2 * r]; a.vy = (const R*)b->vd[2 * r + 1];
    a.cx = (const R*)b->cdx[2 * r]; a.cy = (const R*)b->cdx[2 * r + 1];
    a.wx = (const R*)b->wd[2 * r]; a.wy = (const R*)b->wd[2 * r + 1];
    a.vz = (const R*)b->ztab;
    a.cz = (const R*)b->ztab;
    a.wz = (const R*)b->ztab + 1;
    a.wscale = b->dx[2 * r] * b->dx[2 * r + 1] / 9.0;  // the tables hold the Simpson coefficients
    ws[r] = a.wscale;
    // rows of 32..256 threads; up to 32 blocks per run (10-100 points per thread on the largest grids)
    const int lg = obs_tx_log2(a.nx), rpb = kObsThreads >> lg;
    const int nblk = std::max(1, std::min(32, (a.ny + rpb - 1) / rpb));
    first[r] = (int)items.size();
    for (int k = 0; k < nblk; ++k) items.push_back(make_int4(r, k, nblk, lg));
  }
  first[b->nruns] = (int)items.size();
  b->nobs_items = (int)items.size();
  int rc;
  if ((rc = b_alloc(b, &b->obs_runs_d, runs.size() * sizeof(ObsArgs<T>))) ||
      (rc = b_upload<ObsArgs<T>>(b, b->obs_runs_d, runs)))
    return rc;
  if ((rc = b_alloc(b, &b->obs_items_d, items.size() * sizeof(int4))) || (rc = b_upload<int4>(b, b->obs_items_d, items)))
    return rc;
  void* p = nullptr;
  if ((rc = b_alloc(b, &p, first.size() * sizeof(int))) || (rc = b_upload<int>(b, p, first))) return rc;
  b->obs_first_d = (int*)p;
  if ((rc = b_alloc(b, &p, ws.size() * sizeof(double))) || (rc = b_upload<double>(b, p, ws))) return rc;
  b->obs_ws_d = (double*)p;
  if ((rc = b_alloc(b, &p, 8 * items.size() * sizeof(double)))) return rc;
  b->obs_parts = (double*)p;
  return GP_OK;
}

// Observables of every run: one launch over all runs' blocks, one to finish.
template <typename T>
int batch_observables(gp_batch* b) {
  batch_obs_kernel<T><<<b->nobs_items, kObsThreads, 0, b->work>>>((const ObsArgs<T>*)b->obs_runs_d,
                                                                    (const int4*)b->obs_items_d, b->obs_parts);
  count_launch();
  obs_finish_kernel<<<b->nruns, kObsThreads, 0, b->work>>>(b->obs_parts, b->obs_first_d, b->obs_ws_d, b->obs_out);
  count_launch();
  GP_CUDA(cudaGetLastError());
  return GP_OK;
}

}  // namespace
}  // namespace gpe

using namespace gpe;

extern "C" {

int gp_batch_destroy(gp_batch* b) {
  if (!b) return GP_OK;
  if (b->work) cudaStreamSynchronize(b->work);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->allocs) guarded_free(p);
  if (b->obs_host) cudaFreeHost(b->obs_host);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->work) cudaStreamDestroy(b->work);
  delete b;
  return GP_OK;
}

int gp_batch_init(gp_batch** out, int nruns, const int* n, const double* dx, double dt, const double* nkl,
                  const double* g, gp_precision prec, void* stream) {
  g_err.clear();
  if (!out || !n || !dx || !nkl || !g) return fail(GP_ERR_INVALID, "gp_batch_init: NULL argument");
  *out = nullptr;
  if (nruns < 1 || nruns > 65536) return fail(GP_ERR_INVALID, "gp_batch_init: nruns must be in [1, 65536]");
  if (prec != GP_F64 && prec != GP_F32 && prec != GP_DF64) return fail(GP_ERR_INVALID, "gp_batch_init: unknown precision");
  if (!std::isfinite(dt) || dt == 0.0) return fail(GP_ERR_INVALID, "gp_batch_init: dt must be finite and nonzero");
  long total = 0;
  for (int r = 0; r < nruns; ++r) {
    for (int a = 0; a < 2; ++a) {
      const int na = n[2 * r + a];
      if (na < 3 || na > 514) return fail(GP_ERR_INVALID, "gp_batch_init: every axis needs 3 <= n <= 514 points");
      if (!(dx[2 * r + a] > 0.0) || !std::isfinite(dx[2 * r + a]))
        return fail(GP_ERR_INVALID, "gp_batch_init: dx must be finite and > 0");
      if (!std::isfinite(nkl[2 * r + a])) return fail(GP_ERR_INVALID, "gp_batch_init: trap frequencies must be finite");
    }
    if (!std::isfinite(g[r])) return fail(GP_ERR_INVALID, "gp_batch_init: g must be finite");
    total += (long)n[2 * r] * n[2 * r + 1];
    if (total > 2147483647L) return fail(GP_ERR_INVALID, "gp_batch_init: more than 2^31-1 points in all");
  }
  gp_batch* b = new gp_batch();
  b->nruns = nruns;
  b->prec = prec;
  b->esize = prec == GP_F64 ? sizeof(double2) : prec == GP_DF64 ? sizeof(df64x2) : sizeof(float2);
  b->dt = dt;
  b->n.assign(n, n + 2 * nruns);
  b->dx.assign(dx, dx + 2 * nruns);
  b->nk.assign(nkl, nkl + 2 * nruns);
  b->g.assign(g, g + nruns);
  b->off.resize(nruns);
  long acc = 0;
  for (int r = 0; r < nruns; ++r) {
    b->off[r] = acc;
    acc += (long)n[2 * r] * n[2 * r + 1];
  }
  b->total = acc;
  b->user = (cudaStream_t)stream;
  auto bail = [&](int code) { gp_batch_destroy(b); return code; };
  {
    cudaError_t e = cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->obs_host, 8 * sizeof(double) * (nruns + 1));
    if (e != cudaSuccess) return bail(fail(GP_ERR_CUDA, std::string("gp_batch_init: ") + cudaGetErrorString(e)));
  }
  int rc;
  if ((rc = b_alloc(b, &b->psi, (size_t)acc * b->esize))) return bail(rc);
  if (prec == GP_DF64 && (rc = b_alloc(b, &b->stage, (size_t)acc * sizeof(double2)))) return bail(rc);
  rc = prec == GP_F64 ? build_tables<double>(b) : prec == GP_DF64 ? build_tables<df64>(b) : build_tables<float>(b);
  if (rc) return bail(rc);
  const bool obs64 = prec != GP_F32;  // the observables' arithmetic (double-float: on the complex128 copy)
  // tables of the observables, per run and axis, in their arithmetic type
  b->vd.resize(2 * nruns);
  b->cdx.resize(2 * nruns);
  b->wd.resize(2 * nruns);
  for (int r = 0; r < nruns; ++r)
    for (int a = 0; a < 2; ++a) {
      const int na = n[2 * r + a];
      const double h = dx[2 * r + a], w = nkl[2 * r + a];
      std::vector<double> x(na), v(na), wt(na);
      const int m = (na % 2 == 1) ? na : na - 1;
      for (int i = 0; i < na; ++i) {
        x[i] = axis_coord(0, a, na, h, i);
        v[i] = 0.5 * w * w * x[i] * x[i];
        double c = 0.0;
        if (i < m) c = (i == 0 || i == m - 1) ? 1.0 : (i % 2 == 1 ? 4.0 : 2.0);
        wt[i] = c;  // exact; the factor h/3 per axis is applied to the FP64 totals
      }
      void *pv, *pc, *pw;
      const size_t rs = obs64 ? sizeof(double) : sizeof(float);
      auto up = [&](void* dst, const std::vector<double>& src) {
        return obs64 ? b_upload<double>(b, dst, src)
                     : b_upload<float>(b, dst, std::vector<float>(src.begin(), src.end()));
      };
      if ((rc = b_alloc(b, &pv, na * rs)) || (rc = up(pv, v))) return bail(rc);
      if ((rc = b_alloc(b, &pc, na * rs)) || (rc = up(pc, x))) return bail(rc);
      if ((rc = b_alloc(b, &pw, na * rs)) || (rc = up(pw, wt))) return bail(rc);
      b->vd[2 * r + a] = pv;
      b->cdx[2 * r + a] = pc;
      b->wd[2 * r + a] = pw;
    }
  {
    const std::vector<double> zw = {0.0, 1.0};
    if ((rc = b_alloc(b, &b->ztab, 2 * sizeof(double)))) return bail(rc);
    if ((rc = obs64 ? b_upload<double>(b, b->ztab, zw)
                    : b_upload<float>(b, b->ztab, std::vector<float>(zw.begin(), zw.end()))))
      return bail(rc);
  }
  if ((rc = b_alloc(b, (void**)&b->partials, 152L * 16 * 8 * sizeof(double)))) return bail(rc);
  if ((rc = b_alloc(b, (void**)&b->counter, 64))) return bail(rc);
  if ((rc = b_alloc(b, (void**)&b->dev_err, 64))) return bail(rc);
  {
    const char* lim = std::getenv("GPE_WAIT_LIMIT_MS");
    const long ms = lim ? std::atol(lim) : 1000;
    b->limit_ns = (unsigned long long)(ms > 0 ? ms : 1000) * 1000000ull;
  }
  if ((rc = b_alloc(b, (void**)&b->obs_out, (8L * nruns + 8) * sizeof(double)))) return bail(rc);
  if ((rc = obs64 ? build_obs<double>(b) : build_obs<float>(b))) return bail(rc);
  *out = b;
  return GP_OK;
}

long gp_batch_offset(const gp_batch* b, int run) {
  if (!b || run < 0 || run >= b->nruns) return -1;
  return b->off[run];
}

int gp_batch_set_state(gp_batch* b, int run, const void* psi, int on_device) {
  if (!b || !psi) return fail(GP_ERR_INVALID, "gp_batch_set_state: NULL argument");
  if (run < -1 || run >= b->nruns) return fail(GP_ERR_INVALID, "gp_batch_set_state: run out of range");
  int rc = b_join_in(b);
  if (rc) return rc;
  const long off = run < 0 ? 0 : b->off[run];
  const long cnt = run < 0 ? b->total : (long)b->n[2 * run] * b->n[2 * run + 1];
  if (b->prec == GP_DF64) {  // complex128 in, split on the device
    const void* src = psi;
    if (!on_device) {
      GP_CUDA(cudaMemcpyAsync((double2*)b->stage + off, psi, (size_t)cnt * sizeof(double2), cudaMemcpyHostToDevice,
                              b->work));
      src = (const double2*)b->stage + off;
    }
    launch_c128_to_df((df64x2*)b->psi + off, src, cnt, b->work);
    GP_CUDA(cudaGetLastError());
  } else {
    GP_CUDA(cudaMemcpyAsync((char*)b->psi + off * b->esize, psi, (size_t)cnt * b->esize,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->work));
  }
  if (!on_device) GP_CUDA(cudaStreamSynchronize(b->work));
  return b_join_out(b);
}

int gp_batch_get_state(gp_batch* b, int run, void* psi, int on_device) {
  if (!b || !psi) return fail(GP_ERR_INVALID, "gp_batch_get_state: NULL argument");
  if (run < -1 || run >= b->nruns) return fail(GP_ERR_INVALID, "gp_batch_get_state: run out of range");
  int rc = b_join_in(b);
  if (rc) return rc;
  const long off = run < 0 ? 0 : b->off[run];
  const long cnt = run < 0 ? b->total : (long)b->n[2 * run] * b->n[2 * run + 1];
  if (b->prec == GP_DF64) {  // rounded to complex128
    void* dst = on_device ? psi : (void*)((double2*)b->stage + off);
    launch_df_to_c128(dst, (const df64x2*)b->psi + off, cnt, b->work);
    GP_CUDA(cudaGetLastError());
    if (!on_device)
      GP_CUDA(cudaMemcpyAsync(psi, dst, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToHost, b->work));
  } else {
    GP_CUDA(cudaMemcpyAsync(psi, (const char*)b->psi + off * b->esize, (size_t)cnt * b->esize,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->work));
  }
  if (!on_device) GP_CUDA(cudaStreamSynchronize(b->work));
  return b_join_out(b);
}

int gp_batch_step_real(gp_batch* b, long nsteps) {
  if (!b) return fail(GP_ERR_INVALID, "gp_batch_step_real: NULL handle");
  if (nsteps < 0) return fail(GP_ERR_INVALID, "gp_batch_step_real: nsteps < 0");
  return b->prec == GP_F64    ? batch_steps<double>(b, nsteps)
         : b->prec == GP_DF64 ? batch_steps<df64>(b, nsteps)
                              : batch_steps<float>(b, nsteps);
}

int gp_batch_observables(gp_batch* b, gp_obs* out) {
  if (!b || !out) return fail(GP_ERR_INVALID, "gp_batch_observables: NULL argument");
  int rc = b_join_in(b);
  if (rc) return rc;
  if (b->prec == GP_DF64) {
    launch_df_to_c128(b->stage, b->psi, b->total, b->work);  // the observables of the rounded states
    GP_CUDA(cudaGetLastError());
  }
  rc = b->prec != GP_F32 ? batch_observables<double>(b) : batch_observables<float>(b);
  if (rc) return rc;
  GP_CUDA(cudaMemcpyAsync(b->obs_host, b->obs_out, 8 * sizeof(double) * b->nruns, cudaMemcpyDeviceToHost, b->work));
  GP_CUDA(cudaMemcpyAsync(b->obs_host + 8L * b->nruns, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost, b->work));
  GP_CUDA(cudaStreamSynchronize(b->work));
  if ((rc = b_join_out(b))) return rc;
  int err = 0;
  std::memcpy(&err, b->obs_host + 8L * b->nruns, sizeof(int));
  if (err) {
    GP_CUDA(cudaMemsetAsync(b->dev_err, 0, sizeof(int), b->work));
    GP_CUDA(cudaStreamSynchronize(b->work));
    return fail(GP_ERR_TIMEOUT, "gp_batch_observables: a step barrier of the one-launch form ran out of time "
                                "(GPE_WAIT_LIMIT_MS); the states are not valid");
  }
  bool finite = true;
  for (int r = 0; r < b->nruns; ++r) {
    const double* S = b->obs_host + 8L * r;
    const double N = S[0];
    gp_obs& o = out[r];
    o.norm = N;
    o.energy = (S[1] + S[2]) / N + 0.5 * b->g[r] * S[3] / (N * N);
    o.mu = (S[1] + S[2]) / N + b->g[r] * S[3] / (N * N);
    o.rms[0] = std::sqrt(S[4] / N);
    o.rms[1] = std::sqrt(S[5] / N);
    o.rms[2] = 0.0;
    o.rms_r = std::sqrt((S[4] + S[5]) / N);
    for (int q = 0; q < 7; ++q) finite = finite && std::isfinite(S[q]);
  }
  if (!finite) return fail(GP_ERR_NONFINITE, "gp_batch_observables: a state holds NaN or Inf");
  return GP_OK;
}

int gp_batch_set_mode(gp_batch* b, int persistent) {
  if (!b) return fail(GP_ERR_INVALID, "gp_batch_set_mode: NULL handle");
  if (persistent != 0 && persistent != 1) return fail(GP_ERR_INVALID, "gp_batch_set_mode: mode must be 0 or 1");
  if (persistent && b->prec != GP_F32)
    return fail(GP_ERR_INVALID, "gp_batch_set_mode: the one-launch form takes FP32 states only");
  if ((bool)persistent != b->persistent) {
    if (b->work) GP_CUDA(cudaStreamSynchronize(b->work));
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->persistent = persistent;
  }
  return GP_OK;
}

int gp_batch_get_mode(const gp_batch* b) { return b ? (int)b->persistent : -1; }

int gp_batch_autotune(gp_batch* b, long nsteps, double* ms_out) {
  if (!b) return fail(GP_ERR_INVALID, "gp_batch_autotune: NULL handle");
  if (nsteps < 1) return fail(GP_ERR_INVALID, "gp_batch_autotune: nsteps < 1");
  if (ms_out) ms_out[0] = ms_out[1] = -1.0;
  if (b->prec != GP_F32) return gp_batch_set_mode(b, 0);  // one form only
  int rc = b_join_in(b);
  if (rc) return rc;
  // the states are kept and put back: timing steps the runs
  void* keep = nullptr;
  GP_CUDA(cudaMallocAsync(&keep, (size_t)b->total * b->esize, b->work));
  GP_CUDA(cudaMemcpyAsync(keep, b->psi, (size_t)b->total * b->esize, cudaMemcpyDeviceToDevice, b->work));
  cudaEvent_t e0, e1;
  GP_CUDA(cudaEventCreate(&e0));
  GP_CUDA(cudaEventCreate(&e1));
  double ms[2] = {0.0, 0.0};
  const bool was = b->persistent;
  for (int m = 0; m < 2 && rc == GP_OK; ++m) {
    if ((rc = gp_batch_set_mode(b, m))) break;
    if ((rc = batch_steps<float>(b, nsteps))) break;  // warm-up (graph capture included)
    cudaEventRecord(e0, b->work);
    if ((rc = batch_steps<float>(b, nsteps))) break;
    cudaEventRecord(e1, b->work);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(GP_ERR_CUDA, "gp_batch_autotune: timing failed"); break; }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms[m] = t;
  }
  int err = 0;
  if (rc == GP_OK) {
    cudaMemcpy(&err, b->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) cudaMemset(b->dev_err, 0, sizeof(int));
  }
  cudaMemcpyAsync(b->psi, keep, (size_t)b->total * b->esize, cudaMemcpyDeviceToDevice, b->work);
  cudaFreeAsync(keep, b->work);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    gp_batch_set_mode(b, was);
    return rc;
  }
  if (err) {
    gp_batch_set_mode(b, 0);
    return fail(GP_ERR_TIMEOUT, "gp_batch_autotune: a step barrier of the one-launch form ran out of time");
  }
  if (ms_out) ms_out[0] = ms[0], ms_out[1] = ms[1];
  if ((rc = gp_batch_set_mode(b, ms[1] < ms[0] ? 1 : 0))) return rc;
  return b_join_out(b);
}

int gp_test_batch_stall(gp_batch* b, int extra) {
  if (!b) return fail(GP_ERR_INVALID, "gp_test_batch_stall: NULL handle");
  if (extra < 0 || extra > (1 << 20)) return fail(GP_ERR_INVALID, "gp_test_batch_stall: extra outside [0, 2^20]");
  if (extra != b->p_stall) {
    if (b->work) GP_CUDA(cudaStreamSynchronize(b->work));
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->p_stall = extra;
  }
  return GP_OK;
}

}  // extern "C"
