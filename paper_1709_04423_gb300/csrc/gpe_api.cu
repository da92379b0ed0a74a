// gpe_api.cu -- C ABI of the GB300 split-step Crank-Nicolson GP propagator
// (declared and documented in include/gpe.h).
//
// Host side of the library: argument validation, device memory owned by the
// handle, the time-invariant elimination coefficients, the per-step launch
// sequence (N fused into the x sweep, then the y and z sweeps, with the
// imaginary-time norm fused into the last sweep), CUDA-graph replay of step
// blocks, and the observables reduction.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gpe.h"
#include "gpe_obs.cuh"
#include "gpe_sweep.cuh"

using gpe::c2_t;
using cd = std::complex<double>;

namespace {

thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};

constexpr int kSweepThreads = 128;
constexpr int kObsThreads = 256;
constexpr int kGraphSteps = 16;  // steps per captured graph (even: keeps the norm-slot parity)

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define GP_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

}  // namespace

struct gp_handle {
  int dim = 0;
  int n[3] = {1, 1, 1};
  double dx[3] = {1, 1, 1};
  double dt = 0, g = 0;
  double nkl[3] = {1, 1, 1};
  int prec = GP_F64;
  long np = 0;
  size_t esize = 0;  // bytes per complex value
  cudaStream_t user = nullptr, work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void* psi = nullptr;
  double* Vd = nullptr;      // user potential (FP64), or nullptr for the trap
  void* Vt = nullptr;        // same potential in the state precision
  double* Vbuf = nullptr;    // storage behind Vd
  float* Vbuf32 = nullptr;   // storage behind Vt for the FP32 form
  void* vt[3] = {nullptr, nullptr, nullptr};        // nu_d^2 x^2/2 per axis, state precision
  double* vd[3] = {nullptr, nullptr, nullptr};      // same in FP64
  double* cdx[3] = {nullptr, nullptr, nullptr};     // coordinates
  double* wd[3] = {nullptr, nullptr, nullptr};      // Simpson weights
  void* cm[2][3] = {{nullptr}};   // [imag][axis] m_k
  void* ccp[2][3] = {{nullptr}};  // [imag][axis] c'_k
  double* scale = nullptr;   // [2] renormalisation slots
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  double* obs_out = nullptr;  // [8]
  double* obs_host = nullptr; // pinned [8]
  double* dens_scratch = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::vector<void*> allocs;
};

namespace {

int dev_alloc(gp_handle* h, void** p, size_t bytes) {
  GP_CUDA(cudaMalloc(p, bytes < 16 ? 16 : bytes));
  h->allocs.push_back(*p);
  GP_CUDA(cudaMemsetAsync(*p, 0, bytes < 16 ? 16 : bytes, h->work));
  return GP_OK;
}

int axis_len(const gp_handle* h, int d) { return d < h->dim ? h->n[d] : 1; }

// Thomas factors of one axis: m_k = 1/(b - a c'_{k-1}), c'_k = a m_k, k = 1..n-2,
// with a = -r, b = 1 + 2r, r = beta (imaginary time) or i beta (real time).
void thomas_factors(int n, double beta, bool imag, std::vector<cd>& m, std::vector<cd>& cp) {
  m.assign(n, cd(0, 0));
  cp.assign(n, cd(0, 0));
  const cd r = imag ? cd(beta, 0) : cd(0, beta);
  const cd a = -r, b = 1.0 + 2.0 * r;
  cd cprev(0, 0);
  for (int k = 1; k <= n - 2; ++k) {
    const cd den = b - a * cprev;
    m[k] = 1.0 / den;
    cp[k] = a * m[k];
    cprev = cp[k];
  }
}

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
int upload_coefs(gp_handle* h) {
  std::vector<cd> m, cp;
  for (int imag = 0; imag < 2; ++imag)
    for (int d = 0; d < h->dim; ++d) {
      const double beta = h->dt / (4.0 * h->dx[d] * h->dx[d]);
      thomas_factors(h->n[d], beta, imag != 0, m, cp);
      int rc = upload_c2<T>(h, h->cm[imag][d], m);
      if (rc) return rc;
      rc = upload_c2<T>(h, h->ccp[imag][d], cp);
      if (rc) return rc;
    }
  return GP_OK;
}

void drop_graphs(gp_handle* h) {
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
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

gpe::LineGeom geom_of(const gp_handle* h, int axis) {
  gpe::LineGeom g;
  g.axis = axis;
  g.nx = axis_len(h, 0);
  g.ny = axis_len(h, 1);
  g.nz = axis_len(h, 2);
  g.n = axis_len(h, axis);
  g.stride = axis == 0 ? 1 : axis == 1 ? g.nx : (long)g.nx * g.ny;
  g.nlines = h->np / g.n;
  return g;
}

template <typename T, bool IMAG, bool FIRST, bool LAST>
void launch_sweep(const gpe::SweepArgs<T>& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.geom.nlines + kSweepThreads - 1) / kSweepThreads);
  gpe::cn_sweep_kernel<T, IMAG, FIRST, LAST><<<blocks, kSweepThreads, 0, s>>>(a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// One step of parity `par`: N fused into the x sweep, then y and z; in
// imaginary time the last sweep produces scale[1-par] from the norm and the
// x sweep consumes scale[par].
template <typename T>
void enqueue_step(gp_handle* h, bool imag, int par, cudaEvent_t* ev = nullptr) {
  for (int d = 0; d < h->dim; ++d) {
    if (ev) cudaEventRecord(ev[2 * d], h->work);
    gpe::SweepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.psi = (c2_t<T>*)h->psi;
    a.geom = geom_of(h, d);
    a.m = (const c2_t<T>*)h->cm[imag][d];
    a.cp = (const c2_t<T>*)h->ccp[imag][d];
    a.beta = (T)(h->dt / (4.0 * h->dx[d] * h->dx[d]));
    a.V = (const T*)h->Vt;
    a.vx = (const T*)h->vt[0];
    a.vy = (const T*)h->vt[1];
    a.vz = (const T*)h->vt[2];
    a.dt = (T)h->dt;
    a.g = (T)h->g;
    a.scale_in = imag ? h->scale + par : nullptr;
    a.w_axis = h->wd[d];
    a.w_a = d == 0 ? h->wd[1] : h->wd[0];
    a.w_b = d == 2 ? h->wd[1] : h->wd[2];
    a.partials = h->partials;
    a.counter = h->counter;
    a.scale_out = h->scale + (1 - par);
    const bool first = d == 0, last = d == h->dim - 1;
    if (imag) {
      if (first && last) launch_sweep<T, true, true, true>(a, h->work);
      else if (first) launch_sweep<T, true, true, false>(a, h->work);
      else if (last) launch_sweep<T, true, false, true>(a, h->work);
      else launch_sweep<T, true, false, false>(a, h->work);
    } else {
      if (first) launch_sweep<T, false, true, false>(a, h->work);
      else launch_sweep<T, false, false, false>(a, h->work);
    }
    if (ev) cudaEventRecord(ev[2 * d + 1], h->work);
  }
}

// Eager steps with an event pair around every sweep launch (recorded on the
// library's stream, read once at the end); returns the mean duration of each
// axis' sweep kernel in ms_out[axis].
template <typename T>
int time_steps(gp_handle* h, bool imag, long nsteps, double* ms_out) {
  std::vector<cudaEvent_t> ev((size_t)nsteps * 2 * h->dim);
  for (auto& e : ev) GP_CUDA(cudaEventCreate(&e));
  int rc = join_in(h);
  if (imag && !rc) {
    gpe::set_scalar_kernel<<<1, 1, 0, h->work>>>(h->scale, 1.0);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  for (long t = 0; t < nsteps && !rc; ++t)
    enqueue_step<T>(h, imag, (int)(t & 1), ev.data() + (size_t)t * 2 * h->dim);
  if (imag && !rc && nsteps > 0) {
    const int blocks = (int)std::min<long>((h->np + 255) / 256, 152L * 8);
    gpe::scale_kernel<T><<<blocks, 256, 0, h->work>>>((c2_t<T>*)h->psi, h->np, h->scale + (nsteps & 1));
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
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

template <typename T>
int run_steps(gp_handle* h, bool imag, long nsteps) {
  if (nsteps == 0) return GP_OK;
  int rc = join_in(h);
  if (rc) return rc;
  if (imag) {
    gpe::set_scalar_kernel<<<1, 1, 0, h->work>>>(h->scale, 1.0);
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  long t = 0;
  if (nsteps >= 2 * kGraphSteps) {
    cudaGraphExec_t& ge = h->graph[imag ? 1 : 0];
    if (!ge) {
      cudaGraph_t graph;
      GP_CUDA(cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal));
      const unsigned long long before = g_launches.load();
      for (int s = 0; s < kGraphSteps; ++s) enqueue_step<T>(h, imag, s & 1);
      g_launches.store(before);  // capture launches nothing
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
      g_launches.fetch_add((unsigned long long)kGraphSteps * h->dim, std::memory_order_relaxed);
    }
  }
  for (; t < nsteps; ++t) enqueue_step<T>(h, imag, (int)(t & 1));
  if (imag) {
    const int blocks = (int)std::min<long>((h->np + 255) / 256, 152L * 8);
    gpe::scale_kernel<T><<<blocks, 256, 0, h->work>>>((c2_t<T>*)h->psi, h->np, h->scale + (nsteps & 1));
    g_launches.fetch_add(1, std::memory_order_relaxed);
  }
  GP_CUDA(cudaGetLastError());
  return join_out(h);
}

template <typename T>
int run_observables(gp_handle* h, double* dens_dev) {
  gpe::ObsArgs<T> a;
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
  a.vx = h->vd[0]; a.vy = h->vd[1]; a.vz = h->vd[2];
  a.cx = h->cdx[0]; a.cy = h->cdx[1]; a.cz = h->cdx[2];
  a.wx = h->wd[0]; a.wy = h->wd[1]; a.wz = h->wd[2];
  a.density = dens_dev;
  a.partials = h->partials;
  a.counter = h->counter;
  a.out = h->obs_out;
  const int blocks = (int)std::min<long>((h->np + kObsThreads - 1) / kObsThreads, 152L * 16);
  gpe::observables_kernel<T><<<blocks, kObsThreads, 0, h->work>>>(a);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  GP_CUDA(cudaGetLastError());
  return GP_OK;
}

bool is_finite_value(double v) { return std::isfinite(v); }

}  // namespace

extern "C" {

const char* gp_last_error(void) { return g_err.c_str(); }

unsigned long long gp_kernel_launches(void) { return g_launches.load(); }

long gp_npoints(const gp_handle* h) { return h ? h->np : 0; }

int gp_precision_of(const gp_handle* h) { return h ? h->prec : -1; }

int gp_destroy(gp_handle* h) {
  if (!h) return GP_OK;
  if (h->work) cudaStreamSynchronize(h->work);
  drop_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->obs_host) cudaFreeHost(h->obs_host);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->work) cudaStreamDestroy(h->work);
  delete h;
  return GP_OK;
}

int gp_init(gp_handle** out, int dim, const int n[3], const double dx[3], double dt,
            const double nkl[3], double g, gp_precision prec, void* stream) {
  g_err.clear();
  if (!out || !n || !dx || !nkl) return fail(GP_ERR_INVALID, "gp_init: NULL argument");
  *out = nullptr;
  if (dim < 1 || dim > 3) return fail(GP_ERR_INVALID, "gp_init: dim must be 1, 2 or 3");
  if (prec != GP_F64 && prec != GP_F32) return fail(GP_ERR_INVALID, "gp_init: unknown precision");
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
  for (int d = 0; d < 3; ++d) {
    h->n[d] = d < dim ? n[d] : 1;
    h->dx[d] = d < dim ? dx[d] : 1.0;
    h->nkl[d] = d < dim ? nkl[d] : 0.0;
  }
  h->dt = dt;
  h->g = g;
  h->prec = prec;
  h->np = np;
  h->esize = prec == GP_F64 ? sizeof(double2) : sizeof(float2);
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
  const size_t tsz = prec == GP_F64 ? sizeof(double) : sizeof(float);
  if ((rc = dev_alloc(h, &h->psi, (size_t)np * h->esize))) return bail(rc);
  for (int d = 0; d < 3; ++d) {
    const int nd = axis_len(h, d);
    std::vector<double> x(nd, 0.0), v(nd, 0.0), w(nd, 1.0);
    if (d < dim) {
      for (int i = 0; i < nd; ++i) {
        x[i] = -0.5 * nd * dx[d] + i * dx[d];
        v[i] = 0.5 * nkl[d] * nkl[d] * x[i] * x[i];
      }
      // composite Simpson on the first m points (m = n odd, n-1 even)
      const int m = (nd % 2 == 1) ? nd : nd - 1;
      for (int i = 0; i < nd; ++i) {
        double c = 0.0;
        if (i < m) c = (i == 0 || i == m - 1) ? 1.0 : (i % 2 == 1 ? 4.0 : 2.0);
        w[i] = c * dx[d] / 3.0;
      }
    }
    if ((rc = dev_alloc(h, &h->vt[d], nd * tsz))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->vd[d], nd * sizeof(double)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->cdx[d], nd * sizeof(double)))) return bail(rc);
    if ((rc = dev_alloc(h, (void**)&h->wd[d], nd * sizeof(double)))) return bail(rc);
    rc = prec == GP_F64 ? upload_real<double>(h, h->vt[d], v) : upload_real<float>(h, h->vt[d], v);
    if (rc) return bail(rc);
    if ((rc = upload_real<double>(h, h->vd[d], v))) return bail(rc);
    if ((rc = upload_real<double>(h, h->cdx[d], x))) return bail(rc);
    if ((rc = upload_real<double>(h, h->wd[d], w))) return bail(rc);
  }
  for (int imag = 0; imag < 2; ++imag)
    for (int d = 0; d < dim; ++d) {
      if ((rc = dev_alloc(h, &h->cm[imag][d], (size_t)h->n[d] * h->esize))) return bail(rc);
      if ((rc = dev_alloc(h, &h->ccp[imag][d], (size_t)h->n[d] * h->esize))) return bail(rc);
    }
  rc = prec == GP_F64 ? upload_coefs<double>(h) : upload_coefs<float>(h);
  if (rc) return bail(rc);
  // reduction scratch: enough partial slots for any sweep or observables grid
  long maxblocks = 152L * 16;
  for (int d = 0; d < dim; ++d) maxblocks = std::max(maxblocks, (h->np / h->n[d] + kSweepThreads - 1) / kSweepThreads);
  if ((rc = dev_alloc(h, (void**)&h->partials, (size_t)maxblocks * 8 * sizeof(double)))) return bail(rc);
  if ((rc = dev_alloc(h, (void**)&h->counter, 64))) return bail(rc);
  if ((rc = dev_alloc(h, (void**)&h->scale, 2 * sizeof(double)))) return bail(rc);
  if ((rc = dev_alloc(h, (void**)&h->obs_out, 8 * sizeof(double)))) return bail(rc);
  {
    cudaError_t e = cudaStreamSynchronize(h->work);
    if (e != cudaSuccess) return bail(fail(GP_ERR_CUDA, std::string("gp_init: ") + cudaGetErrorString(e)));
  }
  *out = h;
  return GP_OK;
}

int gp_set_state(gp_handle* h, const void* psi, int on_device) {
  if (!h || !psi) return fail(GP_ERR_INVALID, "gp_set_state: NULL argument");
  int rc = join_in(h);
  if (rc) return rc;
  GP_CUDA(cudaMemcpyAsync(h->psi, psi, (size_t)h->np * h->esize,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->work));
  if (!on_device) GP_CUDA(cudaStreamSynchronize(h->work));
  return join_out(h);
}

int gp_get_state(gp_handle* h, void* psi, int on_device) {
  if (!h || !psi) return fail(GP_ERR_INVALID, "gp_get_state: NULL argument");
  int rc = join_in(h);
  if (rc) return rc;
  GP_CUDA(cudaMemcpyAsync(psi, h->psi, (size_t)h->np * h->esize,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->work));
  if (!on_device) GP_CUDA(cudaStreamSynchronize(h->work));
  return join_out(h);
}

int gp_set_potential(gp_handle* h, const double* V, int on_device) {
  if (!h) return fail(GP_ERR_INVALID, "gp_set_potential: NULL handle");
  int rc = join_in(h);
  if (rc) return rc;
  drop_graphs(h);
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
  }
  GP_CUDA(cudaMemcpyAsync(h->Vbuf, V, (size_t)h->np * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->work));
  h->Vd = h->Vbuf;
  if (h->prec == GP_F64) {
    h->Vt = h->Vbuf;
  } else {
    const int blocks = (int)std::min<long>((h->np + 255) / 256, 152L * 8);
    gpe::to_float_kernel<<<blocks, 256, 0, h->work>>>(h->Vbuf32, h->Vbuf, h->np);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    h->Vt = h->Vbuf32;
  }
  GP_CUDA(cudaGetLastError());
  if (!on_device) GP_CUDA(cudaStreamSynchronize(h->work));
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
  rc = h->prec == GP_F64 ? upload_coefs<double>(h) : upload_coefs<float>(h);
  if (rc) return rc;
  return join_out(h);
}

int gp_step_imag(gp_handle* h, long nsteps) {
  if (!h) return fail(GP_ERR_INVALID, "gp_step_imag: NULL handle");
  if (nsteps < 0) return fail(GP_ERR_INVALID, "gp_step_imag: nsteps < 0");
  return h->prec == GP_F64 ? run_steps<double>(h, true, nsteps) : run_steps<float>(h, true, nsteps);
}

int gp_step_real(gp_handle* h, long nsteps) {
  if (!h) return fail(GP_ERR_INVALID, "gp_step_real: NULL handle");
  if (nsteps < 0) return fail(GP_ERR_INVALID, "gp_step_real: nsteps < 0");
  return h->prec == GP_F64 ? run_steps<double>(h, false, nsteps) : run_steps<float>(h, false, nsteps);
}

int gp_time_sweeps(gp_handle* h, int imag, long nsteps, double* ms_per_launch) {
  if (!h || !ms_per_launch) return fail(GP_ERR_INVALID, "gp_time_sweeps: NULL argument");
  if (nsteps < 0 || nsteps > 4096) return fail(GP_ERR_INVALID, "gp_time_sweeps: nsteps must be in [0, 4096]");
  return h->prec == GP_F64 ? time_steps<double>(h, imag != 0, nsteps, ms_per_launch)
                           : time_steps<float>(h, imag != 0, nsteps, ms_per_launch);
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
  rc = h->prec == GP_F64 ? run_observables<double>(h, ddev) : run_observables<float>(h, ddev);
  if (rc) return rc;
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
    if (!is_finite_value(S[q])) return fail(GP_ERR_NONFINITE, "gp_observables: the state holds NaN or Inf");
  return GP_OK;
}

}  // extern "C"
