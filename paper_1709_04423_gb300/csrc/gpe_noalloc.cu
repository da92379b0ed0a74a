// gpe_noalloc.cu -- gp_observables_noalloc: the observables reduction for
// callers that cannot allocate device memory (declared in include/gpe.h).
//
// Some callers cannot call cudaMalloc when they need the observables of a
// state: a host application that owns the whole device-memory budget and
// forbids allocations after start-up (its own pool holds every byte), and a
// loop that must never synchronise the device (cudaMalloc and cudaFree may
// synchronise).  For them this entry point computes the same quantities as
// gp_observables without a handle and without allocating: its scratch space
// (per-axis tables, per-block partial sums, the raw sums and the completion
// counter) is the file-scope array below, which every GPU that loads the
// library holds until the process ends.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "gpe_internal.h"
#include "gpe_obs.cuh"

namespace {

constexpr int kMaxAxis = 4096;          // points per axis at most
constexpr int kBlocks = 152 * 16;       // reduction grid (at most)
// layout, in doubles: [3 axes][v, coord, weight][kMaxAxis] | the same tables
// as floats (FP32 states) | partials | sums | counter
constexpr long kAxisOff = 0;
constexpr long kAxisOffF = kAxisOff + 3L * 3 * kMaxAxis;
constexpr long kPartOff = kAxisOffF + 3L * 3 * kMaxAxis / 2;
constexpr long kSumOff = kPartOff + 8L * kBlocks;
constexpr long kCntOff = kSumOff + 8;
constexpr long kScratchDoubles = kCntOff + 32;  // about 600 KB in all
static_assert(kBlocks >= gpe::kObsBlocks, "partial slots for every block of the reduction");

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Fills the per-axis tables (nu_d^2 x^2/2, x, Simpson weight; absent axes get
// a single point with 0, 0, 1) and clears the completion counter.
__global__ void noalloc_setup_kernel(double* scratch, int dim, int nx, int ny, int nz, double hx, double hy,
                                     double hz, double nu, double ka, double la) {
  const int nn[3] = {nx, ny, nz};
  const double hh[3] = {hx, hy, hz}, ff[3] = {nu, ka, la};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * kMaxAxis; t += gridDim.x * blockDim.x) {
    const int d = t / kMaxAxis, i = t % kMaxAxis;
    double* v = scratch + kAxisOff + (3L * d + 0) * kMaxAxis;
    double* c = scratch + kAxisOff + (3L * d + 1) * kMaxAxis;
    double* w = scratch + kAxisOff + (3L * d + 2) * kMaxAxis;
    float* vf = (float*)(scratch + kAxisOffF) + (3L * d + 0) * kMaxAxis;
    float* cf = (float*)(scratch + kAxisOffF) + (3L * d + 1) * kMaxAxis;
    float* wf = (float*)(scratch + kAxisOffF) + (3L * d + 2) * kMaxAxis;
    if (i >= nn[d]) continue;
    if (d >= dim) {
      v[i] = 0.0; c[i] = 0.0; w[i] = 1.0;
      vf[i] = 0.f; cf[i] = 0.f; wf[i] = 1.f;
      continue;
    }
    const int n = nn[d];
    const double x = -0.5 * n * hh[d] + i * hh[d];
    v[i] = 0.5 * ff[d] * ff[d] * x * x;
    c[i] = x;
    const int m = (n % 2 == 1) ? n : n - 1;  // composite Simpson on the first m points
    double wc = 0.0;
    if (i < m) wc = (i == 0 || i == m - 1) ? 1.0 : (i % 2 == 1 ? 4.0 : 2.0);
    w[i] = wc * hh[d] / 3.0;
    vf[i] = (float)v[i];
    cf[i] = (float)c[i];
    wf[i] = (float)wc;  // FP32 tables: the exact Simpson coefficient (factor applied to the totals)
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *(unsigned int*)(scratch + kCntOff) = 0u;
}

// Turns the seven Simpson sums into the gp_obs fields.
__global__ void noalloc_finish_kernel(const double* S, double g, double* out) {
  const double N = S[0];
  out[0] = N;
  out[1] = (S[1] + S[2]) / N + 0.5 * g * S[3] / (N * N);
  out[2] = (S[1] + S[2]) / N + g * S[3] / (N * N);
  double r2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    out[3 + d] = sqrt(S[4 + d] / N);
    r2 += S[4 + d] / N;
  }
  out[6] = sqrt(r2);
}

// Device address of the scratch array on the current device.  Host code only
// holds a host-side stand-in for the array's name, so the address is looked
// up with cudaGetSymbolAddress with the device current.  It is looked up
// again on every call made while the stream is not being captured (a device
// reset, or a released and re-created primary context, may move the array);
// a call made during a capture takes the address found by the last call
// outside one, so the first call on a device must come before any capture.
int scratch_address(cudaStream_t s, double** out) {
  int dev = 0;
  GP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: device ordinal too large");
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!capturing) {
    void* p = nullptr;
    GP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = p;
  }
  if (!g_scratch_addr[dev])
    return gpe::fail(GP_ERR_STATE,
                     "gp_observables_noalloc: the first call on a device must come before any stream capture");
  *out = (double*)g_scratch_addr[dev];
  return GP_OK;
}

template <typename T>
void launch_obs(double* scratch, int dim, const int* n3, const double* dx3, const void* psi, const double* V,
                cudaStream_t s) {
  gpe::ObsArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.psi = (const gpe::c2_t<T>*)psi;
  a.dim = dim;
  a.nx = n3[0]; a.ny = n3[1]; a.nz = n3[2];
  a.hx = dx3[0]; a.hy = dx3[1]; a.hz = dx3[2];
  a.V = V;
  using R = gpe::obs_r<T>;
  const R* tab = std::is_same<R, float>::value ? (const R*)(scratch + kAxisOffF) : (const R*)(scratch + kAxisOff);
  a.vx = tab + 0L * kMaxAxis;
  a.cx = tab + 1L * kMaxAxis;
  a.wx = tab + 2L * kMaxAxis;
  a.vy = tab + 3L * kMaxAxis;
  a.cy = tab + 4L * kMaxAxis;
  a.wy = tab + 5L * kMaxAxis;
  a.vz = tab + 6L * kMaxAxis;
  a.cz = tab + 7L * kMaxAxis;
  a.wz = tab + 8L * kMaxAxis;
  a.wscale = 1.0;
  if (std::is_same<R, float>::value)
    for (int d = 0; d < dim; ++d) a.wscale *= dx3[d] / 3.0;
  a.density = nullptr;
  a.partials = scratch + kPartOff;
  a.counter = (unsigned int*)(scratch + kCntOff);
  a.out = scratch + kSumOff;
  gpe::launch_observables<T>(a, s);
  gpe::count_launch();
}

}  // namespace

extern "C" int gp_observables_noalloc(int dim, const int n[3], const double dx[3], const double nkl[3], double g,
                                      gp_precision prec, const void* psi, const double* V, double* out,
                                      void* stream) {
  if (!n || !dx || !nkl || !psi || !out) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: NULL argument");
  if (dim < 1 || dim > 3) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: dim must be 1, 2 or 3");
  if (prec == GP_DF64)
    return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: GP_DF64 is not supported here (GP_F64 or GP_F32 states only)");
  if (prec != GP_F64 && prec != GP_F32) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: unknown precision");
  int n3[3] = {1, 1, 1};
  double dx3[3] = {1.0, 1.0, 1.0};
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 3) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: every axis needs n >= 3 points");
    if (n[d] > kMaxAxis)
      return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: at most 4096 points per axis (static scratch size)");
    if (!(dx[d] > 0.0) || !std::isfinite(dx[d]))
      return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: dx must be finite and > 0");
    if (!std::isfinite(nkl[d])) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: trap frequencies must be finite");
    n3[d] = n[d];
    dx3[d] = dx[d];
  }
  if ((long)n3[0] * n3[1] * n3[2] > 2147483647L)
    return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: more than 2^31-1 grid points");
  if (!std::isfinite(g)) return gpe::fail(GP_ERR_INVALID, "gp_observables_noalloc: g must be finite");
  double* scratch = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = scratch_address(s, &scratch);
  if (rc) return rc;
  noalloc_setup_kernel<<<36, 256, 0, s>>>(scratch, dim, n3[0], n3[1], n3[2], dx3[0], dx3[1], dx3[2],
                                          nkl[0], dim > 1 ? nkl[1] : 0.0, dim > 2 ? nkl[2] : 0.0);
  gpe::count_launch();
  if (prec == GP_F64) launch_obs<double>(scratch, dim, n3, dx3, psi, V, s);
  else launch_obs<float>(scratch, dim, n3, dx3, psi, V, s);
  noalloc_finish_kernel<<<1, 1, 0, s>>>(scratch + kSumOff, g, out);
  gpe::count_launch();
  GP_CUDA(cudaGetLastError());
  return GP_OK;
}
