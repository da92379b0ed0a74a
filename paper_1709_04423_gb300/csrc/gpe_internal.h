// gpe_internal.h -- host-side internals shared by the translation units of
// libgpe.so: the handle layout, error helpers, stream joins and the
// per-precision step launchers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <complex>
#include <string>
#include <vector>

#include "gpe.h"

namespace gpe {

extern thread_local std::string g_err;
extern std::atomic<unsigned long long> g_launches;

inline int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define GP_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ::gpe::fail(GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

inline void count_launch(unsigned long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Programmatic dependent launch of consecutive kernels: on unless GPE_PDL=0.
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("GPE_PDL");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Segment lengths for which segment-product tables are kept.
constexpr int kNumSegs = 6;
constexpr int kSegs[kNumSegs] = {1, 2, 4, 8, 16, 32};
inline int seg_index(int seg) {
  for (int i = 0; i < kNumSegs; ++i)
    if (kSegs[i] == seg) return i;
  return -1;
}

// Coefficient modes: real-time step, imaginary-time step, and the real-time
// step with dt -> -dt (the conjugate-transposed sweep used by the adjoint).
enum { MODE_REAL = 0, MODE_IMAG = 1, MODE_REAL_ADJ = 2, NUM_MODES = 3 };

}  // namespace gpe

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
  void* vt[3] = {nullptr, nullptr, nullptr};     // nu_d^2 x^2/2 per axis, state precision
  // potential factors of the sub-step N, state precision, complex:
  // fac[0][d][i] = exp(-i dt v_d(x_i)), fac[1][d][i] = exp(-dt v_d(x_i)) (real);
  // with a user potential fV[0][q] = exp(-i dt V_q), fV[1][q] = exp(-dt V_q)
  void* fac[2][3] = {{nullptr}};
  void* fV[2] = {nullptr, nullptr};
  // double-float state: the factors as exact triple-floats (tf3c) -- per x
  // index, per x line (fy[j] fz[k]) and, with a user potential, per point --
  // and a complex128 staging buffer for the state exchange and observables
  void* tfx[2] = {nullptr, nullptr};
  void* tfyz[2] = {nullptr, nullptr};
  void* tfV[2] = {nullptr, nullptr};
  void* df_stage = nullptr;
  double* vd[3] = {nullptr, nullptr, nullptr};   // same in FP64
  double* cdx[3] = {nullptr, nullptr, nullptr};  // coordinates
  double* wd[3] = {nullptr, nullptr, nullptr};   // Simpson weights
  void* wt[3] = {nullptr, nullptr, nullptr};     // Simpson weights, state precision
  void* ct[3] = {nullptr, nullptr, nullptr};     // coordinates, state precision (FP32 observables)
  double wscale = 1.0;                           // prod_d dx_d/3: wt holds the Simpson coefficients
  // per (mode, axis): [0] alpha_k, [1 + 2 s] forward and [2 + 2 s] backward
  // segment products for segment length kSegs[s]; each n complex values
  void* coef[gpe::NUM_MODES][3] = {{nullptr}};
  // per (mode, axis): for each segment length, the carry tables Pf and Pb
  // (16 x 16 complex each) of the segment scans
  void* ctab[gpe::NUM_MODES][3] = {{nullptr}};
  // FP32 2d/3d grids, x axis, real and imaginary time: the tables of segments
  // aligned to even points (TMA x sweep): gf, gb for SEG 8 then 16 (n complex
  // values each), then the carry tables (512) for SEG 8 and 16
  void* coef_even[gpe::NUM_MODES] = {nullptr};
  // per mode and even segment length (8, 16): points at a segment's start (end)
  // that take a carry, and segments a carry crosses, above 2^-48 (gpe_tma.cuh)
  int even_nj[gpe::NUM_MODES][2] = {{0}};
  int even_depth[gpe::NUM_MODES][2] = {{0}};
  // per mode, axis and segment length: the segment carries' reach (Sweep2Args cdepth, cpts)
  int cdepth[gpe::NUM_MODES][3][gpe::kNumSegs] = {};
  int cpts[gpe::NUM_MODES][3][gpe::kNumSegs] = {};
  // circular / axial traps (geom 2): per mode, the rho axis' backward
  // coefficients, forward right-hand-side factors and stencil factors
  // (vab, vbf, vh of Sweep2Args; 3 n[0] complex values)
  void* cvar[gpe::NUM_MODES] = {nullptr};
  // legacy thread-per-line factors (m_k, c'_k) per (imag, axis), used when a
  // line is too long for the segmented kernels
  void* cm[2][3] = {{nullptr}};
  void* ccp[2][3] = {{nullptr}};
  // kernel shapes: segment length per x / y,z lines (0 = thread-per-line
  // kernel) and whether the x lines are staged through a shared-memory tile
  int seg_x = 0, seg_c = 0;
  bool tile_x = false;
  int keep_c = 1;  // y/z sweeps keep their input segment in registers (when short enough)
  // persistent double-buffered sweeps (x needs tile_x); only where two
  // shared-memory stages of 32 lines fit
  bool pipe_x = false, pipe_c = false;
  // y/z sweeps of an FP32 state as persistent TMA-pipelined kernels
  // (gpe_tma.cuh); their mbarrier waits give up after tma_limit_ns and then
  // set *dev_err, which the next synchronising call turns into GP_ERR_TIMEOUT
  bool tma_c = false;
  bool tma_x = false;  // the x sweep too (FP32, nx a multiple of 16, at most 256)
  int* dev_err = nullptr;
  unsigned long long tma_limit_ns = 1000000000ull;
  int tma_expect_extra = 0;  // bytes added to every expected TMA transaction (a test's way to make a wait run out)
  // imaginary time: per-block norm sums of a step's last sweep, two slots
  // alternating with the step parity, their count and grid factor
  double* parts[2] = {nullptr, nullptr};
  int parts_n = 0;
  double parts_ws = 1.0;
  bool pdl_now = false;
  double* red_parts = nullptr;  // reduced-density chunk sums (+ host-bound output)
  size_t red_cap = 0;
  // 0: Cartesian; 1: spherically symmetric 3d trap solved for u = sqrt(4 pi) r phi
  // on r_i = i dr (1d), whose nonlinear term carries gw[i] = 1/(4 pi r_i^2)
  int geom = 0;
  // a real imaginary-time state (gp_set_real_state): np values of the state
  // precision in rpsi; psi then serves as the complex staging copy
  bool xyfuse = false;  // 3d FP32: the x and y sweeps as one kernel per xy plane
  bool real_mode = false;
  void* rpsi = nullptr;
  int* real_flag = nullptr;  // device flag: a nonzero imaginary part was seen
  // Strang splitting (N/2, sweeps, N/2): the factors for dt/2
  bool strang = false;
  void* fac_h[2][3] = {{nullptr}};
  void* fV_h[2] = {nullptr, nullptr};
  void* tfx_h[2] = {nullptr, nullptr};
  void* tfyz_h[2] = {nullptr, nullptr};
  void* tfV_h[2] = {nullptr, nullptr};
  void* gw_t = nullptr;      // gw in the state precision (sweeps' sub-step N)
  void* gw_o = nullptr;      // gw in the observables' arithmetic type
  double* series_buf = nullptr;  // gp_step_series: raw sums (8 per record) + host-bound records
  size_t series_cap = 0;  // launch the sweeps as programmatic dependents (inside gp_step_*)
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  double* obs_out = nullptr;  // [8]
  double* obs_host = nullptr; // pinned [8]
  double* dens_scratch = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // adjoint: checkpoints of the last gp_adjoint_forward and scratch
  long adj_nsteps = -1;       // -1: no forward recorded
  long pot_version = 0;       // bumped by gp_set_potential
  long adj_pot_version = 0;
  int adj_K = 0;
  double adj_g = 0, adj_dt = 0;
  void* adj_ckpt = nullptr;   // ceil(nsteps / K) states
  long adj_ckpt_cap = 0;      // states the buffer holds
  void* adj_traj = nullptr;   // K states
  long adj_traj_cap = 0;
  void* adj_lam = nullptr;    // one state
  double* adj_dJdV = nullptr; // npoints doubles
  double* adj_dJdg = nullptr; // one double
  std::vector<void*> allocs;
};

namespace gpe {

// Thomas factors of one axis (m_k, c'_k, alpha_k = r m_k for k = 1..n-2) of
// the Crank-Nicolson system with beta = dt/(4 dx^2) (signed), imaginary or
// real time; segment products and carry tables for a segment length.
struct AxisFactors {
  std::vector<std::complex<double>> m, cp, alpha;
};
AxisFactors thomas_factors(int n, double beta, bool imag);
void segment_products(const std::vector<std::complex<double>>& alpha, int n, int seg,
                      std::vector<std::complex<double>>& gf, std::vector<std::complex<double>>& gb);
void carry_tables(const std::vector<std::complex<double>>& alpha, int n, int sg, std::complex<double>* out);
// the same with separate forward (af) and backward (ab) coefficients
double axis_coord(int geom, int d, int n, double dx, int i);  // grid coordinate (Cartesian, r, or rho)
// first: the first point of segment 0 -- 1 (segments over the interior points
// 1..n-2) or 0 (segments aligned to even points, over 0..n-1; alpha is 0 at
// both end points, so they take part in the recurrences as zeros)
void segment_products(const std::vector<std::complex<double>>& af, const std::vector<std::complex<double>>& ab, int n,
                      int seg, std::vector<std::complex<double>>& gf, std::vector<std::complex<double>>& gb,
                      int first = 1);
void carry_tables(const std::vector<std::complex<double>>& af, const std::vector<std::complex<double>>& ab, int n,
                  int sg, std::complex<double>* out, int first = 1);
// How far the segment carries reach above tau, read off one segmentation's
// tables (gf, gb: n values; tabs: its 512 carry-table values): depth =
// segments a carry crosses, pts = points at a segment's start (end) that take
// one (both >= 1).
void carry_reach(const std::complex<double>* gf, const std::complex<double>* gb, const std::complex<double>* tabs,
                 int n, int sg, int first, double tau, int& depth, int& pts);
// The class of carried points the block-wide sweeps are unrolled for: 4, 8, 12 or 0 (every point).
int carry_pts_class(int pts);
int tile_seg(int M);
bool plane_fits(const gp_handle* h, int seg);  // the fused x + y sweep kernel takes this grid and segment length
bool tma_fits(const gp_handle* h, int seg);    // the TMA y/z sweeps take this grid and segment length
bool tma_x_fits(const gp_handle* h, int seg);  // the TMA x sweep takes this grid and segment length
int read_dev_err(gp_handle* h, const char* who);  // GP_ERR_TIMEOUT (and clears it) if a device wait gave up

int dev_alloc(gp_handle* h, void** p, size_t bytes);
// Device buffers of handles and batches: cudaMalloc / cudaFree, and in the
// checking build (GPE_BOUNDS_CHECK) each buffer sits between two guard bands
// filled with 0xFF bytes, checked by gp_check_status.
cudaError_t guarded_malloc(void** p, size_t bytes);
void guarded_free(void* p);
int join_in(gp_handle* h);
int join_out(gp_handle* h);
inline int axis_len(const gp_handle* h, int d) { return d < h->dim ? h->n[d] : 1; }
void drop_graphs(gp_handle* h);
int upload_coefs(gp_handle* h);
int upload_factors(gp_handle* h);

// per-precision entry points (gpe_step_f32.cu / gpe_step_f64.cu)
int run_steps_any(gp_handle* h, bool imag, long nsteps);  // dispatch on h->prec
int time_steps_any(gp_handle* h, bool imag, long nsteps, double* ms_out);
// sums_out: where the seven FP64 sums go (default: the handle's slot)
int run_observables_any(gp_handle* h, double* dens_dev, double* sums_out = nullptr);
int time_graph_f32(gp_handle* h, bool imag, int reps, double* ms_out);
int time_graph_f64(gp_handle* h, bool imag, int reps, double* ms_out);
int time_graph_df(gp_handle* h, bool imag, int reps, double* ms_out);
int run_steps_df(gp_handle* h, bool imag, long nsteps);
int time_steps_df(gp_handle* h, bool imag, long nsteps, double* ms_out);
int run_observables_df(gp_handle* h, double* dens_dev, double* sums_out = nullptr);
// double-float state <-> complex128 (device buffers, on the library stream)
void df_from_c128(gp_handle* h, const void* src);
void df_to_c128(gp_handle* h, void* dst);
void launch_c128_to_df(void* dst, const void* src, long n, cudaStream_t s);
void launch_df_to_c128(void* dst, const void* src, long n, cudaStream_t s);
// real imaginary-time state: its complex copy into psi (no-op for a complex
// state); the real state from psi (synchronises; GP_ERR_STATE if an
// imaginary part is nonzero)
void materialize_complex(gp_handle* h);
int real_from_complex(gp_handle* h);
void tf_from_c128(gp_handle* h, void* dst, const void* src, long n);  // exact triple-float split
int run_steps_f32(gp_handle* h, bool imag, long nsteps);
int run_steps_f64(gp_handle* h, bool imag, long nsteps);
int time_steps_f32(gp_handle* h, bool imag, long nsteps, double* ms_out);
int time_steps_f64(gp_handle* h, bool imag, long nsteps, double* ms_out);
int run_observables_f32(gp_handle* h, double* dens_dev, double* sums_out = nullptr);
int run_observables_f64(gp_handle* h, double* dens_dev, double* sums_out = nullptr);
void to_float(gp_handle* h, float* dst, const double* src, long n);
// per-point factors of the FP64 potential for the step dt_eff (state precision; double-float: + triple-float)
void potential_factors(gp_handle* h, double dt_eff, void* const (&fV)[2], void* const (&tfV)[2]);
int adjoint_forward_f32(gp_handle* h, long nsteps, int K);
int adjoint_forward_f64(gp_handle* h, long nsteps, int K);
int adjoint_backward_f32(gp_handle* h, double* dJdV_dev, void* lam0_dev);
int adjoint_backward_f64(gp_handle* h, double* dJdV_dev, void* lam0_dev);

}  // namespace gpe
