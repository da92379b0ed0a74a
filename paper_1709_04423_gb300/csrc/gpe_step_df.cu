// gpe_step_df.cu -- instantiates the step launchers for the double-float
// state (GP_DF64) and its conversions from and to complex128.
#include "gpe_step.cuh"

namespace gpe {

namespace {

__global__ void c128_to_df_kernel(df64x2* dst, const double2* src, long n) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const double2 v = src[q];
    dst[q] = df64x2{df64(v.x), df64(v.y)};
  }
}

__global__ void df_to_c128_kernel(double2* dst, const df64x2* src, long n) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const df64x2 v = src[q];
    dst[q] = make_double2((double)v.x, (double)v.y);
  }
}

__global__ void c128_to_tf_kernel(tf3c* dst, const double2* src, long n) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const double2 v = src[q];
    tf3c f;
    tf_split(v.x, f.re);
    tf_split(v.y, f.im);
    dst[q] = f;
  }
}

int grid_for(long n) { return (int)std::min<long>((n + 255) / 256, 152L * 8); }

}  // namespace

// complex128 <-> double-float states of n points on stream s (the batch's)
void launch_c128_to_df(void* dst, const void* src, long n, cudaStream_t s) {
  c128_to_df_kernel<<<grid_for(n), 256, 0, s>>>((df64x2*)dst, (const double2*)src, n);
  count_launch();
}
void launch_df_to_c128(void* dst, const void* src, long n, cudaStream_t s) {
  df_to_c128_kernel<<<grid_for(n), 256, 0, s>>>((double2*)dst, (const df64x2*)src, n);
  count_launch();
}

void df_from_c128(gp_handle* h, const void* src) {
  c128_to_df_kernel<<<grid_for(h->np), 256, 0, h->work>>>((df64x2*)h->psi, (const double2*)src, h->np);
  count_launch();
}

void df_to_c128(gp_handle* h, void* dst) {
  df_to_c128_kernel<<<grid_for(h->np), 256, 0, h->work>>>((double2*)dst, (const df64x2*)h->psi, h->np);
  count_launch();
}

void tf_from_c128(gp_handle* h, void* dst, const void* src, long n) {
  c128_to_tf_kernel<<<grid_for(n), 256, 0, h->work>>>((tf3c*)dst, (const double2*)src, n);
  count_launch();
}

int run_steps_df(gp_handle* h, bool imag, long nsteps) { return run_steps_t<df64>(h, imag, nsteps); }

int time_steps_df(gp_handle* h, bool imag, long nsteps, double* ms_out) {
  return time_steps_t<df64>(h, imag, nsteps, ms_out);
}

int time_graph_df(gp_handle* h, bool imag, int reps, double* ms_out) {
  return time_sweeps_graph_t<df64>(h, imag, reps, ms_out);
}

// The observables take the state rounded to complex128 (the sums are FP64).
int run_observables_df(gp_handle* h, double* dens_dev, double* sums_out) {
  df_to_c128(h, h->df_stage);
  void* psi = h->psi;
  h->psi = h->df_stage;
  const int rc = run_observables_t<double>(h, dens_dev, sums_out);
  h->psi = psi;
  return rc;
}

}  // namespace gpe
