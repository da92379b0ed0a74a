// gpe_step_f32.cu -- instantiates the step launchers for the float state.
#include "gpe_step.cuh"

namespace gpe {

int run_steps_f32(gp_handle* h, bool imag, long nsteps) { return run_steps_t<float>(h, imag, nsteps); }

int time_steps_f32(gp_handle* h, bool imag, long nsteps, double* ms_out) {
  return time_steps_t<float>(h, imag, nsteps, ms_out);
}

int time_graph_f32(gp_handle* h, bool imag, int reps, double* ms_out) {
  return time_sweeps_graph_t<float>(h, imag, reps, ms_out);
}

int run_observables_f32(gp_handle* h, double* dens_dev, double* sums_out) {
  return run_observables_t<float>(h, dens_dev, sums_out);
}

int adjoint_forward_f32(gp_handle* h, long nsteps, int K) { return adjoint_forward_t<float>(h, nsteps, K); }

int adjoint_backward_f32(gp_handle* h, double* dJdV_dev, void* lam0_dev) {
  return adjoint_backward_t<float>(h, dJdV_dev, lam0_dev);
}

}  // namespace gpe

namespace gpe {
void potential_factors(gp_handle* h, double dt_eff, void* const (&fV)[2], void* const (&tfV)[2]) {
  const int blocks = (int)std::min<long>((h->np + 255) / 256, 152L * 8);
  if (h->prec != GP_F32)
    potential_factor_kernel<double><<<blocks, 256, 0, h->work>>>((double2*)fV[0], (double2*)fV[1], h->Vbuf,
                                                                dt_eff, h->np);
  else
    potential_factor_kernel<float><<<blocks, 256, 0, h->work>>>((float2*)fV[0], (float2*)fV[1], h->Vbuf,
                                                               dt_eff, h->np);
  count_launch();
  if (h->prec == GP_DF64)  // exact triple-float images for the double-float sweeps
    for (int m = 0; m < 2; ++m) tf_from_c128(h, tfV[m], fV[m], h->np);
}

void to_float(gp_handle* h, float* dst, const double* src, long n) {
  const int blocks = (int)std::min<long>((n + 255) / 256, 152L * 8);
  to_float_kernel<<<blocks, 256, 0, h->work>>>(dst, src, n);
  count_launch();
}
}  // namespace gpe
