// gpe_step_f64.cu -- instantiates the step launchers for the double state.
#include "gpe_step.cuh"

namespace gpe {

int run_steps_f64(gp_handle* h, bool imag, long nsteps) { return run_steps_t<double>(h, imag, nsteps); }

int time_steps_f64(gp_handle* h, bool imag, long nsteps, double* ms_out) {
  return time_steps_t<double>(h, imag, nsteps, ms_out);
}

int time_graph_f64(gp_handle* h, bool imag, int reps, double* ms_out) {
  return time_sweeps_graph_t<double>(h, imag, reps, ms_out);
}

int run_observables_f64(gp_handle* h, double* dens_dev, double* sums_out) {
  return run_observables_t<double>(h, dens_dev, sums_out);
}

int adjoint_forward_f64(gp_handle* h, long nsteps, int K) { return adjoint_forward_t<double>(h, nsteps, K); }

int adjoint_backward_f64(gp_handle* h, double* dJdV_dev, void* lam0_dev) {
  return adjoint_backward_t<double>(h, dJdV_dev, lam0_dev);
}

}  // namespace gpe
