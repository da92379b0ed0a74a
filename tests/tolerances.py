"""Tolerances of the FP32 form's chemical potential against the FP64 oracle.

The 1e-6 bound on |d mu| is the gate at the end of a configuration's run (the
128^3 imaginary-time job: tests/test_gpu_parity.py::test_headline_job_as_tuned).
Part way through a run, and on a single line, an FP32 state carries more: the
state is rounded to FP32 after every sub-step, and
- in imaginary time, the library expf's error varies smoothly with the phase
  angle, so until the iteration settles it acts as a small perturbation of the
  potential: 2.1e-6 after 100 steps of the 128^3 job (mu = 5.17), 1.1e-6 after
  300 steps of a 2d grid (mu = 3.9); the job then ends at 8.6e-7;
- on one line of a few hundred points the rounding noise averages over only
  ~sqrt(n) points: an FP32 emulation with exact arithmetic moves mu by 7.7e-7
  at mu = 14 (257 points, 300 real-time steps) from the storage rounding alone.
Both are about 4e-7 of mu (seven FP32 ulps); transient checks and 1d lines
are held to 5e-7 |mu|, and never to less than 1e-6."""


def mu_tol_f32(mu, transient=True):
    return max(1e-6, 5e-7 * abs(mu)) if transient else 1e-6
