/*
 * gpe.h -- C ABI of the GB300 split-step Crank-Nicolson propagator for the
 * time-dependent Gross-Pitaevskii (GP) equation
 *
 *     i d(phi)/dt = [ -lap/2 + V(r) + g |phi|^2 ] phi
 *
 * in imaginary time (stationary states) and real time (dynamics) on 1d, 2d and
 * 3d Cartesian grids.  The paper's "Solution method" names the scheme:
 * split-step Crank-Nicolson with imaginary- and real-time propagation; its
 * "Nature of problem" gives the 1d/2d/3d fully anisotropic traps, and its
 * abstract and "Summary of revisions" list the outputs: energy, chemical
 * potential, root-mean-square sizes and densities.
 *
 * Discrete scheme (the paper prints no formula; these are the readings the
 * library implements):
 *   grid       x_i = -n dx/2 + i dx, i = 0..n-1 per axis;
 *   potential  V = (nu^2 x^2 + kappa^2 y^2 + lambda^2 z^2)/2, or a user array;
 *   one step   N, then L_x, L_y, L_z (Lie splitting, full dt each), where
 *              N:   phi <- exp(-i dt (V + g|phi|^2)) phi      (real time)
 *                   phi <- exp(-dt (V + g|phi|^2)) phi        (imaginary time)
 *              L_d: Crank-Nicolson along axis d with Dirichlet ends held at 0:
 *                   -r u[k-1] + (1+2r) u[k] - r u[k+1]
 *                        = r p[k-1] + (1-2r) p[k] + r p[k+1],  k = 1..n-2,
 *                   r = i dt/(4 dx^2) (real) or dt/(4 dx^2) (imaginary);
 *   imaginary time renormalises phi <- phi/sqrt(Norm) after every step, with
 *   Norm the composite-Simpson integral of |phi|^2 (Simpson on the first n
 *   points for odd n, the first n-1 for even n; tensor product across axes).
 *
 * Memory layout of every grid array: x fastest, idx = i + nx*(j + ny*k).
 * States are complex, interleaved (re, im), in the handle's precision:
 * double2 for GP_F64, float2 for GP_F32, and double2 (complex128) at the API
 * for GP_DF64, whose device state is double-float.  Potentials and densities
 * are double.
 *
 * Errors: every call returns GP_OK (0) or a negative code; gp_last_error()
 * returns a thread-local message for the last failure.  No call aborts or
 * throws.  Arguments are validated on the host before anything is launched.
 *
 * Streams: a handle is bound to the CUDA stream given at creation (NULL means
 * the legacy default stream).  Work is enqueued in order on that stream; calls
 * that return host data synchronise it.  Internally the library runs on its
 * own non-blocking stream joined to the caller's stream by events, so that it
 * can replay step loops as CUDA graphs.
 *
 * Ownership: the handle owns the state, coefficients and scratch memory, all
 * allocated at creation and freed by gp_destroy.  Caller buffers are only read
 * or written during the call (host buffers) or in stream order (device
 * buffers); the library keeps no pointer to them.
 */
#ifndef GPE_H
#define GPE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GP_OK = 0,
  GP_ERR_INVALID = -1,   /* bad argument (size, spacing, NaN, NULL, ...) */
  GP_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  GP_ERR_NONFINITE = -3, /* a reduction found NaN or Inf in the state */
  GP_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up */
  GP_ERR_STATE = -5      /* call not valid in the handle's current state */
};

/* GP_DF64: the state and the sweeps in double-float arithmetic (each real a
 * pair of floats hi + lo, about 48 significant bits) on the FP32 pipes, for
 * FP64-class results on parts whose FP64 rate is a small fraction of FP32;
 * the potential factors are exact triple-float images of the FP64 ones, and
 * the reductions are FP64. */
typedef enum { GP_F64 = 0, GP_F32 = 1, GP_DF64 = 2 } gp_precision;

typedef struct gp_handle gp_handle;

/* Observables of psi = phi/sqrt(norm):
 *   norm   = Simpson integral of |phi|^2 (of the stored state),
 *   energy = int[ 1/2 sum_d |d_d psi|^2 + V|psi|^2 + g/2 |psi|^4 ],
 *   mu     = int[ 1/2 sum_d |d_d psi|^2 + V|psi|^2 + g   |psi|^4 ],
 *   rms[d] = sqrt(int x_d^2 |psi|^2) (0 for absent axes), rms_r = sqrt(sum rms^2).
 * Derivatives: 4th-order central differences for 2 <= i <= n-3, 2nd-order at
 * i = 1 and n-2, zero at the end points.  All sums are accumulated in FP64. */
typedef struct {
  double norm, energy, mu, rms[3], rms_r;
} gp_obs;

/* Creates a propagator.
 *   dim      1, 2 or 3.
 *   n        points per axis, n[d] >= 3 for d < dim (entries >= dim ignored);
 *            at most 2^31-1 points in total.
 *   dx       grid spacing per axis, > 0.
 *   dt       time step, finite and != 0 (the same dt serves imaginary time).
 *   nkl      trap frequencies nu, kappa, lambda of the harmonic potential.
 *   g        nonlinearity, finite.
 *   prec     GP_F64, GP_F32 (FP32 state and sweeps; norm, energy, mu and
 *            the renormalisation factor are still computed in FP64) or
 *            GP_DF64 (double-float state and sweeps; at most 514 points per
 *            axis; no adjoint, no pipelined shapes, not in batches).
 *   stream   cudaStream_t to order work on (NULL = legacy default stream).
 * The state starts at zero: call gp_set_state before stepping. */
int gp_init(gp_handle** out, int dim, const int n[3], const double dx[3], double dt,
            const double nkl[3], double g, gp_precision prec, void* stream);

/* Creates a propagator for a spherically symmetric 3d trap, V = nu^2 r^2/2
 * ("spherically symmetric" traps are among the paper's programs; "Nature of
 * problem").  The state is u(r) = sqrt(4 pi) r phi(r) on r_i = i dr,
 * i = 0..n-1, held at zero at r = 0 and r = (n-1) dr; it obeys the 1d
 * equation  i du/dt = [-1/2 d^2/dr^2 + V(r) + g |u|^2/(4 pi r^2)] u,  so the
 * same sweeps run with the nonlinear term weighted by 1/(4 pi r^2).
 * int |u|^2 dr is the 3d norm; gp_observables returns the 3d energy and mu
 * and, in rms[0], the rms radius sqrt(<r^2>) (rms[1] = rms[2] = 0).  A user
 * potential (gp_set_potential) is given on the r grid.  Arguments as gp_init
 * (n >= 3, dr > 0); no adjoint for this geometry. */
int gp_init_spherical(gp_handle** out, int n, double dr, double dt, double nu, double g, gp_precision prec,
                      void* stream);

/* Circularly symmetric 2d trap, V = nu^2 rho^2/2 (gp_init_circular), and
 * axially symmetric 3d trap, V = (nu^2 rho^2 + lambda^2 z^2)/2
 * (gp_init_axial): the paper's other symmetric programs ("Nature of
 * problem").  The state is phi(rho) (npoints = n) or phi(rho, z) (rho
 * fastest, npoints = n_rho n_z) with rho_i = (i - 1/2) drho, i = 0..n-1:
 * point 0 is the mirror image of point 1 across the axis (held at zero and
 * never coupled: the conservative difference of (1/rho)(rho phi')' puts the
 * factor 1 - drho/(2 rho_1) = 0 on it) and point n-1 is the outer wall (held
 * at zero); z as gp_init's grid.  The rho sweeps solve the non-symmetric
 * Crank-Nicolson system with rows (-(1 - h_k), 2, -(1 + h_k)) r, h_k =
 * drho/(2 rho_k).  Integrals take the weight 2 pi rho_i drho along rho
 * (Simpson along z): the norm is the 2d (circular) or 3d (axial) norm, the
 * energy and mu are those of the 2d / 3d problem, rms[0] is the rms radius
 * sqrt(<rho^2>) and (axial) rms[1] the rms z.  The derivative along rho in the
 * observables reads point 0 as point 1.  At most 514 points per axis; the
 * pipelined x sweep and the adjoint are not offered; the Strang splitting,
 * user potentials, reduced densities and the recorded series are.  Errors as
 * gp_init. */
int gp_init_circular(gp_handle** out, int n, double drho, double dt, double nu, double g, gp_precision prec,
                     void* stream);
int gp_init_axial(gp_handle** out, int n_rho, int n_z, double drho, double dz, double dt, double nu, double lambda,
                  double g, gp_precision prec, void* stream);

/* Copies a state in (interleaved re, im, in the handle's precision -- double
 * for GP_DF64 -- npoints values).  on_device != 0: psi is a device pointer
 * read in stream order. */
int gp_set_state(gp_handle* h, const void* psi, int on_device);

/* Copies the state out in the handle's precision (GP_DF64: rounded to
 * double).  With on_device == 0 the call synchronises the stream. */
int gp_get_state(gp_handle* h, void* psi, int on_device);

/* Replaces the harmonic trap by a potential array (double, npoints values);
 * V == NULL restores the harmonic trap. */
int gp_set_potential(gp_handle* h, const double* V, int on_device);

/* Changes the nonlinearity (e.g. the quench g -> 2g before real-time runs). */
int gp_set_g(gp_handle* h, double g);

/* Changes the time step and recomputes the elimination coefficients. */
int gp_set_dt(gp_handle* h, double dt);

/* Chooses the splitting of one step ("Solution method": the step is split
 * into the sub-step N -- potential and nonlinear term -- and one
 * Crank-Nicolson sweep per axis).  strang = 0 (the default, as in the
 * paper's programs): N with dt, then the sweeps (first order in dt).
 * strang = 1: N with dt/2, the sweeps with dt, N with dt/2 on the sweeps'
 * output (second order in dt); imaginary time renormalises after the second
 * half, as after N and the sweeps in the Lie form.  Costs one extra pass over
 * the state per step.  Takes effect for the next step; the adjoint
 * (gp_adjoint_forward/backward) and the batched runs (gp_batch_*) take the
 * Lie splitting only.  Errors: GP_ERR_INVALID for a NULL handle or a value
 * other than 0 or 1; GP_ERR_CUDA if the dt/2 tables cannot be allocated. */
int gp_set_splitting(gp_handle* h, int strang);

/* Holds the state as real numbers (real = 1) or as complex ones (real = 0,
 * the default).  In imaginary time the Crank-Nicolson coefficients and the
 * sub-step N are real ("Solution method"), so a state with zero imaginary
 * parts stays real: a real state takes half the bytes and half the
 * arithmetic per step and gives the complex path's real parts.  Takes
 * GP_F64 or GP_F32 handles of 2d or 3d Cartesian grids with an even number
 * of x points, at most 514 points per axis, the shared-memory x tile (its
 * 36 nx + 512 complex values within 200 KB: FP64 nx <= 341; real = 1 moves
 * the x sweep to the tile if another shape was chosen) and the Lie
 * splitting; gp_set_shapes may not turn the tile off while the state is real.
 * real = 1 converts the current state; it synchronises the stream and
 * fails with GP_ERR_STATE (leaving the complex state) if an imaginary part
 * is nonzero.  While real: gp_set_state still takes complex values, checks
 * them the same way (and on GP_ERR_STATE leaves real mode with the state it
 * was given), gp_get_state and the observables see the state with zero
 * imaginary parts, and gp_step_real, gp_time_sweeps/gp_step_series in real
 * time, gp_set_splitting(h, 1) and the adjoint return GP_ERR_STATE;
 * gp_autotune (imaginary time) picks among the shapes a real state takes and
 * keeps its result apart from the complex state's.  Errors: GP_ERR_INVALID for a NULL handle, a value other
 * than 0 or 1, or a grid or precision it does not take; GP_ERR_CUDA if the
 * real buffer (npoints values) cannot be allocated. */
int gp_set_real_state(gp_handle* h, int real);

/* Runs nsteps >= 0 imaginary-time steps, renormalising after each one.
 * Asynchronous: enqueued on the handle's stream. */
int gp_step_imag(gp_handle* h, long nsteps);

/* Runs nsteps >= 0 real-time steps.  Asynchronous. */
int gp_step_real(gp_handle* h, long nsteps);

/* Computes the observables of the current state; density (optional, may be
 * NULL) receives |phi|^2 as npoints doubles, on the device if
 * density_on_device != 0.  Synchronises the stream.  Returns GP_ERR_NONFINITE
 * if the state holds NaN or Inf. */
int gp_observables(gp_handle* h, gp_obs* out, double* density, int density_on_device);

/* Runs nsteps imaginary-time (imag != 0) or real-time steps and records the
 * observables every `every` steps, for the series the paper's real-time
 * programs report (rms sizes during the dynamics; "Summary of revisions"):
 * after steps every, 2 every, ..., floor(nsteps/every) every, a record of 7
 * doubles -- norm, energy, mu, rms_x, rms_y, rms_z, rms_r, as gp_observables
 * -- goes to out[7 r + q] (floor(nsteps/every) records; nothing else is
 * written).  With out_on_device != 0 the call is asynchronous (no host
 * synchronisation between records; the energy and mu use the g current at the
 * call); else the records are copied to the host at the end (synchronises).
 * Imaginary time: each record is of the renormalised state.  Leftover steps
 * (nsteps mod every) run after the last record.  The handle keeps a scratch
 * buffer of 8 doubles per record (grown on demand). */
int gp_step_series(gp_handle* h, int imag, long nsteps, int every, double* out, int out_on_device);

/* Reduced (integrated) density: |phi|^2 summed with the composite-Simpson
 * weights over the axes NOT in keep_mask, on the grid of the kept axes (the
 * paper's programs write reduced 1d and 2d densities; "Summary of
 * revisions").  keep_mask: bit d set keeps axis d (0 = x); at least one bit,
 * only bits d < dim (all bits: the density itself).  out: the product of the
 * kept axes' lengths, in doubles, kept coordinates x fastest; on the device if
 * out_on_device != 0 (asynchronous, stream order), else on the host (the call
 * synchronises).  Sums in FP64, deterministic.  The handle keeps a scratch
 * buffer of about 1 MB (allocated on the first call or when a larger one is
 * needed). */
int gp_reduced_density(gp_handle* h, int keep_mask, double* out, int out_on_device);

/* Instrumentation: runs nsteps steps (imaginary time if imag != 0) launched
 * one by one, with CUDA events on the library's stream around every sweep
 * kernel, and stores the mean duration in milliseconds of the sweep along
 * axis d in ms_per_launch[d] (d < 3; 0 for absent axes).  The state advances
 * exactly as with gp_step_imag / gp_step_real.  0 <= nsteps <= 4096.
 * Synchronises the stream. */
int gp_time_sweeps(gp_handle* h, int imag, long nsteps, double* ms_per_launch);

/* The same per-axis durations as the kernels run inside a step's CUDA graph:
 * for each axis, reps (1..1024) launches of that axis' sweep back to back in a
 * captured graph, with the programmatic-dependent-launch edges of the step
 * graph, one warm-up replay and one timed replay (events on the library's
 * stream); ms_per_launch[d] = mean per launch (0 for y when the fused x + y
 * kernel runs both).  Uses one temporary state-sized device buffer; the state
 * is restored.  For instrumentation. */
int gp_time_sweeps_graph(gp_handle* h, int imag, int reps, double* ms_per_launch);

/* Measured arithmetic rates of this GPU (the current device): FP64 and FP32
 * fused multiply-adds per second (thread instructions), from a kernel of
 * independent FMA chains on every SM timed with events.  The denominators of
 * an ALU roofline; synchronises the device.  For instrumentation. */
int gp_fp_fma_rates(double* dfma_per_s, double* ffma_per_s);

/* ---- Differentiation form: adjoint of real-time propagation.
 * Objective J(phi(T)) of the state after nsteps real-time steps; gradients
 * with respect to the potential values V (per grid point), g and phi(0).
 * Convention: the adjoint of a complex state is lambda = dJ/dRe(phi) +
 * i dJ/dIm(phi) (torch.autograd's convention for complex tensors), with the
 * real inner product <a, b> = Re sum conj(a) b.  The reverse step applies the
 * Crank-Nicolson sweeps with dt -> -dt in the order z, y, x (the conjugate
 * transposes of the forward sweeps) and then the adjoint of N at the step's
 * input p: with u = exp(-i th) p, th = dt (V + g|p|^2), s = Im(conj(lam) u):
 *     lam <- exp(i th) lam + 2 g dt s p,  dJ/dV += dt s,  dJ/dg += dt sum s|p|^2.
 *
 * gp_adjoint_forward: runs nsteps >= 1 real-time steps from the current state
 * (which becomes phi(T), as with gp_step_real), keeping the state every
 * ckpt_every steps in library memory (ceil(nsteps/ckpt_every) + ckpt_every
 * states).  Lines must have at most 514 points.
 * gp_adjoint_backward: given lambda(T) (npoints complex values in the handle's
 * precision, host or device), recomputes each checkpoint segment and runs the
 * reverse steps.  Writes dJdV (npoints doubles, host or device per flag; may be
 * NULL), *dJdg (may be NULL) and lambda(0) (device buffer in the handle's
 * precision; may be NULL).  FP64 accumulation of dJ/dV and dJ/dg.  Returns
 * GP_ERR_STATE if no forward was recorded or dt or the potential changed
 * since; g may be changed in between (the forward's g is used).  The handle's
 * state is left as phi(T).  Synchronises the stream. */
int gp_adjoint_forward(gp_handle* h, long nsteps, int ckpt_every);
int gp_adjoint_backward(gp_handle* h, const void* lambda_T, int lambda_on_device, double* dJdV, int dJdV_on_device,
                        double* dJdg, void* lambda_0);

/* ---- Batched form: many independent 2d real-time runs stepped together.
 * Each run r has its own grid (n[2r] x n[2r+1] points, spacing dx[2r],
 * dx[2r+1]), harmonic trap (nu = nkl[2r], kappa = nkl[2r+1]) and nonlinearity
 * g[r]; all runs share dt.  One batch step advances every run by one
 * split-step Crank-Nicolson step with the same discretisation as gp_step_real
 * (a run in a batch gives the same result as the same run in its own handle).
 * Runs are stored back to back: run r starts at element gp_batch_offset(r).
 * Precisions: GP_F64, GP_F32 (FP64 reductions) and GP_DF64 (double-float
 * state, FP64-class results on the FP32 pipes; its observables are those of
 * the states rounded to complex128).
 * Limits: 1 <= nruns <= 65536, 3 <= n <= 514 per axis, < 2^31 points in all. */
typedef struct gp_batch gp_batch;

int gp_batch_init(gp_batch** out, int nruns, const int* n, const double* dx, double dt, const double* nkl,
                  const double* g, gp_precision prec, void* stream);

/* Copies run `run`'s state in or out (run = -1: all runs, back to back), in
 * the batch's precision -- complex128 for GP_DF64, split into double-floats
 * on the way in and rounded on the way out; host copies synchronise the
 * stream. */
int gp_batch_set_state(gp_batch* b, int run, const void* psi, int on_device);
int gp_batch_get_state(gp_batch* b, int run, void* psi, int on_device);

/* Runs nsteps >= 0 real-time steps of every run.  Asynchronous. */
int gp_batch_step_real(gp_batch* b, long nsteps);

/* Observables of every run (out has nruns entries; rms[2] = 0).  FP64
 * reductions.  Synchronises the stream; GP_ERR_NONFINITE on NaN/Inf. */
int gp_batch_observables(gp_batch* b, gp_obs* out);

/* Element offset of run `run` in the back-to-back state, or -1. */
long gp_batch_offset(const gp_batch* b, int run);

/* How a batch step is launched (the paper has no counterpart: its programs
 * run one problem at a time).  Mode 0: one launch per sweep direction and
 * segment-length class per step (every run's x lines, then every run's y
 * lines).  Mode 1 (FP32 batches only): one persistent launch per block of
 * steps; CTAs claim (step, axis, run, 32-line tile) items in order and each
 * item waits, on per-run completion counters, for the sweep it depends on
 * (a run's x sweep of step t for its y sweep of step t-1, its y sweep for
 * its x sweep), so different runs' sweeps overlap with no grid-wide barrier.
 * The per-line arithmetic is the same in both modes: the states agree bit
 * for bit.  Each wait is bounded (GPE_WAIT_LIMIT_MS at gp_batch_init, default
 * 1000 ms); a wait that runs out stops the launch and the next
 * gp_batch_observables returns GP_ERR_TIMEOUT (the states are then not
 * valid).  gp_batch_set_mode: GP_ERR_INVALID for mode 1 on an FP64 or double-float batch.
 * gp_batch_get_mode returns the mode (-1 for NULL).  gp_batch_autotune times
 * nsteps >= 1 steps in each mode (after nsteps untimed ones), keeps the faster
 * and writes the two times in ms to ms_out[0..1] when ms_out is not NULL
 * (-1 where not timed; FP64 and double-float batches keep mode 0 untimed); the states are put
 * back.  Synchronises the stream. */
int gp_batch_set_mode(gp_batch* b, int persistent);
int gp_batch_get_mode(const gp_batch* b);
int gp_batch_autotune(gp_batch* b, long nsteps, double* ms_out);

/* Frees the batch (NULL is a no-op). */
int gp_batch_destroy(gp_batch* b);

/* Observables without a handle and without allocating.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory at the moment they need the observables -- an application
 * that owns the whole device-memory budget and forbids allocations after
 * start-up, or a loop that must not synchronise the device (cudaMalloc and
 * cudaFree may).  It computes what gp_observables computes, for a state the
 * caller passes, and calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *   dim, n, dx, nkl, g  as for gp_init; at most 4096 points per axis
 *                       (GP_ERR_INVALID beyond that).
 *   prec     GP_F64 or GP_F32 only (GP_DF64 states: GP_ERR_INVALID).
 *   psi      device state (npoints complex values in precision prec).
 *   V        device potential (npoints doubles), or NULL for the harmonic trap.
 *   out      device buffer of 7 doubles, written in stream order with
 *            {norm, energy, mu, rms_x, rms_y, rms_z, rms_r} (the gp_obs layout).
 *   stream   cudaStream_t the work is enqueued on (asynchronous).
 * Scratch space: one file-scope device array of about 600 KB, which every GPU
 * that loads the library holds until the process exits.  All calls share it
 * and it keeps the last call's contents (each call clears what must start at
 * zero), so calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised by the caller.  The
 * array's device address is looked up on each call whose stream is not being
 * captured (so it follows a device reset); a call during a stream capture
 * reuses the address found by the last call outside one, so the first call on
 * a device must come before any stream capture begins (GP_ERR_STATE
 * otherwise). */
int gp_observables_noalloc(int dim, const int n[3], const double dx[3], const double nkl[3], double g,
                           gp_precision prec, const void* psi, const double* V, double* out, void* stream);

/* ---- Kernel shapes and the autotuner.
 * A handle's sweeps run with a segment length per line (seg_x for x lines,
 * seg_c for y/z lines: 1..32, a power of two), for x lines in 2d/3d an
 * optional shared-memory tile (tile_x); flags (GP_SHAPE_*) select whether the
 * y/z input segment is kept in registers or streamed and read again, and
 * whether the x and y/z sweeps run as persistent double-buffered kernels
 * (possible where two 32-line tiles fit in shared memory); shape 0 means the
 * thread-per-line kernels used for lines longer than 514 points.  Defaults are set by
 * gp_init.  gp_autotune times every valid shape of the x sweep and of the y/z
 * sweeps on this handle's grid (2 warm-up + nsteps timed steps each, imaginary
 * time if imag != 0; 1 <= nsteps <= 256), keeps the fastest, restores the
 * state, and remembers the result for this process (a later call for the same
 * grid, precision and mode applies it without timing unless best_ms != NULL,
 * which receives the best mean x-sweep and y+z-sweep times in ms).  Uses one
 * temporary state-sized device buffer.  gp_set_shapes applies shapes (e.g.
 * from a cache file); GP_ERR_INVALID if they do not fit the grid.
 * GP_SHAPE_FUSE_XY (3d GP_F32 grids with nx, ny <= 128 and seg_x 8, 16 or 32
 * for both x and y): the x and y sweeps run as one kernel per xy plane held in
 * shared memory -- one read and one write of the state instead of two -- with
 * the same per-line arithmetic (bit-identical results); the tuner keeps it
 * where it is faster.
 * GP_SHAPE_TMA_YZ (GP_F32 complex states of 2d/3d grids with nx even, y/z
 * lines of at most 256 points, seg_c 8, 16 or 32 with at most 16 segments):
 * the y/z sweeps run as persistent kernels that move 32-line tiles between
 * global and shared memory with the TMA unit, three stages deep, and solve
 * them in place with the same per-line arithmetic as the other y/z sweeps.
 * Their waits for a tile give up after a limit (1 s, or GPE_WAIT_LIMIT_MS
 * milliseconds at gp_init); the next synchronising call (gp_observables) then
 * returns GP_ERR_TIMEOUT.
 * GP_SHAPE_TMA_X (GP_F32 complex states of Cartesian 2d/3d grids with nx a
 * multiple of 16 and at most 256, the x tile with seg_x 8 or 16): the x sweep,
 * with the sub-step N and the pending renormalisation, runs the same way, its
 * segments aligned to even points; not with GP_SHAPE_PIPE_X or
 * GP_SHAPE_FUSE_XY. */
enum {
  GP_SHAPE_KEEP_YZ = 1, /* y/z sweeps keep their input segment in registers */
  GP_SHAPE_PIPE_X = 2,  /* x sweep: persistent double-buffered tile kernel (needs tile_x) */
  GP_SHAPE_PIPE_YZ = 4, /* y/z sweeps: persistent double-buffered kernel */
  GP_SHAPE_FUSE_XY = 8, /* x and y sweeps fused, one block per xy plane (3d FP32) */
  GP_SHAPE_TMA_YZ = 16, /* y/z sweeps: persistent kernel, tiles moved by TMA (FP32) */
  GP_SHAPE_TMA_X = 32   /* x sweep (with N): persistent kernel, tiles moved by TMA (FP32) */
};
int gp_autotune(gp_handle* h, int imag, int nsteps, double* best_ms);
int gp_set_shapes(gp_handle* h, int tile_x, int seg_x, int seg_c, int flags);
int gp_get_shapes(const gp_handle* h, int* tile_x, int* seg_x, int* seg_c, int* flags);

/* Grid queries. */
long gp_npoints(const gp_handle* h);
int gp_precision_of(const gp_handle* h);

/* Frees the handle and everything it owns (NULL is a no-op). */
int gp_destroy(gp_handle* h);

/* Thread-local message for the last error ("" if none). */
const char* gp_last_error(void);

/* Number of kernels this library has launched in this process (graph
 * replays count every kernel node); for instrumentation. */
unsigned long long gp_kernel_launches(void);

/* The checking build (the paper has no counterpart): libgpe_check.so is this
 * library compiled with GPE_BOUNDS_CHECK, in which every sweep and
 * observables kernel tests its state and shared-memory indices before each
 * access -- a failed test records a code and skips the access (no assert, no
 * trap) -- and every device buffer of a handle or batch sits between two
 * 64 KB guard bands filled with 0xFF bytes (NaN to a kernel that reads them).
 * gp_check_status synchronises the device and sets *first_failure to 0 when
 * no check failed and every live buffer's guard bands are intact (GP_OK); to
 * the code of the first failed index check, or to 1 for an overwritten guard
 * band (GP_ERR_STATE, with the detail in gp_last_error); and to -1 in the
 * normal library, which has no checks (GP_OK).  The failed-check record is
 * cleared by the call. */
int gp_check_status(int* first_failure);

/* Test hook of the bounded device-side waits (the paper has no counterpart).
 * With extra_bytes > 0 every TMA tile load of this handle's sweeps
 * (GP_SHAPE_TMA_X / GP_SHAPE_TMA_YZ) announces extra_bytes more than it
 * moves, so its wait on the tile can never complete: each such sweep gives up
 * after the wait limit (GPE_WAIT_LIMIT_MS at gp_init, default 1000 ms), and
 * the next gp_observables returns GP_ERR_TIMEOUT -- the way the tests check
 * that a wait that runs out ends the kernel and leaves the context usable.
 * 0 restores normal operation; the state is not valid after a timeout
 * (set it again).  0 <= extra_bytes <= 1024, else GP_ERR_INVALID. */
int gp_test_stall_transfers(gp_handle* h, int extra_bytes);

/* Test hook of the one-launch batch form's bounded step waits (the paper has
 * no counterpart).  With extra > 0 every wait of mode 1 asks for extra more
 * finished items than the launch will ever count, so the first y sweep's
 * waits run out after the wait limit and the next gp_batch_observables
 * returns GP_ERR_TIMEOUT with the context still usable.  0 restores normal
 * operation (set the states again).  0 <= extra <= 1 << 20, else
 * GP_ERR_INVALID. */
int gp_test_batch_stall(gp_batch* b, int extra);

#ifdef __cplusplus
}
#endif
#endif /* GPE_H */
