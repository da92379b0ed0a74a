/*
 * gpo.h -- FP64 CPU oracle for the split-step Crank-Nicolson propagator of the
 * time-dependent Gross-Pitaevskii equation
 *     i dphi/dt = [ -lap/2 + V(r) + g |phi|^2 ] phi
 * (paper: "Solution method" of the program summary -- split-step Crank-Nicolson,
 * imaginary- and real-time propagation; "Nature of problem" -- 1d, 2d, 3d,
 * fully anisotropic Cartesian traps).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library.
 *
 * The paper names the method but prints none of its formulas, so every
 * discretisation detail below is a reading of the method; the readings are
 * listed where each function is defined.
 *
 * Layout: complex interleaved (re, im) doubles, x fastest:
 *     idx = i + nx * (j + ny * k).
 */
#ifndef GPO_H
#define GPO_H
#include <complex.h>

typedef struct {
  int dim;            /* 1, 2 or 3 */
  int n[3];           /* points per axis (trailing entries ignored) */
  double dx[3];       /* grid spacing per axis */
  double dt;          /* time step (imaginary-time step in imag mode) */
  double nkl[3];      /* trap frequencies nu, kappa, lambda */
  double g;           /* nonlinearity */
  const double* V;    /* NULL: harmonic trap; else full potential on the grid */
  int geom;           /* 0: Cartesian; 1: spherically symmetric 3d trap (dim 1, R13);
                         2: circularly (dim 1) / axially (dim 2) symmetric trap, axis 0 = rho (R15) */
  int split;          /* 0: Lie N, L_x, L_y, L_z (R3); 1: Strang N/2, L_x, L_y, L_z, N/2 (R14) */
} gpo_problem;

long gpo_npoints(const gpo_problem* p);
void gpo_coords(int n, double dx, double* x);
/* R13 radial grid r_i = i dr, and the weight 1/(4 pi r^2) of the nonlinear
 * term (0 at r = 0, where u is held at zero) */
void gpo_radial_coords(int n, double dr, double* r);
double gpo_radial_gweight(double r);
void gpo_axisym_coords(int n, double drho, double* rho);     /* R15: rho_i = (i - 1/2) drho */
void gpo_axisym_weights(int n, double drho, double* w);      /* R15: 2 pi rho_i drho on 1..n-2 */
void gpo_potential(const gpo_problem* p, double* V);
void gpo_simpson_weights(int n, double dx, double* w);

void gpo_phase(const gpo_problem* p, int imag, double complex* phi);
void gpo_sweep(const gpo_problem* p, int imag, int axis, double sign, double complex* phi);
void gpo_step(const gpo_problem* p, int imag, double complex* phi);
void gpo_run(const gpo_problem* p, int imag, long nsteps, double complex* phi);

double gpo_norm(const gpo_problem* p, const double complex* phi);
/* R12: reduced (integrated) density on the axes in keep_mask (bit d = axis d
 * kept): out[kept coordinates, x fastest] = sum over the other axes of the
 * Simpson weights times |phi|^2 (the paper's programs write reduced 1d and 2d
 * densities; "Summary of revisions"). */
void gpo_reduced_density(const gpo_problem* p, const double complex* phi, int keep_mask, double* out);
void gpo_observables(const gpo_problem* p, const double complex* phi, double out[7], double* density);

double gpo_adjoint_real(const gpo_problem* p, long nsteps, const double complex* phi0,
                        const double complex* target, double complex* phiT,
                        double* dJdV, double* dJdg);
void gpo_adjoint_phase(const gpo_problem* p, const double complex* phi_in,
                       double complex* lam, double* dJdV, double* dJdg);

int gpo_num_threads(void);
#endif
