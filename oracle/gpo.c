/*
 * gpo.c -- FP64 CPU oracle for the split-step Crank-Nicolson (CN) propagator of
 * the Gross-Pitaevskii equation  i dphi/dt = [-lap/2 + V + g|phi|^2] phi.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct reference that
 * the CUDA library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * library.
 *
 * The paper ("Solution method" of its program summary) names the scheme --
 * split-step Crank-Nicolson, imaginary- and real-time propagation, 1d/2d/3d
 * Cartesian traps ("Nature of problem") -- and the outputs it reports (energy,
 * chemical potential, rms sizes, densities: abstract, "Summary of revisions").
 * It prints no formula.  The readings used here, step by step:
 *
 *  R1 grid       x_i = -n*dx/2 + i*dx, i = 0..n-1, per axis.
 *  R2 potential  V = (nu^2 x^2 + kappa^2 y^2 + lambda^2 z^2)/2, or a given array.
 *  R3 splitting  one step = N, then L_x, L_y, L_z (Lie order, full dt each).
 *  R4 N          real: phi <- exp(-i dt (V + g|phi|^2)) phi;
 *                imag: phi <- exp(-dt (V + g|phi|^2)) phi; |phi| taken before.
 *  R5 L_d        CN along axis d: with r = i dt/(4 dx^2) (real) or dt/(4 dx^2)
 *                (imag), on every line solve for the interior unknowns
 *                  -r u[k-1] + (1+2r) u[k] - r u[k+1]
 *                      = r p[k-1] + (1-2r) p[k] + r p[k+1],   k = 1..n-2,
 *                with p[0] = p[n-1] = u[0] = u[n-1] = 0 (Dirichlet, ends held
 *                at zero whatever the input holds there).
 *  R6 renorm     imag only: phi <- phi / sqrt(Nrm[phi]) after each step.
 *  R7 Simpson    composite Simpson on the first m points, m = n (n odd) or
 *                n-1 (n even): weights dx/3*(1,4,2,...,2,4,1); tensor product
 *                across axes.
 *  R8 observables on psi = phi/sqrt(Nrm):
 *                E  = int[ 1/2 sum_d |d_d psi|^2 + V|psi|^2 + g/2 |psi|^4 ],
 *                mu = int[ 1/2 sum_d |d_d psi|^2 + V|psi|^2 + g   |psi|^4 ],
 *                rms_d = sqrt(int x_d^2 |psi|^2), rms_r = sqrt(sum_d rms_d^2);
 *                derivative: 4th-order central difference for 2 <= i <= n-3,
 *                2nd-order central at i = 1, n-2, zero at the end points.
 *  R13 spherical  a spherically symmetric 3d trap (the paper's programs cover
 *                "spherically symmetric" traps; "Nature of problem") is solved
 *                for u(r) = sqrt(4 pi) r phi(r) on r_i = i dr, i = 0..n-1:
 *                  i du/dt = [-1/2 d^2/dr^2 + V(r) + g |u|^2/(4 pi r^2)] u,
 *                with u held at zero at r = 0 and r = (n-1) dr, so that R4-R8
 *                apply to u unchanged except for the weight 1/(4 pi r^2) on
 *                the nonlinear term (in N and in the |psi|^4 integral);
 *                int |u|^2 dr = int |phi|^2 d^3r, int |u'|^2 dr = int |grad
 *                phi|^2 d^3r, and rms_x is the 3d rms radius sqrt(<r^2>).
 *                u'(0) is not zero (u ~ sqrt(4 pi) phi(0) r): the derivative
 *                at r = 0 comes from the odd extension u(-r) = -u(r), second
 *                order like the one at i = 1: u'(0) = u_1/dr.
 *  R14 Strang    an optional symmetric splitting (not what the paper's
 *                programs do; second order in dt): N with dt/2, the sweeps
 *                L_x, L_y, L_z with dt, N with dt/2 (|phi| of its own input),
 *                then (imaginary time) the renormalisation of R6.
 *  R15 axisym    circularly symmetric 2d traps (dim 1: phi(rho)) and axially
 *                symmetric 3d traps (dim 2: phi(rho, z)), the paper's other
 *                symmetric programs ("Nature of problem"): axis 0 is rho on
 *                the staggered grid rho_i = (i - 1/2) drho, i = 0..n-1, where
 *                i = 0 is a phantom point at the mirror image of rho_1 and
 *                i = n-1 the outer wall (both held at zero, as in R5); z as
 *                in R1.  The rho part of the Laplacian, (1/rho)(rho phi')',
 *                is the conservative difference
 *                  [(1 + h_i) phi_{i+1} - 2 phi_i + (1 - h_i) phi_{i-1}]/drho^2,
 *                h_i = drho/(2 rho_i), whose coupling to the phantom vanishes
 *                (h_1 = 1): the axis needs no boundary condition.  CN along
 *                rho then has the sub-diagonal -r(1 - h_k) and the super-
 *                diagonal -r(1 + h_k).  Integrals take the midpoint weight
 *                2 pi rho_i drho on i = 1..n-2 along rho (Simpson along z);
 *                the derivative along rho in R8 reads phi_0 as phi_1 (the even
 *                extension across the axis).  N as R4, no extra weight.
 *
 * The tridiagonal solve is written as a back-to-front elimination followed by
 * a front-to-back substitution, with a plain division at every point.
 */
#include "gpo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int gpo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int axis_n(const gpo_problem* p, int d) { return d < p->dim ? p->n[d] : 1; }

long gpo_npoints(const gpo_problem* p) {
  return (long)axis_n(p, 0) * axis_n(p, 1) * axis_n(p, 2);
}

/* R1 */
void gpo_coords(int n, double dx, double* x) {
  for (int i = 0; i < n; ++i) x[i] = -0.5 * n * dx + i * dx;
}

/* R13 */
void gpo_radial_coords(int n, double dr, double* r) {
  for (int i = 0; i < n; ++i) r[i] = i * dr;
}

double gpo_radial_gweight(double r) {
  const double pi = 3.14159265358979323846;
  return r > 0.0 ? 1.0 / (4.0 * pi * r * r) : 0.0;
}

/* R15 */
void gpo_axisym_coords(int n, double drho, double* rho) {
  for (int i = 0; i < n; ++i) rho[i] = (i - 0.5) * drho;
}

void gpo_axisym_weights(int n, double drho, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) w[i] = (i >= 1 && i <= n - 2) ? 2.0 * pi * (i - 0.5) * drho * drho : 0.0;
}

static void axis_coords(const gpo_problem* p, int d, double* x) {
  if (p->geom == 1) gpo_radial_coords(p->n[d], p->dx[d], x);
  else if (p->geom == 2 && d == 0) gpo_axisym_coords(p->n[d], p->dx[d], x);
  else gpo_coords(p->n[d], p->dx[d], x);
}

/* integration weights along axis d < dim (R7, or R15's midpoint rho weight) */
static void axis_weights(const gpo_problem* p, int d, double* w) {
  if (p->geom == 2 && d == 0) gpo_axisym_weights(p->n[d], p->dx[d], w);
  else gpo_simpson_weights(p->n[d], p->dx[d], w);
}

/* weight of the nonlinear term at point q (1, or R13's 1/(4 pi r^2)) */
static double gweight(const gpo_problem* p, long q) {
  return p->geom == 1 ? gpo_radial_gweight(q * p->dx[0]) : 1.0;
}

/* R2 */
void gpo_potential(const gpo_problem* p, double* V) {
  int nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  if (p->V) {
    memcpy(V, p->V, sizeof(double) * gpo_npoints(p));
    return;
  }
  double* x = malloc(sizeof(double) * nx);
  double* y = malloc(sizeof(double) * ny);
  double* z = malloc(sizeof(double) * nz);
  axis_coords(p, 0, x);
  if (p->dim > 1) axis_coords(p, 1, y); else y[0] = 0.0;
  if (p->dim > 2) axis_coords(p, 2, z); else z[0] = 0.0;
  double nu = p->nkl[0], ka = p->dim > 1 ? p->nkl[1] : 0.0, la = p->dim > 2 ? p->nkl[2] : 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        V[i + (long)nx * (j + (long)ny * k)] =
            0.5 * (nu * nu * x[i] * x[i] + ka * ka * y[j] * y[j] + la * la * z[k] * z[k]);
  free(x); free(y); free(z);
}

/* R7 */
void gpo_simpson_weights(int n, double dx, double* w) {
  int m = (n % 2 == 1) ? n : n - 1;
  for (int i = 0; i < n; ++i) w[i] = 0.0;
  if (m == 1) { w[0] = dx; return; }
  for (int i = 0; i < m; ++i) {
    double c;
    if (i == 0 || i == m - 1) c = 1.0;
    else if (i % 2 == 1) c = 4.0;
    else c = 2.0;
    w[i] = c * dx / 3.0;
  }
}

/* R4 */
static void phase_dt(const gpo_problem* p, int imag, double dt, double complex* phi);

void gpo_phase(const gpo_problem* p, int imag, double complex* phi) { phase_dt(p, imag, p->dt, phi); }

static void phase_dt(const gpo_problem* p, int imag, double dt, double complex* phi) {
  long np = gpo_npoints(p);
  double* V = malloc(sizeof(double) * np);
  gpo_potential(p, V);
#pragma omp parallel for schedule(static)
  for (long q = 0; q < np; ++q) {
    double dens = creal(phi[q]) * creal(phi[q]) + cimag(phi[q]) * cimag(phi[q]);
    double theta = dt * (V[q] + p->g * gweight(p, q) * dens);
    if (imag) phi[q] = exp(-theta) * phi[q];
    else phi[q] = cexp(-I * theta) * phi[q];
  }
  free(V);
}

/* R5: one tridiagonal CN solve on a single line of n points, in place.
 * `sign` = +1 for the forward step, -1 for the step with dt -> -dt (used by
 * the adjoint, whose sweep is the conjugate-transposed map). */
/* hl, hr (R15, NULL for 1): the sub- and super-diagonal of row k are
 * -r hl[k] and -r hr[k] (1 - h_k and 1 + h_k along rho). */
static void cn_line(int n, double complex r, double complex* line, long stride,
                    double complex* p, double complex* q, double complex* rhs,
                    const double* hl, const double* hr) {
  if (n < 3) {
    for (int i = 0; i < n; ++i) line[i * stride] = 0.0;
    return;
  }
  int M = n - 2;                 /* unknowns are points 1..n-2 */
  double complex b = 1.0 + 2.0 * r;
  for (int k = 1; k <= M; ++k) {
    double complex left = (k - 1 >= 1) ? line[(k - 1) * stride] : 0.0;
    double complex mid = line[k * stride];
    double complex right = (k + 1 <= M) ? line[(k + 1) * stride] : 0.0;
    double complex rl = hl ? r * hl[k] : r, rr = hr ? r * hr[k] : r;
    rhs[k] = rl * left + (1.0 - 2.0 * r) * mid + rr * right;
  }
  /* back-to-front elimination: u[k] = p[k] - q[k] u[k-1] */
  double complex am = hl ? -r * hl[M] : -r;
  double complex den = b;
  q[M] = am / den;
  p[M] = rhs[M] / den;
  for (int k = M - 1; k >= 1; --k) {
    double complex ak = hl ? -r * hl[k] : -r;   /* sub-diagonal of row k */
    double complex ck = hr ? -r * hr[k] : -r;   /* super-diagonal of row k */
    den = b - ck * q[k + 1];
    q[k] = ak / den;
    p[k] = (rhs[k] - ck * p[k + 1]) / den;
  }
  /* front-to-back substitution, u[0] = 0 */
  double complex prev = 0.0;
  for (int k = 1; k <= M; ++k) {
    double complex u = p[k] - q[k] * prev;
    line[k * stride] = u;
    prev = u;
  }
  line[0] = 0.0;
  line[(long)(n - 1) * stride] = 0.0;
}

void gpo_sweep(const gpo_problem* p, int imag, int axis, double sign, double complex* phi) {
  int nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  int n = axis_n(p, axis);
  double h = p->dx[axis];
  double complex r = imag ? sign * p->dt / (4.0 * h * h) : sign * I * p->dt / (4.0 * h * h);
  long stride = axis == 0 ? 1 : axis == 1 ? nx : (long)nx * ny;
  /* lines: every combination of the other two indices */
  long nlines = gpo_npoints(p) / n;
  /* R15: the rho axis' off-diagonal factors 1 -/+ h_k, h_k = drho/(2 rho_k) */
  double* hl = NULL;
  double* hr = NULL;
  if (p->geom == 2 && axis == 0) {
    hl = malloc(sizeof(double) * n);
    hr = malloc(sizeof(double) * n);
    for (int k = 0; k < n; ++k) {
      double hk = k >= 1 ? 1.0 / (2.0 * k - 1.0) : 0.0;   /* drho / (2 (k - 1/2) drho) */
      hl[k] = 1.0 - hk;
      hr[k] = 1.0 + hk;
    }
  }
#pragma omp parallel
  {
    double complex* pp = malloc(sizeof(double complex) * (n + 1));
    double complex* qq = malloc(sizeof(double complex) * (n + 1));
    double complex* rr = malloc(sizeof(double complex) * (n + 1));
#pragma omp for schedule(static)
    for (long L = 0; L < nlines; ++L) {
      long base;
      if (axis == 0) base = L * nx;                               /* (j,k) */
      else if (axis == 1) base = (L % nx) + (L / nx) * (long)nx * ny; /* (i,k) */
      else base = L;                                              /* (i,j) */
      cn_line(n, r, phi + base, stride, pp, qq, rr, hl, hr);
    }
    free(pp); free(qq); free(rr);
  }
  free(hl);
  free(hr);
  (void)nz;
}

/* R6 helper: plain tensor-product Simpson integral of |phi|^2 */
double gpo_norm(const gpo_problem* p, const double complex* phi) {
  int nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  double* wx = malloc(sizeof(double) * nx);
  double* wy = malloc(sizeof(double) * ny);
  double* wz = malloc(sizeof(double) * nz);
  axis_weights(p, 0, wx);
  if (p->dim > 1) axis_weights(p, 1, wy); else wy[0] = 1.0;
  if (p->dim > 2) axis_weights(p, 2, wz); else wz[0] = 1.0;
  double s = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double complex v = phi[i + (long)nx * (j + (long)ny * k)];
        s += wx[i] * wy[j] * wz[k] * (creal(v) * creal(v) + cimag(v) * cimag(v));
      }
  free(wx); free(wy); free(wz);
  return s;
}

/* R12: the Simpson weights of every dropped axis times |phi|^2, summed;
 * kept axes index the output (their own points are not weighted). */
void gpo_reduced_density(const gpo_problem* p, const double complex* phi, int keep_mask, double* out) {
  int n[3], keep[3];
  double* w[3];
  long stride_out[3], nout = 1;
  for (int d = 0; d < 3; ++d) {
    n[d] = axis_n(p, d);
    keep[d] = d < p->dim && ((keep_mask >> d) & 1);
    w[d] = malloc(sizeof(double) * n[d]);
    if (d < p->dim && !keep[d]) axis_weights(p, d, w[d]);
    else for (int i = 0; i < n[d]; ++i) w[d][i] = 1.0;
    stride_out[d] = keep[d] ? nout : 0;
    if (keep[d]) nout *= n[d];
  }
  for (long o = 0; o < nout; ++o) out[o] = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        const double complex v = phi[i + (long)n[0] * (j + (long)n[1] * k)];
        const long o = i * stride_out[0] + j * stride_out[1] + k * stride_out[2];
        out[o] += w[0][i] * w[1][j] * w[2][k] * (creal(v) * creal(v) + cimag(v) * cimag(v));
      }
  for (int d = 0; d < 3; ++d) free(w[d]);
}

/* R3 + R6 */
void gpo_step(const gpo_problem* p, int imag, double complex* phi) {
  if (p->split == 1) {  /* R14 */
    phase_dt(p, imag, 0.5 * p->dt, phi);
    for (int d = 0; d < p->dim; ++d) gpo_sweep(p, imag, d, 1.0, phi);
    phase_dt(p, imag, 0.5 * p->dt, phi);
  } else {
    gpo_phase(p, imag, phi);
    for (int d = 0; d < p->dim; ++d) gpo_sweep(p, imag, d, 1.0, phi);
  }
  if (imag) {
    double s = 1.0 / sqrt(gpo_norm(p, phi));
    long np = gpo_npoints(p);
    for (long q = 0; q < np; ++q) phi[q] *= s;
  }
}

void gpo_run(const gpo_problem* p, int imag, long nsteps, double complex* phi) {
  for (long t = 0; t < nsteps; ++t) gpo_step(p, imag, phi);
}

/* R8: derivative of a line-sampled function at index i (stride s) */
static double complex deriv(const double complex* f, int n, int i, long s, double h) {
  if (i == 0 || i == n - 1) return 0.0;
  if (i == 1 || i == n - 2) return (f[(i + 1) * s] - f[(i - 1) * s]) / (2.0 * h);
  return (f[(i - 2) * s] - 8.0 * f[(i - 1) * s] + 8.0 * f[(i + 1) * s] - f[(i + 2) * s]) / (12.0 * h);
}

/* R8: out = {norm, energy, mu, rms_x, rms_y, rms_z, rms_r}; density = |phi|^2 */
void gpo_observables(const gpo_problem* p, const double complex* phi, double out[7], double* density) {
  int nx = axis_n(p, 0), ny = axis_n(p, 1), nz = axis_n(p, 2);
  long np = gpo_npoints(p);
  double* V = malloc(sizeof(double) * np);
  gpo_potential(p, V);
  double* w[3];
  double* c[3];
  int nn[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    w[d] = malloc(sizeof(double) * nn[d]);
    c[d] = malloc(sizeof(double) * nn[d]);
    if (d < p->dim) {
      axis_weights(p, d, w[d]);
      axis_coords(p, d, c[d]);
    } else {
      w[d][0] = 1.0;
      c[d][0] = 0.0;
    }
  }
  long stride[3] = {1, nx, (long)nx * ny};
  double nrm = 0, kin = 0, pot = 0, quart = 0, x2[3] = {0, 0, 0};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        long q = i + (long)nx * (j + (long)ny * k);
        double wt = w[0][i] * w[1][j] * w[2][k];
        double dens = creal(phi[q]) * creal(phi[q]) + cimag(phi[q]) * cimag(phi[q]);
        int idx[3] = {i, j, k};
        double grad2 = 0.0;
        for (int d = 0; d < p->dim; ++d) {
          double complex dd = deriv(phi + q - idx[d] * stride[d], nn[d], idx[d], stride[d], p->dx[d]);
          if (p->geom == 1 && idx[d] == 0) dd = phi[q + 1] / p->dx[0];   /* R13 */
          if (p->geom == 2 && d == 0 && (idx[0] == 1 || (idx[0] == 2 && nn[0] >= 5))) {  /* R15: phi_0 as phi_1 */
            double complex f0 = phi[q - idx[0] + 1];
            if (idx[0] == 1) dd = (phi[q + 1] - f0) / (2.0 * p->dx[0]);
            else dd = (f0 - 8.0 * phi[q - 1] + 8.0 * phi[q + 1] - phi[q + 2]) / (12.0 * p->dx[0]);
          }
          grad2 += creal(dd) * creal(dd) + cimag(dd) * cimag(dd);
        }
        nrm += wt * dens;
        kin += wt * 0.5 * grad2;
        pot += wt * V[q] * dens;
        quart += wt * dens * dens * gweight(p, q);
        for (int d = 0; d < p->dim; ++d) x2[d] += wt * c[d][idx[d]] * c[d][idx[d]] * dens;
        if (density) density[q] = dens;
      }
  out[0] = nrm;
  out[1] = kin / nrm + pot / nrm + 0.5 * p->g * quart / (nrm * nrm);
  out[2] = kin / nrm + pot / nrm + p->g * quart / (nrm * nrm);
  double r2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    out[3 + d] = sqrt(x2[d] / nrm);
    r2 += x2[d] / nrm;
  }
  out[6] = sqrt(r2);
  for (int d = 0; d < 3; ++d) { free(w[d]); free(c[d]); }
  free(V);
}

/*
 * Adjoint of the real-time step (the differentiation form of the propagator).
 * Inner product <a,b> = Re sum conj(a) b over grid points; the adjoint state
 * lam = dJ/dRe(phi) + i dJ/dIm(phi).
 *  - L_d is complex-linear, u = C p with C = (1+iA)^-1 (1-iA), A real
 *    symmetric, so lam_in = C^H lam_out, which is the same sweep with dt -> -dt.
 *  - N: u = exp(-i th) p, th = dt (V + g|p|^2).  With s = Im(conj(lam_out) u):
 *        lam_in = exp(+i th) lam_out + 2 g dt s p,
 *        dJ/dV  += dt s (per grid value),   dJ/dg += dt sum s |p|^2.
 * Step order is N, L_x, L_y, L_z, so the reverse is L_z^H, L_y^H, L_x^H, N^H.
 */
void gpo_adjoint_phase(const gpo_problem* p, const double complex* phi_in,
                       double complex* lam, double* dJdV, double* dJdg) {
  long np = gpo_npoints(p);
  double* V = malloc(sizeof(double) * np);
  gpo_potential(p, V);
  double sg = 0.0;
  for (long q = 0; q < np; ++q) {
    double dens = creal(phi_in[q]) * creal(phi_in[q]) + cimag(phi_in[q]) * cimag(phi_in[q]);
    double theta = p->dt * (V[q] + p->g * dens);
    double complex u = cexp(-I * theta) * phi_in[q];
    double s = cimag(conj(lam[q]) * u);
    if (dJdV) dJdV[q] += p->dt * s;
    sg += p->dt * s * dens;
    lam[q] = cexp(I * theta) * lam[q] + 2.0 * p->g * p->dt * s * phi_in[q];
  }
  if (dJdg) *dJdg += sg;
  free(V);
}

/* J = |sum conj(target) phi(T) dV|^2 with dV the cell volume; returns J and
 * fills phiT (optional), dJdV (n points, overwritten) and *dJdg. */
double gpo_adjoint_real(const gpo_problem* p, long nsteps, const double complex* phi0,
                        const double complex* target, double complex* phiT,
                        double* dJdV, double* dJdg) {
  long np = gpo_npoints(p);
  double dvol = 1.0;
  for (int d = 0; d < p->dim; ++d) dvol *= p->dx[d];
  /* forward, keeping the state at the start of every step */
  double complex* hist = malloc(sizeof(double complex) * np * (nsteps + 1));
  memcpy(hist, phi0, sizeof(double complex) * np);
  for (long t = 0; t < nsteps; ++t) {
    memcpy(hist + (t + 1) * np, hist + t * np, sizeof(double complex) * np);
    gpo_step(p, 0, hist + (t + 1) * np);
  }
  const double complex* fin = hist + nsteps * np;
  if (phiT) memcpy(phiT, fin, sizeof(double complex) * np);
  double complex c = 0.0;
  for (long q = 0; q < np; ++q) c += conj(target[q]) * fin[q] * dvol;
  double J = creal(c) * creal(c) + cimag(c) * cimag(c);
  /* terminal adjoint: dJ/dphi* form, lam = 2 c target dV */
  double complex* lam = malloc(sizeof(double complex) * np);
  for (long q = 0; q < np; ++q) lam[q] = 2.0 * c * target[q] * dvol;
  if (dJdV) memset(dJdV, 0, sizeof(double) * np);
  double gsum = 0.0;
  for (long t = nsteps - 1; t >= 0; --t) {
    for (int d = p->dim - 1; d >= 0; --d) gpo_sweep(p, 0, d, -1.0, lam);
    gpo_adjoint_phase(p, hist + t * np, lam, dJdV, &gsum);
  }
  if (dJdg) *dJdg = gsum;
  free(lam);
  free(hist);
  return J;
}
