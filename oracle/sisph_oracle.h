/*
 * FP64 CPU oracle of the SISPH time step (Muta, Ramachandran & Negi,
 * "An efficient, open source, iterative ISPH scheme", arXiv 1908.01762).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded
 * restatement of the paper's Algorithm 1 used to check the CUDA library and
 * to time a CPU baseline.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA path.
 *
 * Conventions: arrays are in the caller's particle order; neighbour sums run
 * over j in ascending index; all arithmetic is IEEE double, built with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#ifndef SISPH_ORACLE_H
#define SISPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_sim or_sim;

typedef struct {
  int32_t dim;
  double lo[3], hi[3];
  int32_t periodic[3];
  double h, dt, rho0, nu, g[3];
  double alpha, c0;         /* artificial viscosity, alpha = 0 switches it off */
  double eta;               /* 0.01: regulariser in the viscous / PPE terms */
  double omega;             /* 0.5: Jacobi damping (Eq. p-sor) */
  double fs_ratio;          /* 0.8: rho/rho0 below it marks a free surface */
  int32_t min_iter, max_iter;
  double tol;
  int32_t pgrad_symm;       /* 1 "symm" (Eq. mom:sph:press:symm), 0 "asymm" */
  int32_t free_surface;     /* free-surface test and wall-pressure clamp */
  int32_t ustar_slip;       /* slip ghost velocity for u* (Sec. 3.4) */
  int32_t pref_mode;        /* 0 fixed, 1 twice max p after the first solve, 2 external */
  double p_ref;
  double gtvf_hfac;         /* h~ = gtvf_hfac * h */
  int32_t gtvf_K;           /* GTVF sub-steps */
  int32_t residual_form;    /* 0: max(Lambda, sum|p|), 1: max(N_F Lambda, sum|p|) */
  int32_t brute_neighbors;  /* 1: O(N^2) search, 0: cell list */
  int32_t adaptive_dt;      /* 1: next dt from max|u^n| and max|f^n| (Sec. 3.2) */
  int32_t ppe_solver;       /* 0 damped Jacobi (Eq. p-sor), 1 BiCGStab */
} or_params;

typedef struct {
  int32_t iters;
  double residual;
  double lambda;
  int32_t converged;
  int32_t nonfinite;
  double umax;
  double dt;                /* time step this step advanced by */
} or_diag;

void or_default_params(or_params *prm);

/* Quintic spline (support 3h) and dW/dr; sigma normalised in 1, 2 or 3 D. */
double or_kernel_w(double r, double h, int32_t dim);
double or_kernel_dwdr(double r, double h, int32_t dim);

/* Neighbour lists of arbitrary points.  counts[n]; idx receives the lists
 * concatenated (ascending j), capacity `cap` entries; returns the total
 * number of pairs, or -1 if `cap` is too small. */
int64_t or_neighbors(const or_params *prm, int64_t n, const double *x, const double *y,
                     const double *z, int32_t *counts, int32_t *idx, int64_t cap);

or_sim *or_create(const or_params *prm, int64_t n, const double *x, const double *y,
                  const double *z, const double *u, const double *v, const double *w,
                  const double *m, const double *rho, const double *p, const int32_t *kind,
                  const double *wall_u, const double *wall_v, const double *wall_w);
void or_destroy(or_sim *s);

/* Fields: "x","y","z","u","v","w","ut","vt","wt","p","rho","m","nx","ny","nz",
 * "ugx","ugy","ugz","rhs","diag","fx","fy","fz","dx","dy","dz".
 * f holds the last force computed (stage 1, pressure gradient, or the first
 * GTVF sub-step); d the GTVF displacement r^K - r^0. */
int32_t or_get(const or_sim *s, const char *field, double *out);
int32_t or_set(or_sim *s, const char *field, const double *in);

/* Individual steps of Algorithm 1 (each cites its passage in the .c file). */
int64_t or_build_neighbors(or_sim *s);
int64_t or_neighbor_list(const or_sim *s, int32_t *counts, int32_t *idx, int64_t cap);
void or_density(or_sim *s);
void or_wall_normals(or_sim *s);
void or_ghost_velocity(or_sim *s, int32_t slip);
void or_stage1(or_sim *s);
void or_ppe_setup(or_sim *s);
void or_ppe_iterate(or_sim *s, or_diag *d);
void or_ppe_bicgstab(or_sim *s, or_diag *d);
void or_ppe_apply(const or_sim *s, const double *p, double *out);
int64_t or_ppe_export(const or_sim *s, double *diag, double *rhs, int32_t *active,
                      double *fac, double *wall_s, double *wall_h, double *wall_w);
void or_pressure_gradient(or_sim *s);
void or_gtvf(or_sim *s);
void or_update(or_sim *s);
int32_t or_step(or_sim *s, int32_t nsteps, or_diag *d);
/* PPE alone on the current state (positions, u* in u, rho, p). */
int32_t or_ppe_solve(or_sim *s, double tol, int32_t max_iter, or_diag *d);
double or_get_pref(const or_sim *s);
/* Time step of the next step (changes with the adaptive rule). */
double or_get_dt(const or_sim *s);

#ifdef __cplusplus
}
#endif
#endif
