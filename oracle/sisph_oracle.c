/*
 * FP64 CPU oracle of the SISPH time step (arXiv 1908.01762).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, obviously-correct restatement of
 * the paper's Algorithm 1 in the paper's order and notation.  It is used by
 * the test suite to check the CUDA library and by the benchmark as a timed
 * CPU baseline.  Nothing in the product path may call it.  It shares no code
 * with the CUDA library.
 *
 * Readings of passages that the paper leaves open are marked "Reading:".
 * The wall normals are pinned by the symmetry of a three-layer wall (no
 * normal on the middle layer, +-y on the others, the bisector at a corner);
 * the two lengths below which a normal is taken as zero are readings whose
 * exact values the paper does not fix: any value between rounding noise and
 * the smallest real gradient gives the same normals.  Both ghost velocity
 * forms are pinned by a uniform flow along a resting floor, the artificial
 * stress by the divergence of a linear tensor field and by momentum
 * conservation.  The
 * artificial-viscosity form (Monaghan's, read from a garbled equation) is
 * pinned by its invariants only: momentum conservation, no force between
 * receding pairs, and a force that opposes compression.
 * Build: gcc -O2 -std=c11 -D_GNU_SOURCE (for M_PI) -ffp-contract=off -fPIC -shared.
 */
#include "sisph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FLUID 0
#define WALL 1

struct or_sim {
  or_params prm;
  int64_t n;
  double *x[3], *xn[3];          /* positions r, and r^n saved during a step */
  double *u[3], *ut[3];          /* velocity u and transport velocity u~ */
  double *ug[3];                 /* wall ghost velocity */
  double *uw[3];                 /* prescribed wall velocity */
  double *nrm[3];                /* wall unit normals (out of the solid) */
  double *m, *rho, *p, *pnew;
  int32_t *kind;
  int64_t *nstart;               /* CSR neighbour lists, ascending j */
  int32_t *nidx;
  int64_t ncap;
  double *rhs, *diag, *fac;      /* PPE: RHS_i, D_ii, fac_ij per CSR entry */
  int32_t *active;
  double *ws, *wh;               /* wall Shepard sums: sum_f W_wf, (g.sum rho_f r_wf W_wf) */
  double *f[3], *d[3], *vg[3];   /* force scratch, GTVF displacement and velocity */
  double lambda;
  int32_t pref_set;
  double p_ref;
  double fmax;                   /* max_i |f_i| over fluid of the last pressure gradient */
  or_diag last;
};

void or_default_params(or_params *prm) {
  memset(prm, 0, sizeof(*prm));
  prm->dim = 2;
  prm->eta = 0.01;
  prm->omega = 0.5;
  prm->fs_ratio = 0.8;
  prm->min_iter = 2;
  prm->max_iter = 1000;
  prm->tol = 1e-2;
  prm->gtvf_hfac = 1.0;
  prm->gtvf_K = 1;
  prm->ustar_slip = 1;
}

/* ---------------------------------------------------------------------------
 * Quintic spline (Sec. 2.1 names "the quintic spline"; reading: the
 * Morris 1997 quintic with support 3h),
 *   W(q) = sigma [ (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5 ],  q = r/h,
 * each bracket only where positive; sigma = 1/(120 h), 7/(478 pi h^2),
 * 1/(120 pi h^3) in 1, 2, 3 dimensions (unit integral).
 * ------------------------------------------------------------------------- */
static double or_sigma(double h, int32_t dim) {
  if (dim == 1) return 1.0 / (120.0 * h);
  if (dim == 2) return 7.0 / (478.0 * M_PI * h * h);
  return 1.0 / (120.0 * M_PI * h * h * h);
}

static double p5(double t) { return t * t * t * t * t; }
static double p4(double t) { return t * t * t * t; }

double or_kernel_w(double r, double h, int32_t dim) {
  double q = r / h;
  double w = 0.0;
  if (q < 3.0) w += p5(3.0 - q);
  if (q < 2.0) w -= 6.0 * p5(2.0 - q);
  if (q < 1.0) w += 15.0 * p5(1.0 - q);
  return or_sigma(h, dim) * w;
}

double or_kernel_dwdr(double r, double h, int32_t dim) {
  double q = r / h;
  double dw = 0.0;
  if (q < 3.0) dw -= 5.0 * p4(3.0 - q);
  if (q < 2.0) dw += 30.0 * p4(2.0 - q);
  if (q < 1.0) dw -= 75.0 * p4(1.0 - q);
  return or_sigma(h, dim) * dw / h;
}

/* ---------------------------------------------------------------------------
 * Pair geometry.  r_ij = r_i - r_j (Sec. 2.1), minimum image in periodic
 * directions.  Reading: the neighbour set N(i) is {j : |r_ij|^2 < (3h)^2}
 * with |r_ij|^2 = dx*dx + dy*dy (+ dz*dz) evaluated left to right without
 * fused multiply-adds; i itself is included.
 * ------------------------------------------------------------------------- */
static double or_min_image(double d, double L, int32_t per) {
  if (per) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
  }
  return d;
}

static double or_pair(const or_params *prm, const double *const x[3], int64_t i, int64_t j,
                      double dx[3]) {
  double r2 = 0.0;
  for (int k = 0; k < 3; ++k) dx[k] = 0.0;
  for (int k = 0; k < prm->dim; ++k) {
    double L = prm->hi[k] - prm->lo[k];
    dx[k] = or_min_image(x[k][i] - x[k][j], L, prm->periodic[k]);
  }
  r2 = dx[0] * dx[0];
  r2 = r2 + dx[1] * dx[1];
  if (prm->dim == 3) r2 = r2 + dx[2] * dx[2];
  return r2;
}

static double or_cut2(const or_params *prm) { return (3.0 * prm->h) * (3.0 * prm->h); }

static void or_wrap(const or_params *prm, double *xk, int k) {
  if (!prm->periodic[k]) return;
  double L = prm->hi[k] - prm->lo[k];
  if (*xk >= prm->hi[k]) *xk -= L;
  else if (*xk < prm->lo[k]) *xk += L;
}

/* ---------------------------------------------------------------------------
 * Neighbour search.  The paper delegates it to PySPH (Sec. 3.3); both
 * variants below return N(i) as defined above, ascending in j.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t *start;
  int32_t *idx;
  int64_t cap;
} or_csr;

static int or_csr_push(or_csr *c, int64_t pos, int32_t j) {
  if (pos >= c->cap) {
    int64_t nc = c->cap ? c->cap * 2 : 1024;
    int32_t *ni = (int32_t *)realloc(c->idx, (size_t)nc * sizeof(int32_t));
    if (!ni) return -1;
    c->idx = ni;
    c->cap = nc;
  }
  c->idx[pos] = j;
  return 0;
}

static int or_cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static int or_search(const or_params *prm, int64_t n, const double *const x[3], or_csr *c) {
  double cut2 = or_cut2(prm);
  int64_t pos = 0;
  c->start[0] = 0;
  int brute = prm->brute_neighbors;
  int64_t nc[3] = {1, 1, 1};
  double lc[3] = {1, 1, 1};
  for (int k = 0; k < prm->dim; ++k) {
    double L = prm->hi[k] - prm->lo[k];
    if (prm->periodic[k]) {
      nc[k] = (int64_t)floor(L / (3.0 * prm->h));
      if (nc[k] < 3) brute = 1;
      lc[k] = L / (double)nc[k];
    } else {
      lc[k] = 3.0 * prm->h;
      nc[k] = (int64_t)ceil(L / lc[k]);
      if (nc[k] < 1) nc[k] = 1;
    }
  }
  if (brute) {
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = 0; j < n; ++j) {
        double dx[3];
        if (or_pair(prm, x, i, j, dx) < cut2) {
          if (or_csr_push(c, pos, (int32_t)j)) return -1;
          ++pos;
        }
      }
      c->start[i + 1] = pos;
    }
    return 0;
  }
  /* cell list: bin particles, then scan the 3^d surrounding cells */
  int64_t ncell = nc[0] * nc[1] * nc[2];
  int64_t *cell = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *fill = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
  int32_t *cand = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!cell || !cnt || !order || !fill || !cand) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cc[3] = {0, 0, 0};
    for (int k = 0; k < prm->dim; ++k) {
      int64_t t = (int64_t)floor((x[k][i] - prm->lo[k]) / lc[k]);
      if (t < 0) t = prm->periodic[k] ? nc[k] - 1 : 0;
      if (t >= nc[k]) t = prm->periodic[k] ? 0 : nc[k] - 1;
      cc[k] = t;
    }
    cell[i] = (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
    cnt[cell[i] + 1]++;
  }
  for (int64_t q = 0; q < ncell; ++q) cnt[q + 1] += cnt[q];
  for (int64_t i = 0; i < n; ++i) order[cnt[cell[i]] + fill[cell[i]]++] = i;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ci[3];
    ci[0] = cell[i] % nc[0];
    ci[1] = (cell[i] / nc[0]) % nc[1];
    ci[2] = cell[i] / (nc[0] * nc[1]);
    int64_t ncand = 0;
    int lim[3];
    for (int k = 0; k < 3; ++k) lim[k] = (k < prm->dim) ? 1 : 0;
    for (int a = -lim[2]; a <= lim[2]; ++a)
      for (int b = -lim[1]; b <= lim[1]; ++b)
        for (int e = -lim[0]; e <= lim[0]; ++e) {
          int64_t cj[3] = {ci[0] + e, ci[1] + b, ci[2] + a};
          int skip = 0;
          for (int k = 0; k < prm->dim; ++k) {
            if (cj[k] < 0 || cj[k] >= nc[k]) {
              if (prm->periodic[k]) cj[k] = (cj[k] + nc[k]) % nc[k];
              else skip = 1;
            }
          }
          if (skip) continue;
          int64_t q = (cj[2] * nc[1] + cj[1]) * nc[0] + cj[0];
          for (int64_t t = cnt[q]; t < cnt[q + 1]; ++t) {
            int64_t j = order[t];
            double dx[3];
            if (or_pair(prm, x, i, j, dx) < cut2) cand[ncand++] = (int32_t)j;
          }
        }
    qsort(cand, (size_t)ncand, sizeof(int32_t), or_cmp_i32);
    for (int64_t t = 0; t < ncand; ++t) {
      if (or_csr_push(c, pos, cand[t])) return -1;
      ++pos;
    }
    c->start[i + 1] = pos;
  }
  free(cell); free(cnt); free(order); free(fill); free(cand);
  return 0;
}

int64_t or_neighbors(const or_params *prm, int64_t n, const double *x, const double *y,
                     const double *z, int32_t *counts, int32_t *idx, int64_t cap) {
  const double *xs[3] = {x, y, z ? z : x};
  or_csr c = {0, 0, 0};
  c.start = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  if (!c.start || or_search(prm, n, xs, &c)) { free(c.start); free(c.idx); return -2; }
  int64_t tot = c.start[n];
  if (tot > cap) { free(c.start); free(c.idx); return -1; }
  for (int64_t i = 0; i < n; ++i) counts[i] = (int32_t)(c.start[i + 1] - c.start[i]);
  if (tot) memcpy(idx, c.idx, (size_t)tot * sizeof(int32_t));
  free(c.start); free(c.idx);
  return tot;
}

/* ---------------------------------------------------------------------------
 * Simulation state
 * ------------------------------------------------------------------------- */
static double *or_alloc(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

or_sim *or_create(const or_params *prm, int64_t n, const double *x, const double *y,
                  const double *z, const double *u, const double *v, const double *w,
                  const double *m, const double *rho, const double *p, const int32_t *kind,
                  const double *wall_u, const double *wall_v, const double *wall_w) {
  or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
  if (!s) return NULL;
  s->prm = *prm;
  s->n = n;
  const double *xi[3] = {x, y, z};
  const double *ui[3] = {u, v, w};
  const double *wi[3] = {wall_u, wall_v, wall_w};
  for (int k = 0; k < 3; ++k) {
    s->x[k] = or_alloc(n); s->xn[k] = or_alloc(n); s->u[k] = or_alloc(n);
    s->ut[k] = or_alloc(n); s->ug[k] = or_alloc(n); s->uw[k] = or_alloc(n);
    s->nrm[k] = or_alloc(n); s->f[k] = or_alloc(n); s->d[k] = or_alloc(n);
    s->vg[k] = or_alloc(n);
    for (int64_t i = 0; i < n; ++i) {
      s->x[k][i] = (k < prm->dim && xi[k]) ? xi[k][i] : 0.0;
      s->u[k][i] = (k < prm->dim && ui[k]) ? ui[k][i] : 0.0;
      s->uw[k][i] = (k < prm->dim && wi[k]) ? wi[k][i] : 0.0;
    }
  }
  s->m = or_alloc(n); s->rho = or_alloc(n); s->p = or_alloc(n); s->pnew = or_alloc(n);
  s->rhs = or_alloc(n); s->diag = or_alloc(n); s->ws = or_alloc(n); s->wh = or_alloc(n);
  s->kind = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->active = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  s->nstart = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    s->kind[i] = kind ? kind[i] : FLUID;
    s->m[i] = m[i];
    /* Reading: wall particles keep rho = rho0; fluid rho starts from input. */
    s->rho[i] = (s->kind[i] == WALL || !rho) ? prm->rho0 : rho[i];
    s->p[i] = p ? p[i] : 0.0;
    for (int k = 0; k < 3; ++k) {
      /* Walls carry their prescribed velocity; fluid starts with u~ = u. */
      if (s->kind[i] == WALL) s->u[k][i] = s->uw[k][i];
      s->ut[k][i] = s->u[k][i];
    }
  }
  s->p_ref = prm->p_ref;
  s->pref_set = (prm->pref_mode == 1) ? 0 : 1;
  /* wall normals from the initial positions (Sec. 3.4.1); walls never move */
  if (or_build_neighbors(s) < 0) { or_destroy(s); return NULL; }
  or_wall_normals(s);
  return s;
}

void or_destroy(or_sim *s) {
  if (!s) return;
  for (int k = 0; k < 3; ++k) {
    free(s->x[k]); free(s->xn[k]); free(s->u[k]); free(s->ut[k]); free(s->ug[k]);
    free(s->uw[k]); free(s->nrm[k]); free(s->f[k]); free(s->d[k]); free(s->vg[k]);
  }
  free(s->m); free(s->rho); free(s->p); free(s->pnew); free(s->rhs); free(s->diag);
  free(s->ws); free(s->wh); free(s->kind); free(s->active); free(s->nstart);
  free(s->nidx); free(s->fac);
  free(s);
}

static double *or_field(const or_sim *s, const char *f) {
  static const char *names3[] = {"x", "y", "z", "u", "v", "w", "ut", "vt", "wt",
                                 "nx", "ny", "nz", "ugx", "ugy", "ugz", "fx", "fy", "fz",
                                 "dx", "dy", "dz"};
  for (int t = 0; t < 21; ++t) {
    if (strcmp(f, names3[t]) == 0) {
      int grp = t / 3, k = t % 3;
      if (grp == 0) return s->x[k];
      if (grp == 1) return s->u[k];
      if (grp == 2) return s->ut[k];
      if (grp == 3) return s->nrm[k];
      if (grp == 4) return s->ug[k];
      if (grp == 5) return s->f[k];
      return s->d[k];
    }
  }
  if (!strcmp(f, "p")) return s->p;
  if (!strcmp(f, "rho")) return s->rho;
  if (!strcmp(f, "m")) return s->m;
  if (!strcmp(f, "rhs")) return s->rhs;
  if (!strcmp(f, "diag")) return s->diag;
  return NULL;
}

int32_t or_get(const or_sim *s, const char *field, double *out) {
  double *a = or_field(s, field);
  if (!a) return -1;
  memcpy(out, a, (size_t)s->n * sizeof(double));
  return 0;
}

int32_t or_set(or_sim *s, const char *field, const double *in) {
  double *a = or_field(s, field);
  if (!a) return -1;
  memcpy(a, in, (size_t)s->n * sizeof(double));
  return 0;
}

double or_get_pref(const or_sim *s) { return s->p_ref; }
double or_get_dt(const or_sim *s) { return s->prm.dt; }

int64_t or_build_neighbors(or_sim *s) {
  or_csr c = {s->nstart, s->nidx, s->ncap};
  const double *xs[3] = {s->x[0], s->x[1], s->x[2]};
  int rc = or_search(&s->prm, s->n, xs, &c);
  s->nidx = c.idx;
  s->ncap = c.cap;
  if (rc) return -1;
  free(s->fac);
  s->fac = or_alloc(s->nstart[s->n]);
  return s->nstart[s->n];
}

int64_t or_neighbor_list(const or_sim *s, int32_t *counts, int32_t *idx, int64_t cap) {
  int64_t tot = s->nstart[s->n];
  if (tot > cap) return -1;
  for (int64_t i = 0; i < s->n; ++i) counts[i] = (int32_t)(s->nstart[i + 1] - s->nstart[i]);
  if (tot) memcpy(idx, s->nidx, (size_t)tot * sizeof(int32_t));
  return tot;
}

/* grad_i W_ij = W'(r) r_ij / r for r > 0, zero at r = 0 (Sec. 2.1). */
static double or_grad(const or_sim *s, int64_t i, int64_t j, double hk, double dx[3],
                      double g[3], double *r2out) {
  double r2 = or_pair(&s->prm, (const double *const *)s->x, i, j, dx);
  double r = sqrt(r2);
  double fr = (r > 0.0) ? or_kernel_dwdr(r, hk, s->prm.dim) / r : 0.0;
  for (int k = 0; k < 3; ++k) g[k] = fr * dx[k];
  if (r2out) *r2out = r2;
  return r;
}

static double or_dot(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ---------------------------------------------------------------------------
 * Summation density, Eq. summation_density: rho_i = sum_j m_j W_ij over all
 * neighbours (fluid and wall).  Reading: walls keep rho = rho0.
 * ------------------------------------------------------------------------- */
void or_density(or_sim *s) {
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->kind[i] != FLUID) { s->rho[i] = s->prm.rho0; continue; }
    double acc = 0.0;
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      double dx[3];
      double r2 = or_pair(&s->prm, (const double *const *)s->x, i, j, dx);
      acc += s->m[j] * or_kernel_w(sqrt(r2), s->prm.h, s->prm.dim);
    }
    s->rho[i] = acc;
  }
}

/* ---------------------------------------------------------------------------
 * Wall normals, Sec. 3.4.1, Eqs. normal-approx and normal:
 *   n*_i = sum_j -(m_j/rho_j) grad_i W_ij, zeroed if |n*| < 1/(4h), else
 *   normalised; n_i = sum_j (m_j/rho_j) n*_j W_ij, normalised.
 * Reading: both sums run over wall neighbours only (the normal of the solid
 * from the solid's own particles, pointing out of the solid), and a smoothed
 * normal shorter than 1e-6 (a cancelled average of unit vectors) is zero.
 * ------------------------------------------------------------------------- */
void or_wall_normals(or_sim *s) {
  int64_t n = s->n;
  double *ns[3];
  for (int k = 0; k < 3; ++k) ns[k] = or_alloc(n);
  double h = s->prm.h;
  for (int64_t i = 0; i < n; ++i) {
    if (s->kind[i] != WALL) continue;
    double acc[3] = {0, 0, 0};
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (s->kind[j] != WALL) continue;
      double dx[3], g[3];
      or_grad(s, i, j, h, dx, g, NULL);
      double vj = s->m[j] / s->rho[j];
      for (int k = 0; k < 3; ++k) acc[k] -= vj * g[k];
    }
    double mag = sqrt(or_dot(acc, acc));
    const int keep = mag >= 1.0 / (4.0 * h);
    for (int k = 0; k < 3; ++k) ns[k][i] = keep ? acc[k] / mag : 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) s->nrm[k][i] = 0.0;
    if (s->kind[i] != WALL) continue;
    double acc[3] = {0, 0, 0};
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (s->kind[j] != WALL) continue;
      double dx[3];
      double r2 = or_pair(&s->prm, (const double *const *)s->x, i, j, dx);
      double wv = (s->m[j] / s->rho[j]) * or_kernel_w(sqrt(r2), h, s->prm.dim);
      for (int k = 0; k < 3; ++k) acc[k] += wv * ns[k][j];
    }
    double mag = sqrt(or_dot(acc, acc));
    if (mag > 1e-6)
      for (int k = 0; k < 3; ++k) s->nrm[k][i] = acc[k] / mag;
  }
  for (int k = 0; k < 3; ++k) free(ns[k]);
}

/* ---------------------------------------------------------------------------
 * Wall ghost velocity, Sec. 3.4, Eqs. vf, vg-adami, vg-no-normal.
 * No-slip (stage 1, used by the viscous and artificial-viscosity terms):
 *   u~_w = sum_f u_f W(r_wf, h/2) / sum_f W(r_wf, h/2),  u_w = 2 u_wall - u~_w,
 * then the component into the solid (u_w . n < 0) is removed.
 * Reading: with no fluid inside the h/2 support, u~_w = u_wall.
 * Slip (stage 2, the u* seen by the PPE source term, Sec. 3.4 last
 * paragraph).  Reading: the wall carries the Shepard extension of the fluid's
 * own u*, u*_w = sum_f u*_f W(r_wf, h) / sum_f W(r_wf, h) (u_wall when no
 * fluid is in range), with no reflection and no normal removal.  The normal
 * condition is then imposed once, by the wall pressure of Eq. p-shepard: a
 * uniform u* (fluid at rest under gravity) gives no source term and the
 * hydrostatic pressure solves the PPE, whereas reflecting the normal
 * component as well would impose the wall condition twice.
 * ------------------------------------------------------------------------- */
void or_ghost_velocity(or_sim *s, int32_t slip) {
  double hk = slip ? s->prm.h : 0.5 * s->prm.h;
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->kind[i] != WALL) continue;
    double sw = 0.0, su[3] = {0, 0, 0};
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (s->kind[j] != FLUID) continue;
      double dx[3];
      double r2 = or_pair(&s->prm, (const double *const *)s->x, i, j, dx);
      double wv = or_kernel_w(sqrt(r2), hk, s->prm.dim);
      sw += wv;
      for (int k = 0; k < 3; ++k) su[k] += s->u[k][j] * wv;
    }
    double ut[3], ug[3], nn[3];
    for (int k = 0; k < 3; ++k) {
      ut[k] = (sw > 0.0) ? su[k] / sw : s->uw[k][i];
      nn[k] = s->nrm[k][i];
    }
    if (slip) {
      for (int k = 0; k < 3; ++k) s->ug[k][i] = ut[k];
      continue;
    }
    for (int k = 0; k < 3; ++k) ug[k] = 2.0 * s->uw[k][i] - ut[k];
    double un = or_dot(ug, nn);
    if (un < 0.0)
      for (int k = 0; k < 3; ++k) ug[k] -= un * nn[k];
    for (int k = 0; k < 3; ++k) s->ug[k][i] = ug[k];
  }
}

static double or_vel(const or_sim *s, int64_t j, int k) {
  return (s->kind[j] == WALL) ? s->ug[k][j] : s->u[k][j];
}

/* ---------------------------------------------------------------------------
 * Stage 1 (Algorithm 1, predict position and velocity):
 *   r*_i = r^n_i + dt u~^n_i                                   (Eq. int:rnp1)
 *   u*_i = u^n_i + dt (f_visc + f_avisc + f_astress + f_b)      (Eq. int:vint)
 * f_visc  (Eq. mom:sph:visc): sum_j m_j 4 nu/(rho_i+rho_j)
 *                             (r_ij . gradW)/(r^2 + eta h^2) u_ij
 * f_avisc (Eq. mom:sph:av; reading: Monaghan's form with the mass and the
 *          sign restored): -sum_j m_j Pi_ij gradW,
 *          Pi_ij = -alpha h c phi_ij / rho_bar when u_ij . r_ij < 0,
 *          phi_ij = u_ij . r_ij / (r^2 + eta h^2), rho_bar = (rho_i+rho_j)/2
 * f_astress (Eq. mom:sph:gtvf:stress; reading: with m_j and . gradW):
 *          sum_j m_j (A_i/rho_i^2 + A_j/rho_j^2) . gradW,
 *          A = rho u (x) (u~ - u), over fluid neighbours
 * f_b = g.  Walls enter through their ghost velocity.
 * ------------------------------------------------------------------------- */
void or_stage1(or_sim *s) {
  const or_params *P = &s->prm;
  double h = P->h, eh2 = P->eta * h * h;
  int64_t n = s->n;
  double *us[3];
  for (int k = 0; k < 3; ++k) us[k] = or_alloc(n);
  for (int64_t i = 0; i < n; ++i) {
    if (s->kind[i] != FLUID) continue;
    double fi[3] = {P->g[0], P->g[1], P->g[2]};
    if (P->dim == 2) fi[2] = 0.0;
    double ui[3] = {s->u[0][i], s->u[1][i], s->u[2][i]};
    double ri = s->rho[i];
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (j == i) continue;
      double dx[3], g[3], r2;
      or_grad(s, i, j, h, dx, g, &r2);
      double rj = s->rho[j], mj = s->m[j];
      double uj[3] = {or_vel(s, j, 0), or_vel(s, j, 1), or_vel(s, j, 2)};
      double uij[3] = {ui[0] - uj[0], ui[1] - uj[1], ui[2] - uj[2]};
      double rdw = or_dot(dx, g);
      double visc = mj * 4.0 * P->nu / (ri + rj) * rdw / (r2 + eh2);
      for (int k = 0; k < 3; ++k) fi[k] += visc * uij[k];
      if (P->alpha > 0.0) {
        double vr = or_dot(uij, dx);
        if (vr < 0.0) {
          double phi = vr / (r2 + eh2);
          double pi_ij = -P->alpha * h * P->c0 * phi / (0.5 * (ri + rj));
          for (int k = 0; k < 3; ++k) fi[k] -= mj * pi_ij * g[k];
        }
      }
      if (s->kind[j] == FLUID) {
        double dti[3] = {s->ut[0][i] - ui[0], s->ut[1][i] - ui[1], s->ut[2][i] - ui[2]};
        double dtj[3] = {s->ut[0][j] - uj[0], s->ut[1][j] - uj[1], s->ut[2][j] - uj[2]};
        double ai = or_dot(dti, g) / ri, aj = or_dot(dtj, g) / rj;
        for (int k = 0; k < 3; ++k) fi[k] += mj * (ui[k] * ai + uj[k] * aj);
      }
    }
    for (int k = 0; k < 3; ++k) {
      s->f[k][i] = fi[k];
      us[k][i] = ui[k] + P->dt * fi[k];
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) s->xn[k][i] = s->x[k][i];
    if (s->kind[i] != FLUID) continue;
    for (int k = 0; k < P->dim; ++k) {
      s->u[k][i] = us[k][i];
      double xk = s->x[k][i] + P->dt * s->ut[k][i];
      or_wrap(P, &xk, k);
      s->x[k][i] = xk;
    }
  }
  for (int k = 0; k < 3; ++k) free(us[k]);
}

/* ---------------------------------------------------------------------------
 * PPE set-up, Eqs. sph-ppe, iterative-p, coeff, coeff1 (Sec. 3):
 *   RHS_i  = sum_j -(m_j / (rho_j dt)) u*_ij . grad_i W_ij
 *   fac_ij = 4 m_j / (rho_i (rho_i + rho_j)) (r_ij . grad_i W_ij)/(r^2 + eta h^2)
 *   D_ii = sum_j fac_ij,  OD_ij = -fac_ij
 * Reading: the regulariser is eta h^2 as in Eq. mom:sph:visc.
 * A fluid particle with D_ii = 0, or with rho_i/rho0 < 0.8 when the free
 * surface is on, keeps p = 0 (Sec. 3).
 * Wall constants of Eq. p-shepard: S_w = sum_f W_wf and
 * H_w = (g - a_w) . sum_f rho_f r_wf W_wf with r_wf = r_w - r_f, a_w = 0.
 * ------------------------------------------------------------------------- */
void or_ppe_setup(or_sim *s) {
  const or_params *P = &s->prm;
  double h = P->h, eh2 = P->eta * h * h;
  double lam = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    s->rhs[i] = 0.0; s->diag[i] = 0.0; s->active[i] = 0; s->ws[i] = 0.0; s->wh[i] = 0.0;
    if (s->kind[i] == FLUID) {
      double ri = s->rho[i];
      double rhs = 0.0, dg = 0.0;
      for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
        int64_t j = s->nidx[t];
        s->fac[t] = 0.0;
        if (j == i) continue;
        double dx[3], g[3], r2;
        or_grad(s, i, j, h, dx, g, &r2);
        double rj = s->rho[j], mj = s->m[j];
        double uij[3];
        for (int k = 0; k < 3; ++k) uij[k] = s->u[k][i] - or_vel(s, j, k);
        rhs += -mj / (rj * P->dt) * or_dot(uij, g);
        double fac = 4.0 * mj / (ri * (ri + rj)) * or_dot(dx, g) / (r2 + eh2);
        s->fac[t] = fac;
        dg += fac;
      }
      s->rhs[i] = rhs;
      s->diag[i] = dg;
      int fs = P->free_surface && (ri / P->rho0 < P->fs_ratio);
      s->active[i] = (dg != 0.0) && !fs;
      if (!s->active[i]) s->p[i] = 0.0;
      else {
        double a = fabs(rhs / dg);
        if (a > lam) lam = a;
      }
    } else {
      double sw = 0.0, acc[3] = {0, 0, 0};
      for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
        int64_t j = s->nidx[t];
        s->fac[t] = 0.0;
        if (s->kind[j] != FLUID) continue;
        double dx[3];
        double r2 = or_pair(P, (const double *const *)s->x, i, j, dx);
        double wv = or_kernel_w(sqrt(r2), h, P->dim);
        s->fac[t] = wv;
        sw += wv;
        for (int k = 0; k < 3; ++k) acc[k] += s->rho[j] * dx[k] * wv;
      }
      double gv[3] = {P->g[0], P->g[1], P->dim == 3 ? P->g[2] : 0.0};
      s->ws[i] = sw;
      s->wh[i] = or_dot(gv, acc);
    }
  }
  s->lambda = lam;
}

/* Eq. p-shepard with the free-surface clamp p_w >= 0 (Sec. 3.4). */
static void or_wall_pressure(or_sim *s) {
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->kind[i] != WALL) continue;
    double acc = 0.0;
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (s->kind[j] != FLUID) continue;
      acc += s->p[j] * s->fac[t];
    }
    double pw = (s->ws[i] > 0.0) ? (acc + s->wh[i]) / s->ws[i] : 0.0;
    if (s->prm.free_surface && pw < 0.0) pw = 0.0;
    s->p[i] = pw;
  }
}

/* ---------------------------------------------------------------------------
 * Damped-Jacobi sweeps, Eq. p-sor with omega = 0.5, and the convergence test
 * of Eq. convergence:
 *   p_i^{k+1} = omega (RHS_i - sum_j OD_ij p_j^k)/D_ii + (1 - omega) p_i^k
 *   res = sum_i |p^{k+1}_i - p^k_i| / max(Lambda, sum_i |p^{k+1}_i|),
 *   Lambda = max_i |RHS_i / D_ii|.
 * Every neighbour uses p^k (Jacobi, double-buffered).  Each sweep first
 * extrapolates the wall pressure from the current fluid pressure (Sec. 3.4).
 * Reading: sums run over fluid particles; iterate while (k < min_iter or
 * res >= tol) and k < max_iter (the inverted test and max(1, .) in the
 * algorithm listing are read as typos); after the last sweep the walls are
 * extrapolated once more so that they match the final fluid pressure.
 * ------------------------------------------------------------------------- */
void or_ppe_iterate(or_sim *s, or_diag *d) {
  const or_params *P = &s->prm;
  int64_t n = s->n;
  int64_t nfluid = 0;
  for (int64_t i = 0; i < n; ++i) nfluid += (s->kind[i] == FLUID);
  int32_t k = 0;
  double res = 0.0;
  int conv = 0, bad = 0;
  while (1) {
    or_wall_pressure(s);
    for (int64_t i = 0; i < n; ++i) {
      if (s->kind[i] != FLUID) { s->pnew[i] = s->p[i]; continue; }
      if (!s->active[i]) { s->pnew[i] = 0.0; continue; }
      double acc = s->rhs[i];
      for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
        int64_t j = s->nidx[t];
        acc += s->fac[t] * s->p[j];
      }
      s->pnew[i] = P->omega * acc / s->diag[i] + (1.0 - P->omega) * s->p[i];
    }
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (s->kind[i] != FLUID) continue;
      num += fabs(s->pnew[i] - s->p[i]);
      den += fabs(s->pnew[i]);
    }
    for (int64_t i = 0; i < n; ++i)
      if (s->kind[i] == FLUID) s->p[i] = s->pnew[i];
    ++k;
    double lam = (P->residual_form == 1) ? (double)nfluid * s->lambda : s->lambda;
    double dd = (lam > den) ? lam : den;
    res = (dd > 0.0) ? num / dd : num;
    if (!isfinite(res)) { bad = 1; break; }
    if (k >= P->min_iter && res < P->tol) { conv = 1; break; }
    if (k >= P->max_iter) break;
  }
  or_wall_pressure(s);
  if (d) {
    d->iters = k; d->residual = res; d->lambda = s->lambda;
    d->converged = conv; d->nonfinite = bad;
  }
}

/* out_i = D_ii p_i + sum_j OD_ij p_j for fluid i (the discrete operator of
 * Eq. sph-ppe applied to p); zero elsewhere. */
void or_ppe_apply(const or_sim *s, const double *p, double *out) {
  for (int64_t i = 0; i < s->n; ++i) {
    out[i] = 0.0;
    if (s->kind[i] != FLUID) continue;
    double acc = s->diag[i] * p[i];
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) acc -= s->fac[t] * p[s->nidx[t]];
    out[i] = acc;
  }
}

/* ---------------------------------------------------------------------------
 * BiCGStab (van der Vorst 1992) for the PPE, the Krylov alternative the
 * paper mentions beside its Jacobi iterations (Sec. 3.1).  Reading: it
 * solves the linear system the Jacobi iteration converges to,
 *   D_ii p_i - sum_j fac_ij p_j = RHS_i   (active fluid i),  p_i = 0 (inactive),
 * with each wall pressure replaced by its extrapolation (Eq. p-shepard)
 *   p_w = (sum_f W_wf p_f + H_w) / S_w,
 * whose affine part H_w / S_w moves to the right-hand side; the free-surface
 * clamp p_w >= 0 is not linear and is applied only in the final wall update,
 * as after the Jacobi sweeps.  Stopping rule: the Jacobi test of Eq.
 * convergence on the update of each iteration,
 *   sum_i |x^{k+1}_i - x^k_i| / max(Lambda, sum_i |x^{k+1}_i|) < tol
 * (at least min_iter, at most max_iter iterations), so that both solvers stop
 * at the same epsilon.  Dot products run over the fluid particles.
 * Without a free-surface (Dirichlet) row -- periodic or enclosed flows -- the
 * system is singular (constant pressures are in its null space) and, with a
 * right-hand side that is consistent only up to rounding and the slight
 * asymmetry of fac_ij, a Krylov solve diverges; such a case is solved by the
 * Jacobi iteration instead (reading).
 * ------------------------------------------------------------------------- */
static void or_wall_linear(const or_sim *s, double *x, int with_h) {
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->kind[i] != WALL) continue;
    double acc = 0.0;
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (s->kind[j] != FLUID) continue;
      acc += x[j] * s->fac[t];
    }
    if (with_h) acc += s->wh[i];
    x[i] = (s->ws[i] > 0.0) ? acc / s->ws[i] : 0.0;
  }
}

/* y = A x over fluid rows (walls of x overwritten by their linear part). */
static void or_apply_linear(const or_sim *s, double *x, double *y) {
  or_wall_linear(s, x, 0);
  for (int64_t i = 0; i < s->n; ++i) {
    y[i] = 0.0;
    if (s->kind[i] != FLUID) continue;
    if (!s->active[i]) { y[i] = x[i]; continue; }
    double acc = s->diag[i] * x[i];
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) acc -= s->fac[t] * x[s->nidx[t]];
    y[i] = acc;
  }
}

static double or_fdot(const or_sim *s, const double *a, const double *b) {
  double acc = 0.0;
  for (int64_t i = 0; i < s->n; ++i)
    if (s->kind[i] == FLUID) acc += a[i] * b[i];
  return acc;
}

void or_ppe_bicgstab(or_sim *s, or_diag *d) {
  const or_params *P = &s->prm;
  const int64_t n = s->n;
  int64_t dirichlet = 0;
  for (int64_t i = 0; i < n; ++i) dirichlet += (s->kind[i] == FLUID && !s->active[i]);
  if (dirichlet == 0) {
    or_ppe_iterate(s, d);
    return;
  }
  double *x = or_alloc(n), *b = or_alloc(n), *r = or_alloc(n), *rh = or_alloc(n);
  double *pv = or_alloc(n), *v = or_alloc(n), *sv = or_alloc(n), *tv = or_alloc(n);
  int64_t nfluid = 0;
  for (int64_t i = 0; i < n; ++i) nfluid += (s->kind[i] == FLUID);
  // right-hand side: RHS plus the affine part of the wall extrapolation
  double *w0 = or_alloc(n);
  or_wall_linear(s, w0, 1);
  for (int64_t i = 0; i < n; ++i) {
    if (s->kind[i] != FLUID || !s->active[i]) continue;
    double acc = s->rhs[i];
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (s->kind[j] == WALL) acc += s->fac[t] * w0[j];
    }
    b[i] = acc;
  }
  for (int64_t i = 0; i < n; ++i) x[i] = (s->kind[i] == FLUID && s->active[i]) ? s->p[i] : 0.0;
  or_apply_linear(s, x, r);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = (s->kind[i] == FLUID) ? b[i] - r[i] : 0.0;
    rh[i] = r[i];
  }
  double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  int32_t k = 0;
  double res = 0.0;
  int conv = 0, bad = 0;
  while (1) {
    // breakdown guards: r = 0 means x solves the system; (r^, r) = 0 or
    // (r^, v) = 0 otherwise stops the iteration (not converged)
    const double rho = or_fdot(s, rh, r);
    if (rho == 0.0) {
      if (or_fdot(s, r, r) == 0.0) { conv = 1; res = 0.0; }
      break;
    }
    const double beta = (rho / rho_prev) * (alpha / omega);
    for (int64_t i = 0; i < n; ++i)
      if (s->kind[i] == FLUID) pv[i] = r[i] + beta * (pv[i] - omega * v[i]);
    or_apply_linear(s, pv, v);
    const double rv = or_fdot(s, rh, v);
    if (rv == 0.0) break;
    alpha = rho / rv;
    for (int64_t i = 0; i < n; ++i)
      if (s->kind[i] == FLUID) sv[i] = r[i] - alpha * v[i];
    or_apply_linear(s, sv, tv);
    const double tt = or_fdot(s, tv, tv);
    omega = tt > 0.0 ? or_fdot(s, tv, sv) / tt : 0.0;
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (s->kind[i] != FLUID) continue;
      const double dx = alpha * pv[i] + omega * sv[i];
      x[i] += dx;
      r[i] = sv[i] - omega * tv[i];
      num += fabs(dx);
      den += fabs(x[i]);
    }
    rho_prev = rho;
    ++k;
    const double lam = (P->residual_form == 1) ? (double)nfluid * s->lambda : s->lambda;
    const double dd = (lam > den) ? lam : den;
    res = (dd > 0.0) ? num / dd : num;
    if (!isfinite(res)) { bad = 1; break; }
    if (k >= P->min_iter && res < P->tol) { conv = 1; break; }
    if (k >= P->max_iter) break;
  }
  for (int64_t i = 0; i < n; ++i)
    if (s->kind[i] == FLUID) s->p[i] = x[i];
  or_wall_pressure(s);
  if (d) {
    d->iters = k; d->residual = res; d->lambda = s->lambda;
    d->converged = conv; d->nonfinite = bad;
  }
  free(x); free(b); free(r); free(rh); free(pv); free(v); free(sv); free(tv); free(w0);
}

int64_t or_ppe_export(const or_sim *s, double *diag, double *rhs, int32_t *active,
                      double *fac, double *wall_s, double *wall_h, double *wall_w) {
  int64_t tot = s->nstart[s->n];
  for (int64_t i = 0; i < s->n; ++i) {
    diag[i] = s->diag[i]; rhs[i] = s->rhs[i]; active[i] = s->active[i];
    wall_s[i] = s->ws[i]; wall_h[i] = s->wh[i];
  }
  for (int64_t t = 0; t < tot; ++t) {
    fac[t] = s->fac[t];
    wall_w[t] = s->fac[t];
  }
  return tot;
}

/* ---------------------------------------------------------------------------
 * Pressure gradient and velocity correction (Eqs. mom:sph:press:symm,
 * mom:sph:press:pij, int:vnp1):
 *   symm : f_p = -sum_j m_j (p_i/rho_i^2 + p_j/rho_j^2) grad W_ij
 *   asymm: f_p = -sum_j m_j/(rho_i rho_j) (p_j - p_i) grad W_ij
 *   u^{n+1} = u* + dt f_p
 * ------------------------------------------------------------------------- */
void or_pressure_gradient(or_sim *s) {
  const or_params *P = &s->prm;
  s->fmax = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->kind[i] != FLUID) continue;
    double fi[3] = {0, 0, 0};
    double ri = s->rho[i], pi = s->p[i];
    for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
      int64_t j = s->nidx[t];
      if (j == i) continue;
      double dx[3], g[3];
      or_grad(s, i, j, P->h, dx, g, NULL);
      double rj = s->rho[j], pj = s->p[j], mj = s->m[j];
      double c;
      if (P->pgrad_symm) c = -mj * (pi / (ri * ri) + pj / (rj * rj));
      else c = -mj / (ri * rj) * (pj - pi);
      for (int k = 0; k < 3; ++k) fi[k] += c * g[k];
    }
    // total acceleration of this step, f_p + (f_visc + f_avisc + f_astress
    // + f_body) from stage 1 (still in f), for the adaptive time step
    double ft[3] = {0, 0, 0};
    for (int k = 0; k < P->dim; ++k) ft[k] = s->f[k][i] + fi[k];
    double fm = sqrt(or_dot(ft, ft));
    if (fm > s->fmax) s->fmax = fm;
    for (int k = 0; k < P->dim; ++k) {
      s->f[k][i] = fi[k];
      s->u[k][i] = s->u[k][i] + P->dt * fi[k];
    }
  }
}

/* ---------------------------------------------------------------------------
 * GTVF homogenisation, Eqs. mom:sph:gtvf, int:gtvf:pos, int:gtvf:vel:tmp:
 *   f_i = -p0_i sum_j (m_j / rho_j^2) grad W(r_ij, h~)
 *   r^k = r^{k-1} + dtau u~^{k-1} + dtau^2/2 f(r^{k-1}),
 *   u~^k = u~^{k-1} + dtau f(r^{k-1}),  dtau = dt/K,  r^0 = r*, u~^0 = 0,
 * on the neighbour lists of r* with distances from the sub-step positions.
 * p0_i = p_ref (internal) or min(10 |p_i|, p_ref) (external).
 * Positions are tracked as the displacement d^k = r^k - r^0.
 * ------------------------------------------------------------------------- */
void or_gtvf(or_sim *s) {
  const or_params *P = &s->prm;
  int64_t n = s->n;
  int K = P->gtvf_K > 0 ? P->gtvf_K : 1;
  double dtau = P->dt / K;
  double hg = P->gtvf_hfac * P->h;
  double *fg[3];
  for (int k = 0; k < 3; ++k) {
    fg[k] = or_alloc(n);
    for (int64_t i = 0; i < n; ++i) { s->d[k][i] = 0.0; s->vg[k][i] = 0.0; }
  }
  for (int sub = 0; sub < K; ++sub) {
    for (int64_t i = 0; i < n; ++i) {
      if (s->kind[i] != FLUID) continue;
      double p0 = (P->pref_mode == 2) ? fmin(10.0 * fabs(s->p[i]), s->p_ref) : s->p_ref;
      double acc[3] = {0, 0, 0};
      for (int64_t t = s->nstart[i]; t < s->nstart[i + 1]; ++t) {
        int64_t j = s->nidx[t];
        if (j == i) continue;
        double dx[3];
        or_pair(P, (const double *const *)s->x, i, j, dx);
        for (int k = 0; k < P->dim; ++k) dx[k] += s->d[k][i] - s->d[k][j];
        double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        double r = sqrt(r2);
        if (r <= 0.0) continue;
        double fr = or_kernel_dwdr(r, hg, P->dim) / r;
        double c = s->m[j] / (s->rho[j] * s->rho[j]);
        for (int k = 0; k < 3; ++k) acc[k] += c * fr * dx[k];
      }
      for (int k = 0; k < 3; ++k) fg[k][i] = -p0 * acc[k];
      if (sub == 0)
        for (int k = 0; k < 3; ++k) s->f[k][i] = fg[k][i];
    }
    for (int64_t i = 0; i < n; ++i) {
      if (s->kind[i] != FLUID) continue;
      for (int k = 0; k < P->dim; ++k) {
        s->d[k][i] = s->d[k][i] + dtau * s->vg[k][i] + 0.5 * dtau * dtau * fg[k][i];
        s->vg[k][i] = s->vg[k][i] + dtau * fg[k][i];
      }
    }
  }
  for (int k = 0; k < 3; ++k) free(fg[k]);
}

/* ---------------------------------------------------------------------------
 * Transport velocity and position update, Eqs. int:vhatnp2, int:rnp2:
 *   u~^{n+1} = u^{n+1} + (r^K - r^0)/dt
 *   r^{n+1}  = r^n + dt (u~^{n+1} + u~^n)/2
 * ------------------------------------------------------------------------- */
void or_update(or_sim *s) {
  const or_params *P = &s->prm;
  double umax = 0.0;
  for (int64_t i = 0; i < s->n; ++i) {
    if (s->kind[i] != FLUID) continue;
    double u2 = 0.0;
    for (int k = 0; k < P->dim; ++k) {
      double old = s->ut[k][i];
      double nw = s->u[k][i] + s->d[k][i] / P->dt;
      double xk = s->xn[k][i] + 0.5 * P->dt * (nw + old);
      or_wrap(P, &xk, k);
      s->x[k][i] = xk;
      s->ut[k][i] = nw;
      u2 += s->u[k][i] * s->u[k][i];
    }
    if (sqrt(u2) > umax) umax = sqrt(u2);
  }
  s->last.umax = umax;
}

int32_t or_ppe_solve(or_sim *s, double tol, int32_t max_iter, or_diag *d) {
  double t0 = s->prm.tol;
  int32_t m0 = s->prm.max_iter;
  s->prm.tol = tol;
  s->prm.max_iter = max_iter;
  or_ghost_velocity(s, s->prm.ustar_slip);
  or_ppe_setup(s);
  if (s->prm.ppe_solver == 1) or_ppe_bicgstab(s, d);
  else or_ppe_iterate(s, d);
  s->prm.tol = t0;
  s->prm.max_iter = m0;
  return d->nonfinite ? -5 : (d->converged ? 0 : -4);
}

/* ---------------------------------------------------------------------------
 * Adaptive time step (Sec. 3.2): from the maximum fluid speed max|u^n| at
 * the start of step n and the maximum total acceleration max|f^n| of that
 * step (pressure gradient + viscous + body + artificial viscosity and
 * stress),
 *   dt^{n+1} = min(0.25 h / max|u^n|, 0.25 sqrt(h / max|f^n|), 0.25 h^2 / nu),
 * with h_ij = h.  Reading: the viscous limit of the fixed rule stays in the
 * minimum (the text notes it is constant, not that it is dropped).  A limit
 * whose denominator is zero is left out; if all are, dt is kept.
 * ------------------------------------------------------------------------- */
static double or_next_dt(const or_params *P, double umax, double fmax) {
  double dt = INFINITY;
  if (umax > 0.0) dt = fmin(dt, 0.25 * P->h / umax);
  if (fmax > 0.0) dt = fmin(dt, 0.25 * sqrt(P->h / fmax));
  if (P->nu > 0.0) dt = fmin(dt, 0.25 * P->h * P->h / P->nu);
  return isfinite(dt) ? dt : P->dt;
}

/* One time step of Algorithm 1 (two neighbour builds: at r^n for stage 1 and
 * at r* for stage 2, as in the two stages of Listing 1). */
int32_t or_step(or_sim *s, int32_t nsteps, or_diag *d) {
  int32_t rc = 0;
  for (int32_t it = 0; it < nsteps; ++it) {
    double umax = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
      if (s->kind[i] != FLUID) continue;
      double ui[3] = {s->u[0][i], s->u[1][i], s->u[2][i]};
      double um = sqrt(or_dot(ui, ui));
      if (um > umax) umax = um;
    }
    const double dt_used = s->prm.dt;
    if (or_build_neighbors(s) < 0) return -2;
    or_density(s);
    or_ghost_velocity(s, 0);
    or_stage1(s);
    if (or_build_neighbors(s) < 0) return -2;
    or_ghost_velocity(s, s->prm.ustar_slip);
    or_ppe_setup(s);
    or_diag dd;
    memset(&dd, 0, sizeof(dd));
    if (s->prm.ppe_solver == 1) or_ppe_bicgstab(s, &dd);
    else or_ppe_iterate(s, &dd);
    if (!s->pref_set) {
      double mx = 0.0;
      int first = 1;
      for (int64_t i = 0; i < s->n; ++i)
        if (s->kind[i] == FLUID && (first || s->p[i] > mx)) { mx = s->p[i]; first = 0; }
      s->p_ref = 2.0 * mx;
      s->pref_set = 1;
    }
    or_pressure_gradient(s);
    or_gtvf(s);
    or_update(s);
    dd.umax = s->last.umax;
    dd.dt = dt_used;
    s->last = dd;
    if (d) d[it] = dd;
    if (s->prm.adaptive_dt) s->prm.dt = or_next_dt(&s->prm, umax, s->fmax);
    if (dd.nonfinite) return -5;
    if (!dd.converged) rc = -4;
  }
  return rc;
}
