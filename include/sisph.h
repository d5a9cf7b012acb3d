/*
 * libsisph: GB300 (sm_103a) implementation of the hot path of the Simple
 * Iterative ISPH scheme (SISPH) of Muta, Ramachandran & Negi, "An efficient,
 * open source, iterative ISPH scheme", arXiv 1908.01762.
 *
 * One time step is Algorithm 1 of the paper: cell-list neighbour search,
 * summation density (Eq. summation_density), wall ghost velocities (Sec. 3.4),
 * predicted position and velocity (Eqs. int:rnp1, int:vint), a second
 * neighbour search at r*, the pressure-Poisson set-up (Eqs. sph-ppe, coeff,
 * coeff1), damped-Jacobi sweeps with Shepard wall pressure (Eqs. p-sor,
 * p-shepard) to the relative tolerance of Eq. convergence, the pressure
 * gradient and velocity correction (Eqs. mom:sph:press:*, int:vnp1), the GTVF
 * homogenisation (Eqs. mom:sph:gtvf, int:gtvf:*) and the transport-velocity
 * position update (Eqs. int:vhatnp2, int:rnp2).
 *
 * Conventions
 *  - Every pointer argument is a HOST pointer unless the name ends in _dev.
 *  - Particle arrays given to and returned by the library are in the caller's
 *    order (case after case for a batch), FP64, one entry per particle.
 *  - The library copies its inputs at creation and owns all device memory;
 *    nothing the caller passes is retained after a call returns.
 *  - All calls return 0 (SISPH_OK) or a negative SISPH_E* code; the message of
 *    the last failure is available from sisph_last_error().  The library never
 *    aborts the process and never traps the device: device-side failures
 *    (barrier timeout, non-finite residual, neighbour-capacity overflow) are
 *    recorded in device status words and returned as codes.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Kernels run on the handle's stream (default: a stream the library creates;
 *    see sisph_set_stream).  Calls synchronise that stream before returning
 *    results to the host.
 */
#ifndef SISPH_H
#define SISPH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SISPH_OK 0
#define SISPH_EINVAL (-1)        /* bad argument, size or handle */
#define SISPH_ENOMEM (-2)        /* device or host allocation failed */
#define SISPH_ECUDA (-3)         /* a CUDA runtime call failed */
#define SISPH_ENOTCONVERGED (-4) /* PPE hit max_iter in some case; results are valid */
#define SISPH_ENONFINITE (-5)    /* NaN/Inf in the PPE residual; state is suspect */
#define SISPH_ETIMEOUT (-6)      /* persistent-kernel grid barrier exceeded its budget */
#define SISPH_EINTERNAL (-7)     /* internal consistency check failed */
#define SISPH_ECAPACITY (-8)     /* a particle has more neighbours than the capacity */

#define SISPH_KIND_FLUID 0
#define SISPH_KIND_WALL 1

#define SISPH_FP64 0   /* every neighbour sum, sweep and update in FP64 */
#define SISPH_MIXED 1  /* FP32 neighbour sums (Kahan-compensated PPE diagonal and
                          source) and FP32 sweeps; FP64 residual reduction and
                          FP64 position/velocity integration */

/* Background-pressure modes (Sec. 2.1, text after Eq. mom:sph:gtvf). */
#define SISPH_PREF_FIXED 0          /* p0_i = p_ref */
#define SISPH_PREF_TWICE_MAX_FIRST 1/* p_ref = 2 max_i p_i after the first PPE solve */
#define SISPH_PREF_EXTERNAL 2       /* p0_i = min(10 |p_i|, p_ref) */

typedef struct sisph_s *sisph_t;

/* One particle set (one case).  Arrays have n entries in the caller's order.
 * z, w, wall_w may be NULL when dim == 2; rho may be NULL (rho0 is used);
 * p may be NULL (zero); kind may be NULL (all fluid); wall_* may be NULL
 * (walls at rest).  lo/hi bound the domain: periodic directions wrap at
 * them, other directions only use them to lay out the cell grid (particles
 * outside are still handled exactly). */
typedef struct {
  int32_t dim;                  /* 2 or 3 */
  int64_t n;
  const double *x, *y, *z;
  const double *u, *v, *w;
  const double *m, *rho, *p;
  const int32_t *kind;          /* SISPH_KIND_FLUID or SISPH_KIND_WALL */
  const double *wall_u, *wall_v, *wall_w; /* prescribed wall velocity */
  double lo[3], hi[3];
  int32_t periodic[3];
} sisph_particles;

/* Per-case physics (all FP64).  Defaults from sisph_default_case(). */
typedef struct {
  double h, dt, rho0, nu;
  double g[3];
  double alpha, c0;             /* artificial viscosity; alpha = 0 disables it */
  double tol;                   /* PPE relative tolerance epsilon (Eq. convergence) */
  int32_t max_iter;             /* PPE iteration cap (1000 in Listing 1) */
  int32_t pgrad_symm;           /* 1 "symm", 0 "asymm" pressure gradient */
  int32_t free_surface;         /* rho/rho0 < fs_ratio -> p = 0; wall clamp p_w >= 0 */
  int32_t ustar_slip;           /* 1: slip ghost u* in the PPE source (Sec. 3.4) */
  int32_t pref_mode;            /* SISPH_PREF_* */
  double p_ref;
  double gtvf_hfac;             /* h~ = gtvf_hfac * h (1 internal, 0.5 external flows) */
  int32_t gtvf_K;               /* GTVF sub-steps per time step */
  int32_t adaptive_dt;          /* 1: the next step's dt from max|u^n| and max|f^n|
                                   (Sec. 3.2): min(0.25 h/max|u|, 0.25 sqrt(h/max|f|),
                                   0.25 h^2/nu); dt is then the first step's */
  int32_t ppe_solver;           /* 0 damped Jacobi (Eq. p-sor, the paper's method);
                                   1 BiCGStab (van der Vorst) on the same stored
                                   coefficients and stopping test, used when the
                                   case has a free-surface row (else its system is
                                   singular and the Jacobi sweeps run) */
} sisph_case_params;

/* Solver-wide options.  Defaults from sisph_default_options(). */
typedef struct {
  int32_t precision;            /* SISPH_FP64 or SISPH_MIXED */
  double omega;                 /* 0.5 (Eq. p-sor) */
  int32_t min_iter;             /* 2 */
  double eta;                   /* 0.01 */
  double fs_ratio;              /* 0.8 */
  int32_t residual_form;        /* 0: max(Lambda, sum|p|); 1: max(N_F Lambda, sum|p|) */
  int32_t nbr_capacity;         /* neighbours per particle; 0 = from dim and h */
  double skin;                  /* Verlet skin s as a fraction of 3h (0.15): the
                                   lists are rebuilt from a cell sort only when a
                                   fluid particle of the case moved more than s/2
                                   since the last rebuild, and filtered exactly to
                                   N(i) at every refresh; 0 rebuilds every time */
  int32_t block;                /* threads per block / tile size (64..256, mult. of 32;
                                   256 by default, autotune.py may pick 128) */
  int32_t use_graph;            /* capture sisph_step in a CUDA graph and replay it */
  double barrier_timeout_ms;    /* budget of one grid-barrier wait */
  int32_t debug_skip_barrier;   /* test hook: block 1 skips its first barrier arrival */
  int32_t ppe_sync;             /* how sweeps synchronise: 0 auto (default: per-tile
                                   flags when each block owns at most one fluid and
                                   one wall tile, else a grid barrier), 1 grid
                                   barrier after every phase, 2 per-tile flags */
  sisph_case_params physics;    /* case defaults used by sisph_create */
} sisph_options;

/* Per-case status of the last PPE solve. */
typedef struct {
  int32_t iters;                /* sweeps performed in the last solve */
  int32_t status;               /* SISPH_OK / SISPH_ENOTCONVERGED / SISPH_ENONFINITE */
  double residual;              /* final value of Eq. convergence */
  double lambda;                /* max_i |RHS_i / D_ii| (Eq. convergence) */
  double p_ref;                 /* background pressure in use */
  int64_t total_iters;          /* sweeps summed over every solve so far */
  int64_t solves;               /* PPE solves so far */
  int64_t rebuilds;             /* cell sorts + skin-list rebuilds so far */
  double dt;                    /* time step of the next step */
  double time;                  /* simulated time so far */
} sisph_case_stats;

/* Field identifiers for sisph_get / sisph_set. */
#define SISPH_F_X 0
#define SISPH_F_Y 1
#define SISPH_F_Z 2
#define SISPH_F_U 3      /* fluid: velocity; wall: last ghost velocity */
#define SISPH_F_V 4
#define SISPH_F_W 5
#define SISPH_F_UT 6     /* transport velocity u~ */
#define SISPH_F_VT 7
#define SISPH_F_WT 8
#define SISPH_F_P 9
#define SISPH_F_RHO 10
#define SISPH_F_M 11
#define SISPH_F_NX 12    /* wall unit normals (zero for fluid) */
#define SISPH_F_NY 13
#define SISPH_F_NZ 14
#define SISPH_F_RHS 15   /* PPE source RHS_i of the last set-up (fluid) */
#define SISPH_F_DIAG 16  /* PPE diagonal D_ii of the last set-up (fluid) */
#define SISPH_F_DX 17    /* GTVF displacement r^K - r^0 of the last step */
#define SISPH_F_DY 18
#define SISPH_F_DZ 19
#define SISPH_F_NSKIN 20 /* length of the particle's skin list (read-only) */
#define SISPH_F_NCOUNT 21 /* length of its neighbour list as the last refresh left it
                             (inside a step without the rim pairs; read-only) */
#define SISPH_F_COUNT 22

/* Fill defaults: FP64, omega 0.5, min_iter 2, eta 0.01, fs_ratio 0.8, ... */
void sisph_default_options(sisph_options *opt);
void sisph_default_case(sisph_case_params *prm);

/* Create a single simulation (Algorithm 1 on one particle set); the signature
 * follows the paper's statement of the problem: particles with m, rho, p, u,
 * r (Sec. 3.3), smoothing length h, time step dt, rest density rho0,
 * kinematic viscosity nu and gravity g (Sec. 2, Sec. 3.2).  opt may be NULL
 * (defaults); other case physics come from opt->physics.  Copies every input
 * to the device, sorts the particles into cells, builds the first neighbour
 * lists and the wall normals (Sec. 3.4.1).  *out receives the handle. */
int sisph_create(const sisph_particles *particles, double h, double dt, double rho0, double nu,
                 const double g[3], const sisph_options *opt, sisph_t *out);

/* Create a batch of ncases independent simulations advanced together (one
 * persistent PPE launch for all of them; each case converges on its own). */
int sisph_batch_create(int32_t ncases, const sisph_particles *particles,
                       const sisph_case_params *params, const sisph_options *opt, sisph_t *out);

void sisph_destroy(sisph_t s);

/* Bring the neighbour lists to the current positions: N(i) = {j : |r_ij|^2 <
 * (3h)^2}, minimum image, exactly.  A case whose fluid moved more than s/2
 * since its last rebuild (every case, after sisph_set moved a wall) is first
 * sorted into Morton-ordered cells and gets new skin lists; then every list is
 * filtered from its skin list.  sisph_step does this twice per step, leaving
 * out the pairs within a relative 4e-5 of the cutoff (|r_ij| > 3h(1 - 3e-5),
 * where the kernel's weight and gradient are below FP64 rounding of every
 * sum); call it after sisph_set of a position before using the lists outside
 * a step. */
int sisph_build_neighbors(sisph_t s);

/* Neighbour lists N(i) at the current positions, exactly (the lists are
 * first brought there as by sisph_build_neighbors), in the caller's order:
 * counts[n] and, if idx is not NULL, the lists concatenated with caller
 * indices in ascending order (capacity idx_cap entries).  *total receives the
 * number of pairs. */
int sisph_neighbors(sisph_t s, int32_t *counts, int32_t *idx, int64_t idx_cap, int64_t *total);

/* Summation density (Eq. summation_density) at the current neighbour lists. */
int sisph_compute_density(sisph_t s);

/* Solve the PPE once on the current state, treating the current velocity as
 * u*: slip ghost velocity, set-up, damped-Jacobi sweeps to tol (at least
 * min_iter, at most max_iter), final wall extrapolation.  iters/residual
 * receive one value per case (may be NULL).  Returns SISPH_ENOTCONVERGED if
 * any case hit max_iter. */
int sisph_ppe_solve(sisph_t s, double tol, int32_t max_iter, int32_t *iters, double *residual);

/* Advance nsteps time steps of Algorithm 1 (replayed from a CUDA graph when
 * opt.use_graph is set).  Returns SISPH_ENOTCONVERGED if a PPE solve hit
 * max_iter in any of the steps (the state is still advanced and valid). */
int sisph_step(sisph_t s, int32_t nsteps);

/* sisph_step on a batch handle (Algorithm 1 for every case at once), with
 * iters_per_case[c] (ncases entries; may be NULL) set to the PPE sweeps case c
 * took over these nsteps steps.  Same return codes as sisph_step. */
int sisph_batch_step(sisph_t s, int32_t nsteps, int32_t *iters_per_case);

/* Read or write a field (SISPH_F_*) for all particles in the caller's order.
 * Writing a position needs no rebuild unless it moves a wall: the next
 * refresh re-sorts the cases whose fluid moved more than s/2. */
int sisph_get(sisph_t s, int32_t field, double *out);
int sisph_set(sisph_t s, int32_t field, const double *in);

/* Several fields in one call: fields[k] from in[k] / into out[k] (host
 * arrays of n doubles each, caller's order), the same as nfields calls of
 * sisph_set / sisph_get, but each field has a device staging column of its
 * own and its host copy runs on a copy stream of the handle, overlapping the
 * reordering of the neighbouring field on the handle's stream; the FP32
 * mirrors are refreshed once after all writes, and the call returns when
 * every copy is done.  The staging (nfields x n doubles) is allocated at
 * the first call that needs it and kept until sisph_destroy.  Host arrays
 * in page-locked memory copy asynchronously.  Every field is checked before
 * anything is copied: an unknown or read-only field (or a third component
 * in 2D) returns SISPH_EINVAL with nothing written.  A step's whole state
 * (positions, velocities, transport velocities, pressure) moves in and out
 * this way. */
int sisph_set_many(sisph_t s, int32_t nfields, const int32_t *fields, const double *const *in);
int sisph_get_many(sisph_t s, int32_t nfields, const int32_t *fields, double *const *out);

/* Per-case statistics of the last PPE solve (stats has ncases entries). */
int sisph_stats(sisph_t s, sisph_case_stats *stats);

/* Sizes: total particles, fluid particles, cases, neighbour capacity. */
int sisph_info(sisph_t s, int64_t *n, int64_t *n_fluid, int32_t *ncases, int32_t *nbr_capacity);

/* Run the library's kernels on a caller stream (a cudaStream_t, e.g. from
 * torch.cuda.current_stream().cuda_stream).  NULL restores the library's own
 * stream.  Drops any captured graph. */
int sisph_set_stream(sisph_t s, void *cuda_stream);

/* Kernel timing with CUDA events on the handle's stream.  on = 0 stops it.
 * With only == NULL every kernel launch is bracketed by events and CUDA
 * graphs are not used (a diagnostic mode).  With only naming one site or a
 * comma-separated list ("ppe_sweeps", "filter,stage1", ...; the sites are
 * check, sort, build, sync, filter, density, ghost, stage1, stage1_walls,
 * ppe_setup, ppe_setup_wall, ppe_sweeps, pref, pgrad_gtvf, pgrad, gtvf,
 * update, speed_max, adapt_dt) only their launches are bracketed, and graph replay stays on: the
 * events are recorded as event nodes of the captured step, so the kernels
 * are timed inside the normal graph-replayed step (the library then waits
 * for each replayed step to read them).  Timing "sort" or "build" takes the
 * neighbour rebuild group out of its conditional graph node (its kernels
 * then run every refresh and return at once when no case needs a rebuild).
 * sisph_profile_get returns, for one site, the launch count, the summed
 * device time in ms and the summed work units (particles). */
int sisph_profile_enable(sisph_t s, int32_t on, const char *only);
int sisph_profile_get(sisph_t s, const char *kernel, int64_t *launches, double *total_ms,
                      double *units);
/* Number of kernels this handle has launched (graph replays count their nodes). */
int64_t sisph_launch_count(sisph_t s);

/* Checkpoint the full state (caller order, FP64) to a file and restore it;
 * a restored handle continues bit-identically to the one that was saved. */
int sisph_save(sisph_t s, const char *path);
int sisph_load(sisph_t s, const char *path);

/* Message of the last failure on this handle (or of the last failed create
 * when s is NULL).  The string is owned by the library. */
const char *sisph_last_error(sisph_t s);
const char *sisph_version(void);

/* Neighbour search that allocates no memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- an
 * application whose device memory is already fully reserved by its own
 * allocator, or a latency-critical loop that must not pay for cudaMalloc and
 * cudaFree, which can synchronise the device.
 *
 * Same search as sisph_build_neighbors (N(i) = {j : |r_ij|^2 < (3h)^2},
 * minimum image in periodic directions, |r_ij|^2 = dx*dx + dy*dy (+ dz*dz)
 * unfused, i itself included) for n points given in DEVICE memory
 * (x_dev, y_dev, z_dev; z_dev may be NULL when dim == 2; positions must lie in
 * [lo, hi) in periodic directions).  Output, also in DEVICE memory the caller
 * allocated: counts_dev[n] and idx_dev[n * cap], row i at idx_dev + i * cap
 * holding the indices of N(i) in ascending order.  Kernels run on `stream`
 * (a cudaStream_t; NULL = the default stream) and the call waits for them.
 *
 * All scratch memory (cell histogram, cell ids, slots, the sort permutation,
 * a status word; about 1 MiB) is one fixed device array reserved when the
 * library is loaded; every GPU that loads the library holds it until the
 * process exits.  Limits: n <= SISPH_NOALLOC_MAX_POINTS points and a cell
 * grid (cells of side >= 3h over [lo, hi)) of at most SISPH_NOALLOC_MAX_CELLS
 * cells; larger inputs are rejected with SISPH_EINVAL and a message.  Points
 * outside [lo, hi) in a non-periodic direction are searched from the edge
 * cell they are clamped into, so their rows are still exact.  A row with more
 * than cap neighbours makes the call return SISPH_ECAPACITY; its count is
 * clipped to cap and the row holds the cap smallest indices of N(i), in
 * ascending order.  Each call looks up the device address of the scratch
 * array on the current device (no allocation).  The call reads a status word
 * back and waits for its kernels, so a `stream` that is capturing a graph is
 * rejected with SISPH_EINVAL before anything is launched.  Every call shares
 * the array and it keeps the last call's contents (each call clears what
 * must start at zero); calls whose kernels overlap on the GPU race on it, so
 * serialise them.  The library calls no cudaMalloc, cudaFree or allocating
 * routine here.  Errors are reported through sisph_last_error(NULL). */
#define SISPH_NOALLOC_MAX_POINTS 65536
#define SISPH_NOALLOC_MAX_CELLS 65536
int sisph_neighbors_noalloc(int32_t dim, int32_t n, const double *x_dev, const double *y_dev,
                            const double *z_dev, double h, const double lo[3], const double hi[3],
                            const int32_t periodic[3], int32_t cap, int32_t *counts_dev,
                            int32_t *idx_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif
