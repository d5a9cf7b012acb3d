// Internal types and device helpers of libsisph (not part of the C-ABI).
//
// Layout.  Particles live on the device in one sorted order: case after case,
// and inside a case its fluid block followed by its wall block:
//   [case0 fluid | case0 wall | case1 fluid | case1 wall | ...]
// Inside each block particles are sorted by (Morton cell, original index), so
// the block boundaries never move and the order is deterministic.  Work is cut
// into tiles of `T` consecutive particles that never straddle a block, so one
// thread block handles one tile and every tile has a single case and kind.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/sisph.h"

namespace sisph {

constexpr int kCodeShift = 26;                   // neighbour entry = j | code << 26
constexpr unsigned kIdxMask = (1u << kCodeShift) - 1u;
constexpr int kMaxParticles = (1 << kCodeShift) - 1;

// Neighbour lists, skin lists and PPE slots are stored in blocks of 32
// consecutive particles, one warp's rows: entry q of particle i at
// ((i / 32) cap + q) 32 + i % 32.  The entries of a warp's rows follow each
// other, so a warp streams one contiguous run (cap entries of 128 or 256
// bytes) and fills whole DRAM pages instead of one piece per page.
constexpr int kEllBlock = 32;    // particles per block (a power of two)
__host__ __device__ __forceinline__ long long ell_base(int cap, long long i) {
  return (i / kEllBlock) * cap * kEllBlock + (i % kEllBlock);
}
__host__ __device__ __forceinline__ long long ell_at(int cap, int q, long long i) {
  return ell_base(cap, i) + (long long)q * kEllBlock;
}
// elements of a blocked list array of n particles
inline size_t ell_size(int cap, long long n) {
  return size_t((n + kEllBlock - 1) / kEllBlock) * kEllBlock * size_t(cap);
}
constexpr int kMaxCellsPerAxis = (1 << 21) - 1;     // packed rebuild cell: 21 bits per axis
constexpr int kDepCap = 96;                         // dependency list of a tile

// Error bits of the device status word.
constexpr int kErrCapacity = 1;   // a neighbour row overflowed its capacity
constexpr int kErrTimeout = 2;    // a grid-barrier wait ran out of budget
constexpr int kErrNonFinite = 4;  // a PPE residual was NaN / Inf
constexpr int kErrNotConv = 8;    // a PPE solve stopped at max_iter
constexpr int kErrInternal = 16;  // a checked build found a gathered index out of range

// A build with SISPH_CHECKED defined bounds-checks every gathered neighbour
// index before the access: an index outside [0, n) raises kErrInternal and
// is replaced by the row's own index, so the access stays in bounds and the
// host reports SISPH_EINTERNAL.  Without it the checks compile to nothing.
#ifdef SISPH_CHECKED
#define SISPH_CHECK_IDX(S, j, self)                        \
  do {                                                      \
    if (unsigned(j) >= unsigned((S).n)) {                   \
      atomicOr((S).err, kErrInternal);                      \
      (j) = (self);                                         \
    }                                                       \
  } while (0)
#define SISPH_CHECK_ENTRY(S, e, self)                       \
  do {                                                      \
    if (((e) & kIdxMask) >= unsigned((S).n)) {              \
      atomicOr((S).err, kErrInternal);                      \
      (e) = (self);                                         \
    }                                                       \
  } while (0)
#else
#define SISPH_CHECK_IDX(S, j, self) \
  do {                              \
  } while (0)
#define SISPH_CHECK_ENTRY(S, e, self) \
  do {                                \
  } while (0)
#endif

struct CaseDev {
  // cell grid
  double lo[3], hi[3], L[3], half[3];
  double lc[3], inv_lc[3];
  float lcf[3];
  int nc[3];
  int per[3];
  int morton;              // 1: Morton-interleaved cell keys, 0: row-major
  int bits;
  long long slots;         // keys per (case, kind) block
  long long key_base;      // first key of this case
  // physics (Sec. 2-3)
  double h, dt, rho0, nu, g[3], alpha, c0, tol, hfac;
  int max_iter, pgrad_symm, free_surface, ustar_slip, pref_mode, K;
  double p_ref0;
  int adaptive;            // next dt from max|u^n|, max|f^n| (Sec. 3.2)
  int solver;              // PPE: 0 damped Jacobi, 1 BiCGStab
  double dt_visc;          // 0.25 h^2 / nu (infinite without viscosity)
  // derived constants
  double cut2;             // (3h)^2, evaluated as (3*h)*(3*h)
  double skin;             // Verlet skin s: lists hold every j within 3h + s
  double cut_s2;           // (3h + s)^2
  double skin_half2;       // (s/2)^2: a larger displacement forces a rebuild
  double eh2;              // eta h^2
  double inv_h, sig_h;     // quintic at h
  double h2, inv_h2, sig_h2;  // quintic at h/2 (no-slip ghost velocity, Eq. vf)
  double hg, inv_hg, sig_hg;  // quintic at h~ = hfac h (GTVF)
  // layout in the sorted order
  int fbeg, nf, wbeg, nw;
  int wrow;                // first row of this case in the wall tables
  int ftile, nftile;       // first fluid tile, count
  int wtile, nwtile;       // first wall tile (in wall-tile numbering), count
};

struct Tile {
  int beg, end, c, kind;
};

struct Barrier {
  unsigned count;
  unsigned gen;
  int err;
  unsigned ticket;         // fluid tiles handed out by the grid-barrier sweeps
};

// Everything a kernel may need, passed by value.  Pointers are device pointers.
struct State {
  int dim, ncases, mixed, T;
  int n, nf, nw, cap, wcap, scap;
  int nft, nwt;
  const CaseDev *cases;
  const Tile *ftiles, *wtiles;
  const int *case_of;      // sorted index -> case
  const int *wall_at;      // wall row -> sorted index
  double omega, fs_ratio, eta;
  int min_iter, residual_form;
  // sort scratch
  unsigned *key, *slot, *hist;
  int *perm;
  long long K;
  // FP64 state (current buffers) and gather targets
  double *x[3], *xn[3], *u[3], *ut[3], *m, *rho, *p;
  int *uid;
  double *bx[3], *bxn[3], *bu[3], *but[3], *bm, *brho, *bp;
  int *buid;
  double *xs[3], *us[3];   // stage-1 outputs r*, u*
  double *xref[3], *bxref[3];  // position at the last rebuild of the case
  long long *cell, *bcell; // cell of the particle at that rebuild (packed)
  double *uw[3], *nrm[3];  // walls: prescribed velocity, unit normal
  double *nstar[3];        // scratch for the raw normals
  // FP32 mirrors (MIXED)
  float4 *pf4;             // cell-relative position, mass
  float4 *vf4;             // velocity, density
  float4 *utf4;            // transport velocity
  float *pf;               // pressure
  // neighbour lists (ELL, column-major: entry k of row i at k*n + i)
  unsigned *nbr;
  int *ncnt;
  unsigned *snbr;          // skin lists, same layout, capacity scap
  int *sncnt;
  int *wfin;               // wall rows: leading wall entries, final at the rebuild
  int *need;               // per case: rebuild at this refresh
  int *anyneed;            // some case needs a rebuild
  int *force;              // next refresh rebuilds every case: 1 at the
                           // current positions, 2 at the stored rebuild ones
  long long *nreb;         // rebuilds per case; [ncases]: refreshes that rebuilt
  long long *nbody;        // rebuild groups run inside conditional graph nodes
  // PPE
  void *coef;              // fac_ij per ELL slot: FP64, or {j, FP32 fac} (MIXED)
  int *pcnt;               // PPE slots per fluid row: N(i) (FP64), N(i) without i (MIXED)
  void *prhs;              // RHS_i (active) else 0
  void *pwd;               // omega / D_ii (active) else 0
  void *pb[4];             // pressure buffers: p^k in pb[k % 2] (grid barrier
                           // form) or pb[k % 4] (point-to-point form)
  double *rhs_out, *diag_out;
  int *wcnt;               // wall Shepard rows (fluid neighbours only)
  int *widx;
  void *wcoef;             // W_wf per entry
  void *wsinv, *wh;        // 1/sum W, (g . sum rho r W)
  double *tile_part;       // per fluid tile: sum|dp|, sum|p|
  double *tile_lam;        // per fluid tile: max |RHS/D|
  int *act;                // [2][ncases] case still iterating
  int *iters, *pstat, *par;// per case: sweeps, status, final buffer parity
  double *resid, *lam;
  long long *iters_tot, *solves;
  double *pref;            // per case background pressure in use
  int *pref_set;
  Barrier *bar;
  int *err;
  // point-to-point PPE sweeps (tiles numbered: fluid tiles, then wall tiles)
  int ppe_sync;            // 0 auto, 1 grid barrier per phase, 2 per-tile flags
  int p2p;                 // the sweeps take the per-tile flag form (set-up collects tile dependencies)
  int grid_cap_p2p;        // co-resident blocks of the point-to-point form
  const int *tile_of;      // sorted index -> tile
  int *deps, *ndeps;       // per tile: tiles its PPE rows read (kDepCap each)
  int *tflag;              // per tile: phases completed in this solve
  int *dsw;                // per case: convergence decisions made in this solve
  // BiCGStab (only allocated when a case uses it)
  int *inact;              // per case: free-surface rows of the last set-up
  void *kv[6];             // r, r^, p, v, t, wall s (the sweep's precision)
  double *kpart;           // per fluid tile: 4 partial sums
  double *kscal;           // per case: 8 scalars
  // GTVF
  double *dg[2][3];        // FP64 displacement ping-pong
  float4 *dgf[2];          // FP32 displacement ping-pong
  double *vgt[3];          // sub-step velocity
  // adaptive time step (only allocated when a case uses it)
  double *fs1[3];          // per fluid particle: total acceleration of the step
  unsigned long long *umax2, *fmax2;  // per case: max |u^n|^2, max |f^n|^2 (bits)
  double *tsim;            // per case: simulated time
  // debug
  long long barrier_budget;
  int debug_skip_barrier;
};

// ---------------------------------------------------------------------------
// Quintic spline with support 3h (reading of "the quintic spline", Sec. 2.1):
//   W = sigma [ (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5 ], each term where positive;
//   sigma = 7/(478 pi h^2) in 2D, 1/(120 pi h^3) in 3D.
// poly_w / poly_dw return the bracket and its derivative in q.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R poly_w(R q) {
  R w = R(0);
  if (q < R(3)) { R t = R(3) - q, t2 = t * t; w = t2 * t2 * t; }
  if (q < R(2)) { R t = R(2) - q, t2 = t * t; w -= R(6) * t2 * t2 * t; }
  if (q < R(1)) { R t = R(1) - q, t2 = t * t; w += R(15) * t2 * t2 * t; }
  return w;
}

template <typename R>
__device__ __forceinline__ R poly_dw(R q) {
  R d = R(0);
  if (q < R(3)) { R t = R(3) - q, t2 = t * t; d = R(-5) * t2 * t2; }
  if (q < R(2)) { R t = R(2) - q, t2 = t * t; d += R(30) * t2 * t2; }
  if (q < R(1)) { R t = R(1) - q, t2 = t * t; d -= R(75) * t2 * t2; }
  return d;
}

__host__ __device__ inline double quintic_sigma(double h, int dim) {
  const double pi = 3.14159265358979323846;
  return dim == 2 ? 7.0 / (478.0 * pi * h * h) : 1.0 / (120.0 * pi * h * h * h);
}

// q = r / h.  The FP64 form divides, exactly as the definition reads, so that
// a pair within rounding of the support edge gets the same (zero or tiny)
// weight as in a plain evaluation; the FP32 form multiplies by 1/h.
template <typename R>
__device__ __forceinline__ R qof(R r, R h, R inv_h) {
  if constexpr (std::is_same<R, float>::value) return r * inv_h;
  else return r / h;
}

// Per-case constants of a neighbour pass, converted once per thread to the
// pass's arithmetic type.
template <typename R>
struct KC {
  R h, ih, sig, dsc;   // support h: q = r/h, W = sig poly_w(q), dW/dr = dsc poly_dw(q)
  float lc[3];
  __device__ __forceinline__ void set(const CaseDev &P, double h_, double ih_, double sig_) {
    h = R(h_);
    ih = R(ih_);
    sig = R(sig_);
    dsc = R(sig_ * ih_);
    lc[0] = P.lcf[0];
    lc[1] = P.lcf[1];
    lc[2] = P.lcf[2];
  }
};

// |r_ij| from |r_ij|^2 in a neighbour sum.  FP64: the correctly rounded
// square root.  FP32 (MIXED): r^2 times its approximate reciprocal square
// root (rsqrtf, relative error about 1e-7, far inside the FP32 error budget
// of those sums and a few instructions where the rounded root takes a
// dozen), 0 at r^2 = 0.
template <typename R>
__device__ __forceinline__ R sqrt_r(R v) {
  if constexpr (std::is_same<R, float>::value) return v > 0.f ? v * rsqrtf(v) : 0.f;
  else return sqrt(v);
}

// The correctly rounded square root in either precision: the summation
// density, whose fused form in the neighbour filter uses the same root.
template <typename R>
__device__ __forceinline__ R sqrt_x(R v) {
  if constexpr (std::is_same<R, float>::value) return sqrtf(v);
  else return sqrt(v);
}

// Minimum-image pair vector r_ij = r_i - r_j from FP64 positions, and
// |r_ij|^2 = dx*dx + dy*dy (+ dz*dz) evaluated left to right, unfused.  B is
// a CaseDev or any type with its per/half/L members (a copy in registers).
template <int DIM, class B>
__device__ __forceinline__ double pair_d(const B &P, const double xi[3],
                                         double *const x[3], int j, double d[3]) {
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    double t = xi[k] - x[k][j];
    if (P.per[k]) {
      if (t > P.half[k]) t -= P.L[k];
      else if (t < -P.half[k]) t += P.L[k];
    }
    d[k] = t;
  }
  double r2 = __dmul_rn(d[0], d[0]);
  r2 = __dadd_rn(r2, __dmul_rn(d[1], d[1]));
  if (DIM == 3) r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
  return r2;
}

// Stencil offset o in {-1,0,1}^3 of j's cell seen from i's cell, stored in
// the top bits of a neighbour entry as 2 bits per axis: (o_x+1) | (o_y+1)<<2
// | (o_z+1)<<4.
__host__ __device__ __forceinline__ unsigned stencil_code(int ox, int oy, int oz) {
  return unsigned(ox + 1) | (unsigned(oy + 1) << 2) | (unsigned(oz + 1) << 4);
}

// Pair vector from FP32 cell-relative positions: r_ij = rel_i - rel_j - o lc.
template <int DIM>
__device__ __forceinline__ float pair_f(const float lc[3], const float4 &pi, const float4 &pj,
                                        unsigned code, float d[3]) {
  const float ox = float(int(code & 3u) - 1);
  const float oy = float(int((code >> 2) & 3u) - 1);
  d[0] = (pi.x - pj.x) - ox * lc[0];
  d[1] = (pi.y - pj.y) - oy * lc[1];
  float r2 = d[0] * d[0] + d[1] * d[1];
  if (DIM == 3) {
    const float oz = float(int(code >> 4) - 1);
    d[2] = (pi.z - pj.z) - oz * lc[2];
    r2 += d[2] * d[2];
  } else {
    d[2] = 0.f;
  }
  return r2;
}

// a / b: exact in FP64; the fast approximate division (a few ulp) in FP32,
// well inside the FP32 error budget of the MIXED form.
template <typename R>
__device__ __forceinline__ R divr(R a, R b) {
  if constexpr (std::is_same<R, float>::value) return __fdividef(a, b);
  else return a / b;
}

// Rows in chunks of 8 slots: the 8 entries are loaded first and every slot
// past the row's end is padded with the particle itself, so the gathers of a
// chunk do not depend on branches and can all be in flight at once; `valid`
// masks the padded slots out of the sums.  The next chunk's entries are
// loaded while this chunk's gathers are in flight.
#define ROW_CHUNKS(S, i, ...)                                                      \
  {                                                                                \
    const int _cnt = S.ncnt[i];                                                    \
    const long long _b = ell_base(S.cap, i);                                       \
    const unsigned _self = unsigned(i) | (stencil_code(0, 0, 0) << kCodeShift);    \
    unsigned _en[8];                                                               \
    _Pragma("unroll") for (int _u = 0; _u < 8; ++_u)                              \
      _en[_u] = _u < _cnt ? S.nbr[_b + (long long)_u * kEllBlock] : _self;        \
    for (int _q0 = 0; _q0 < _cnt; _q0 += 8) {                                      \
      unsigned _e[8];                                                              \
      _Pragma("unroll") for (int _u = 0; _u < 8; ++_u) {                          \
        _e[_u] = _en[_u];                                                          \
        SISPH_CHECK_ENTRY(S, _e[_u], _self);                                       \
        const int _q = _q0 + 8 + _u;                                               \
        _en[_u] = _q < _cnt ? S.nbr[_b + (long long)_q * kEllBlock] : _self;      \
      }                                                                            \
      _Pragma("unroll") for (int _u = 0; _u < 8; ++_u) {                          \
        const unsigned e = _e[_u];                                                 \
        const bool valid = _q0 + _u < _cnt;                                        \
        __VA_ARGS__                                                                \
      }                                                                            \
    }                                                                              \
  }

__device__ __forceinline__ void store_r(void *base, long long i, double v, int mixed) {
  if (mixed) static_cast<float *>(base)[i] = float(v);
  else static_cast<double *>(base)[i] = v;
}

// ---------------------------------------------------------------------------
// Host-side launchers (one translation unit each).
// ---------------------------------------------------------------------------
struct Launch {
  cudaStream_t stream;
  void (*before)(void *ctx, const char *name);
  void (*after)(void *ctx, const char *name, double units, int nkernels);
  void *ctx;
};

// nbr.cu: one refresh of the neighbour lists = check, rebuild, finish;
// mode 0 at the positions x, mode 1 at the stage-1 output r* (committed).
cudaError_t launch_refresh_check(const State &S, const Launch &L, int mode);
cudaError_t launch_refresh_rebuild(const State &S, const Launch &L, int mode, bool gather_static,
                                   bool count_on_device);
// density: in MIXED the in-step filter also sums the fluid rows' summation
// density (the step's refresh at r^n), replacing launch_density there
cudaError_t launch_refresh_finish(const State &S, const Launch &L, int mode, bool exact,
                                  bool density = false);
cudaError_t launch_set_conditional(const State &S, const Launch &L, cudaGraphConditionalHandle h);
constexpr int kRebuildKernels = 10;   // kernels of launch_refresh_rebuild
// passes.cu
cudaError_t launch_density(const State &S, const Launch &L);
cudaError_t launch_normals(const State &S, const Launch &L);
cudaError_t launch_ghost(const State &S, const Launch &L, int slip_stage);
cudaError_t launch_stage1(const State &S, const Launch &L);
cudaError_t launch_pgrad(const State &S, const Launch &L);
cudaError_t launch_pref(const State &S, const Launch &L);
cudaError_t launch_gtvf(const State &S, const Launch &L, int kmax, int skip_k1);
cudaError_t launch_update(const State &S, const Launch &L, int skip_k1);
cudaError_t launch_pgrad_gtvf1(const State &S, const Launch &L);
cudaError_t launch_speed_max(const State &S, const Launch &L, int which);
cudaError_t launch_adapt_dt(const State &S, const Launch &L);
cudaError_t launch_scatter_field(const State &S, const Launch &L, const void *src, int is_float,
                                 int stride_f4, int comp, double *dst_user);
cudaError_t launch_gather_field(const State &S, const Launch &L, const double *src_user, double *dst,
                                bool positions);
cudaError_t launch_scatter_disp(const State &S, const Launch &L, int comp, double *dst_user);
cudaError_t launch_refresh_mirrors(const State &S, const Launch &L);
// ppe.cu
cudaError_t launch_ppe_setup(const State &S, const Launch &L);
cudaError_t launch_ppe_reset(const State &S, const Launch &L);
cudaError_t launch_ppe_sweeps(const State &S, const Launch &L, int grid);
// krylov.cu
cudaError_t launch_ppe_krylov(const State &S, const Launch &L, int grid);
int krylov_max_blocks_per_sm(const State &S, int block);
int ppe_max_blocks_per_sm(const State &S, int block, bool p2p);

}  // namespace sisph
