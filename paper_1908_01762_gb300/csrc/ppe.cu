// Pressure-Poisson solve of SISPH (Sec. 3): set-up of the source term and of
// the per-pair coefficients (Eqs. sph-ppe, iterative-p, coeff, coeff1), the
// wall-pressure rows of Eq. p-shepard, and one persistent kernel that runs
// every damped-Jacobi sweep (Eq. p-sor) with its wall extrapolation and the
// FP64 convergence test of Eq. convergence for all cases at once.
//
// Coefficients are stored for the duration of one solve (one number per
// neighbour slot) so that each sweep streams coefficients instead of
// recomputing the kernel gradient; there is still no global matrix assembly.
#include <cooperative_groups.h>

#include "sisph_internal.h"
#include "ppe_sync.cuh"

namespace sisph {

template <typename R>
__device__ __forceinline__ void kahan_add(R &sum, R &comp, R v) {
  R y = v - comp;
  R t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// ---------------------------------------------------------------------------
// Tile dependencies of the point-to-point sweeps: the set of other tiles
// whose rows a tile's PPE rows read, collected in a shared-memory hash set
// while the rows are set up (only when the handle's sweeps take that form),
// then written as a list (ndeps = -1 when the list would exceed kDepCap or
// the set overflows: the tile then waits for every tile of its case).
// ---------------------------------------------------------------------------
constexpr int kHash = 512;

struct DepSet {
  int *tab;        // kHash slots, -1 empty
  int *over;       // overflow flag
  __device__ __forceinline__ void init() {
    for (int q = threadIdx.x; q < kHash; q += blockDim.x) tab[q] = -1;
    if (threadIdx.x == 0) *over = 0;
    __syncthreads();
  }
  __device__ __forceinline__ void insert(int key) {
    unsigned h = (unsigned(key) * 2654435761u) >> 23;
    for (int probe = 0; probe < kHash; ++probe) {
      const int cur = tab[h];
      if (cur == key) return;
      if (cur == -1) {
        const int old = atomicCAS(tab + h, -1, key);
        if (old == -1 || old == key) return;
      }
      h = (h + 1) & unsigned(kHash - 1);
    }
    *over = 1;
  }
  __device__ __forceinline__ void write(const State &S, int b, int *cnt) {
    __syncthreads();
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < kHash; q += blockDim.x) {
      const int key = tab[q];
      if (key >= 0) {
        const int pos = atomicAdd(cnt, 1);
        if (pos < kDepCap) S.deps[(long long)b * kDepCap + pos] = key;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) S.ndeps[b] = (*over || *cnt > kDepCap) ? -1 : *cnt;
  }
};

// ---------------------------------------------------------------------------
// Fluid set-up: RHS_i = sum_j -(m_j/(rho_j dt)) u*_ij . grad_i W_ij and
// fac_ij = 4 m_j/(rho_i (rho_i+rho_j)) (r_ij . grad_i W_ij)/(r^2 + eta h^2),
// D_ii = sum_j fac_ij (Kahan-compensated in FP32 for the MIXED form).  A
// particle with D_ii = 0 or on the free surface (rho_i/rho0 < fs_ratio) is
// inactive: p = 0 for the whole solve.  Lambda = max |RHS_i/D_ii| per tile.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void __launch_bounds__(256, MX ? 4 : 2) k_setup_fluid(State S) {
  using R = typename std::conditional<MX, float, double>::type;
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  const CaseDev &P = S.cases[t.c];
  __shared__ int dtab[kHash];
  __shared__ int dover, dcnt;
  DepSet deps{dtab, &dover};
  deps.init();
  double lam = 0.0;
  bool inactive = false;
  if (i < t.end) {
    KC<R> K;
    K.set(P, P.h, P.inv_h, P.sig_h);
    double xi[3] = {0, 0, 0};
    float4 pi4 = make_float4(0.f, 0.f, 0.f, 0.f);
    R ri, ui[3];
    if constexpr (MX) {
      pi4 = S.pf4[i];
      float4 v = S.vf4[i];
      ri = v.w; ui[0] = v.x; ui[1] = v.y; ui[2] = v.z;
    } else {
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) { xi[k] = S.x[k][i]; ui[k] = S.u[k][i]; }
      if (DIM == 2) ui[2] = 0.0;
      ri = S.rho[i];
    }
    const R eh2 = R(P.eh2);
    const R idt = R(1.0 / P.dt);
    const R four_iri = R(4) / ri;
    R rhs = R(0), rc = R(0), dg = R(0), dc = R(0);
    // MIXED rows whose list starts with i itself (every list a step builds)
    // leave its zero coefficient out of the packed slots: entry k goes to
    // slot k - 1; other rows keep one slot per entry
    const int shift = (MX && (S.nbr[ell_at(S.cap, 0, i)] & kIdxMask) == unsigned(i)) ? 1 : 0;
    // the row loop is compiled with and without the collection of tile
    // dependencies (point-to-point form only)
    auto rows = [&](auto p2p_form) {
    constexpr bool P2P = decltype(p2p_form)::value;
    ROW_CHUNKS(S, i, {
      const int k = _q0 + _u;
      int j = int(e & kIdxMask);
      R fac = R(0);
      // 3D: the row itself and the padding run the pair arithmetic too and
      // add nothing (no branch); 2D rows keep the branch
      const bool on = j != i;
      if (DIM == 3 || on) {
        R d[3], r2, rj, mj, uj[3];
        if constexpr (MX) {
          float4 pj = S.pf4[j];
          r2 = pair_f<DIM>(K.lc, pi4, pj, e >> kCodeShift, d);
          float4 v = S.vf4[j];
          rj = v.w; uj[0] = v.x; uj[1] = v.y; uj[2] = v.z;
          mj = fabsf(pj.w);      // the sign holds the near-range test
        } else {
          double dd[3];
          r2 = pair_d<DIM>(P, xi, S.x, j, dd);
          _Pragma("unroll") for (int q = 0; q < DIM; ++q) { d[q] = dd[q]; uj[q] = S.u[q][j]; }
          if (DIM == 2) { d[2] = 0.0; uj[2] = 0.0; }
          rj = S.rho[j];
          mj = S.m[j];
        }
        R r = sqrt_r(r2);
        R fr = r > R(0) ? divr(K.dsc * poly_dw<R>(qof<R>(r, K.h, K.ih)), r) : R(0);
        R ud = R(0);
        _Pragma("unroll") for (int q = 0; q < DIM; ++q) ud += (ui[q] - uj[q]) * d[q];
        R src = -divr(mj * idt * fr * ud, rj);
        fac = divr(four_iri * mj * (fr * r2), (ri + rj) * (r2 + eh2));
        if (!valid || !on) { src = R(0); fac = R(0); }
        if constexpr (MX) {
          if (on) {          // a compensated sum must not see the extra zeros
            kahan_add(rhs, rc, src);
            kahan_add(dg, dc, fac);
          }
        } else {
          rhs += src;
          dg += fac;
        }
      }
      if (valid && k >= shift)
        store_coef<R>(S.coef, slot_at(S, k - shift, i), j, fac);
      if (valid) {
        if (P2P && j != i) {
          const int dt = S.tile_of[j];
          if (dt != int(blockIdx.x)) deps.insert(dt);
        }
      }
    })
    };
    if (S.p2p) rows(std::true_type{});
    else rows(std::false_type{});
    S.pcnt[i] = S.ncnt[i] - shift;
    bool fs = P.free_surface && (double(ri) / P.rho0 < S.fs_ratio);
    bool active = (dg != R(0)) && !fs;
    static_cast<R *>(S.prhs)[i] = active ? rhs : R(0);
    static_cast<R *>(S.pwd)[i] = active ? R(S.omega) / dg : R(0);
    S.rhs_out[i] = double(rhs);
    S.diag_out[i] = double(dg);
    double p0 = active ? (MX ? double(S.pf[i]) : S.p[i]) : 0.0;
    static_cast<R *>(S.pb[0])[i] = R(p0);
    if (!active) {
      S.p[i] = 0.0;
      if constexpr (MX) S.pf[i] = 0.f;
    }
    if (active) lam = fabs(double(rhs) / double(dg));
    inactive = !active;
  }
  // free-surface (Dirichlet) rows per case: the BiCGStab solve needs one
  const int ninact = __syncthreads_count(inactive);
  if (threadIdx.x == 0 && ninact) atomicAdd(S.inact + t.c, ninact);
  if (S.p2p) deps.write(S, blockIdx.x, &dcnt);
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sh[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    S.tile_lam[blockIdx.x] = m;
  }
}

// ---------------------------------------------------------------------------
// Wall set-up for Eq. p-shepard: for wall w the fluid neighbours f, W_wf,
// 1/sum_f W_wf and H_w = (g - a_w) . sum_f rho_f r_wf W_wf (a_w = 0,
// r_wf = r_w - r_f), stored as compact rows so that a sweep only streams
// fluid entries.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__device__ __forceinline__ void wall_row(const State &S, const Tile &t, int i, DepSet &deps) {
  using R = typename std::conditional<MX, float, double>::type;
  const CaseDev &P = S.cases[t.c];
  KC<R> K;
  K.set(P, P.h, P.inv_h, P.sig_h);
  const int r = P.wrow + (i - P.wbeg);
  const int fend = P.fbeg + P.nf;
  double xi[3] = {0, 0, 0};
  float4 pi4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (MX) pi4 = S.pf4[i];
  else {
    _Pragma("unroll") for (int k = 0; k < DIM; ++k) xi[k] = S.x[k][i];
  }
  R sw = R(0), acc[3] = {R(0), R(0), R(0)};
  int cnt = 0;
  const int cnti = S.ncnt[i];
  R *wc = static_cast<R *>(S.wcoef);
  // fluid neighbours only: they follow the row's wall head.  Chunks of 8:
  // the entries, then the gathers, go out together before any store.
  const unsigned self = unsigned(i) | (stencil_code(0, 0, 0) << kCodeShift);
  for (int q0 = S.wfin[i]; q0 < cnti; q0 += 8) {
    unsigned e[8];
    _Pragma("unroll") for (int u = 0; u < 8; ++u) {
      e[u] = q0 + u < cnti ? S.nbr[ell_at(S.cap, q0 + u, i)] : self;
      SISPH_CHECK_ENTRY(S, e[u], self);
    }
    float4 pj[8];
    float rjf[8];
    if constexpr (MX) {
      _Pragma("unroll") for (int u = 0; u < 8; ++u) {
        const int j = int(e[u] & kIdxMask);
        pj[u] = S.pf4[j];
        rjf[u] = S.vf4[j].w;
      }
    }
    _Pragma("unroll") for (int u = 0; u < 8; ++u) {
      const int j = int(e[u] & kIdxMask);
      if (q0 + u >= cnti || j >= fend) continue;
      R d[3], r2, rj;
      if constexpr (MX) {
        r2 = pair_f<DIM>(K.lc, pi4, pj[u], e[u] >> kCodeShift, d);
        rj = rjf[u];
      } else {
        double dd[3];
        r2 = pair_d<DIM>(P, xi, S.x, j, dd);
        _Pragma("unroll") for (int q = 0; q < DIM; ++q) d[q] = dd[q];
        if (DIM == 2) d[2] = 0.0;
        rj = S.rho[j];
      }
      R w = K.sig * poly_w<R>(qof<R>(sqrt_r(r2), K.h, K.ih));
      if (S.p2p) deps.insert(S.tile_of[j]);
      S.widx[ell_at(S.wcap, cnt, r)] = j;
      wc[ell_at(S.wcap, cnt, r)] = w;
      ++cnt;
      sw += w;
      _Pragma("unroll") for (int q = 0; q < DIM; ++q) acc[q] += rj * d[q] * w;
    }
  }
  R hw = R(0);
  _Pragma("unroll") for (int q = 0; q < DIM; ++q) hw += R(P.g[q]) * acc[q];
  S.wcnt[r] = cnt;
  static_cast<R *>(S.wsinv)[r] = sw > R(0) ? R(1) / sw : R(0);
  static_cast<R *>(S.wh)[r] = hw;
}

template <int DIM, bool MX>
__global__ void k_setup_wall(State S) {
  const Tile &t = S.wtiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  __shared__ int dtab[kHash];
  __shared__ int dover, dcnt;
  DepSet deps{dtab, &dover};
  deps.init();
  if (i < t.end) wall_row<DIM, MX>(S, t, i, deps);
  if (S.p2p) deps.write(S, S.nft + blockIdx.x, &dcnt);
}


// One fluid row of Eq. p-sor: RHS_i + sum_j fac_ij p^k_j, in chunks of 8
// slots (8 independent index/coefficient loads, then 8 independent
// gathers); slots past the row's end read the row itself with a zero
// coefficient.
template <typename R>
__device__ __forceinline__ R jacobi_sum(const State &S, const R *pc, int i, R acc, int cnt) {
  const long long sb = slot_base(S, i);
  for (int q0 = 0; q0 < cnt; q0 += 8) {
    int jj[8];
    R cf[8];
    _Pragma("unroll") for (int u = 0; u < 8; ++u)
      load_coef<R>(S, sb, q0 + u, q0 + u < cnt, i, jj[u], cf[u]);
    R pj[8];
    _Pragma("unroll") for (int u = 0; u < 8; ++u) pj[u] = pc[jj[u]];
    _Pragma("unroll") for (int u = 0; u < 8; ++u) acc = fma_r(cf[u], pj[u], acc);
  }
  return acc;
}

// Block sums of |p^{k+1} - p^k| and |p^{k+1}| of one tile: in the sweep's
// precision over the tile's 256 rows, returned in FP64 in thread 0.
template <bool MX>
__device__ __forceinline__ void tile_sums(double &dn, double &dp, double *sh,
                                          typename std::conditional<MX, float, double>::type dnr,
                                          typename std::conditional<MX, float, double>::type dpr) {
  if constexpr (MX) {
    block_sum2f(dnr, dpr, sh);
    dn = double(dnr);
    dp = double(dpr);
  } else {
    dn = dnr;
    dp = dpr;
    block_sum2(dn, dp, sh);
  }
}

// Eq. convergence for case c after sweep k, by the block that completed the
// case's last tile: the tile sums are added in tile order -- thread q adds
// tiles q, q+T, q+2T, ..., then the block tree -- so the result does not
// depend on which block arrives last.  At least min_iter sweeps, at most
// max_iter.  Thread 0 records the decision; *fin_out (thread 0) receives the
// sweep count at which the case stopped, or 0 if it continues.  The result
// lives in buffer (sweeps % ring).
__device__ __forceinline__ int decide_case(const State &S, int c, int k, const double *part, double *sh,
                                           int ring) {
  const CaseDev &P = S.cases[c];
  const int T = blockDim.x;
  double num = 0.0, den = 0.0, lm = 0.0;
  for (int q = threadIdx.x; q < P.nftile; q += T) {
    num += __ldcg(part + 2 * (P.ftile + q));
    den += __ldcg(part + 2 * (P.ftile + q) + 1);
    if (k == 0) lm = fmax(lm, __ldcg(S.tile_lam + P.ftile + q));
  }
  block_sum2(num, den, sh);
  if (k == 0) {
    for (int o = 16; o > 0; o >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = sh[0];
      for (int w = 1; w < (T >> 5); ++w) m = fmax(m, sh[w]);
      S.lam[c] = m;
    }
  }
  int stop_at = 0;
  if (threadIdx.x == 0) {
    const int kk = k + 1;                    // sweeps completed
    const double lamc = S.lam[c];
    double lam = S.residual_form == 1 ? double(P.nf) * lamc : lamc;
    double dd = lam > den ? lam : den;
    double res = dd > 0.0 ? num / dd : num;
    int go = 1, st = 0;
    if (!isfinite(res)) { go = 0; st = SISPH_ENONFINITE; }
    else if (kk >= S.min_iter && res < P.tol) go = 0;
    else if (kk >= P.max_iter) { go = 0; st = SISPH_ENOTCONVERGED; }
    S.iters[c] = kk;
    S.resid[c] = res;
    if (!go) {
      S.pstat[c] = st;
      S.par[c] = kk % ring;
      S.iters_tot[c] += kk;
      S.solves[c] += 1;
      if (st == SISPH_ENONFINITE) atomicOr(S.err, kErrNonFinite);
      if (st == SISPH_ENOTCONVERGED) atomicOr(S.err, kErrNotConv);
      stop_at = kk;
    }
  }
  return stop_at;
}

// A case without fluid has nothing to solve; its solve still counts (one
// block calls this).
__device__ __forceinline__ void count_empty_solves(const State &S) {
  if (threadIdx.x == 0)
    for (int c = 0; c < S.ncases; ++c)
      if (S.cases[c].nf == 0) S.solves[c] += 1;
}

// ---------------------------------------------------------------------------
// Persistent damped-Jacobi solve for all cases, one launch, grid barrier form.
//   W phase k: every case that swept in F phase k-1 (or k = 0) extrapolates
//     its wall pressure from p^k (Eq. p-shepard, clamped at 0 for
//     free-surface flows); for a case that has just finished this is the
//     final wall update.  Skipped, with its barrier, when no case has walls.
//   F phase k: for every unfinished case
//       p^{k+1}_i = omega/D_ii (RHS_i + sum_j fac_ij p^k_j) + (1 - omega) p^k_i
//     with per-tile FP64 sums of |p^{k+1}-p^k| and |p^{k+1}|; the block that
//     completes the last tile of a case (per-case arrival counter) applies
//     Eq. convergence (decide_case).
//   grid barrier after each phase.
// Tail: once the unfinished cases have fewer fluid tiles than the grid has
// blocks (and at most kBalCases cases), block a owns the a-th of those tiles
// for the rest of the solve and every case runs its remaining sweeps on its
// own: the owners of a case meet at a per-case barrier after each phase
// (the F barrier is the arrival counter itself, released by the block that
// decides), split the case's wall rows among them, and publish what they
// wrote once the case stops; the other blocks publish the cases that had
// already stopped and leave.  No grid barrier runs in the tail, and a case
// that converges early no longer waits for the slowest one.  Every row and
// every decision is computed as in the phases above, so the result is the
// same bit for bit.
// p^k lives in buffer k&1.  Pressures written by other blocks are read with
// ordinary (L1-cached) loads: every grid (or per-case) barrier ends with an
// acquire fence in the block's master thread followed by a block barrier,
// which orders those reads after the other blocks' writes.  Flags and
// partial sums are read with ld.global.cg.
// A fluid row's slots (and a wall row's entries) go in chunks of CH: the
// chunk's index/coefficient loads, then its CH gathers.  Longer chunks shorten the chain of dependent
// loads behind each row (the tail of a phase waits for the longest chain),
// fewer registers keep more blocks per SM to hide the latency of each load:
// MIXED 3D rows (about 92 slots) take 16 at 4 blocks per SM, MIXED 2D rows
// (24-44) 12 at 4 (5 blocks spill the claim of the next tile and run no
// faster), FP64 rows 8 at 4 (wider chunks would spill).
// ---------------------------------------------------------------------------
constexpr int sweep_blocks_per_sm(bool mx, int ch) { return !mx ? 4 : ch >= 12 ? 4 : 8; }

template <bool MX>
using SweepReal = typename std::conditional<MX, float, double>::type;

// Row i of Eq. p-sor: p^{k+1}_i into pn from p^k in pc; dnr, dpr receive
// |p^{k+1}_i - p^k_i| and |p^{k+1}_i|.
template <bool MX, int CH>
__device__ __forceinline__ void sweep_row(const State &S, int i, const SweepReal<MX> *pc,
                                          SweepReal<MX> *pn, SweepReal<MX> om1, SweepReal<MX> &dnr,
                                          SweepReal<MX> &dpr) {
  using R = SweepReal<MX>;
  R acc = static_cast<const R *>(S.prhs)[i];
  const int cnt = S.pcnt[i];
  const long long sb = slot_base(S, i);
  for (int q0 = 0; q0 < cnt; q0 += CH) {
    int jj[CH];
    R cf[CH];
    _Pragma("unroll") for (int u = 0; u < CH; ++u)
      load_coef<R>(S, sb, q0 + u, q0 + u < cnt, i, jj[u], cf[u]);
    R pj[CH];
    _Pragma("unroll") for (int u = 0; u < CH; ++u) pj[u] = pc[jj[u]];
    _Pragma("unroll") for (int u = 0; u < CH; ++u) acc = fma_r(cf[u], pj[u], acc);
  }
  const R po = pc[i];
  const R pnew = jacobi_update(static_cast<const R *>(S.pwd)[i], acc, om1, po);
  pn[i] = pnew;
  dnr = fabs(pnew - po);
  dpr = fabs(pnew);
}

// Master thread: wait until the per-case generation counter leaves g0.
// false after the barrier budget (the timeout flag is raised) or when
// another block has raised an error.
__device__ __forceinline__ bool case_wait(const State &S, const unsigned *gen, unsigned g0) {
  volatile const unsigned *vg = gen;
  volatile const int *verr = &S.bar->err;
  const long long t0 = clock64();
  while (*vg == g0) {
    if (*verr) return false;
    if (clock64() - t0 > S.barrier_budget) {
      atomicExch(&S.bar->err, kErrTimeout);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Final pressure of row i from buffer b into the FP64 state (and its FP32
// mirror).
template <bool MX>
__device__ __forceinline__ void publish_row(const State &S, int i, int b) {
  const SweepReal<MX> v = __ldcg(static_cast<const SweepReal<MX> *>(S.pb[b]) + i);
  S.p[i] = double(v);
  if constexpr (MX) S.pf[i] = v;
}

// The tail of the grid-barrier solve from F phase k on (see above).  apre is
// the prefix of the unfinished cases' fluid tiles at that point (ntiles in
// all, fewer than the grid's blocks).  Returns false when a wait failed (the
// error word is set).
template <bool MX, int CH>
__device__ __forceinline__ bool sweep_tail(const State &S, const int *apre, int ntiles, int k, int kcap,
                                           bool skip, double *sh, int *shv) {
  using R = SweepReal<MX>;
  // chunks of at most 12 here: the tail's own state would otherwise push
  // the 16-wide 3D rows past the kernel's registers (the sums do not depend
  // on the chunk width)
  constexpr int CT = CH < 12 ? CH : 12;
  const int T = blockDim.x;
  const int nc = S.ncases;
  const R om1 = R(1.0 - S.omega);
  int *done = S.act;
  int *fin = S.act + nc;
  unsigned *arrive = reinterpret_cast<unsigned *>(S.par + nc);       // [nc]
  unsigned *wbar = reinterpret_cast<unsigned *>(S.par + 2 * nc);     // [nc] wall-phase arrivals
  unsigned *gen = reinterpret_cast<unsigned *>(S.par + 3 * nc);      // [nc] barrier generations
  if (int(blockIdx.x) >= ntiles) {
    // cases that stopped before the tail (or never swept) are final:
    // their last writes came before the grid barrier that preceded it
    for (int i = (int(blockIdx.x) - ntiles) * T + threadIdx.x; i < S.n;
         i += (int(gridDim.x) - ntiles) * T) {
      const int c = S.case_of[i];
      if (!jacobi_case(S, c) || apre[c + 1] > apre[c]) continue;
      publish_row<MX>(S, i, __ldcg(S.par + c));
    }
    return true;
  }
  const int a = blockIdx.x;
  const int c = case_of_index(apre, nc, a);
  const int q = a - apre[c];                 // this block's rank among the case's owners
  const CaseDev &P = S.cases[c];
  const int m = P.nftile;                    // owners: every fluid tile of the case
  const int tt = P.ftile + q;
  const Tile &t = S.ftiles[tt];
  const int i = t.beg + threadIdx.x;
  int kk = k;
  int stop = 0;                              // sweep count at which the case stopped
  for (;;) {
    const R *pc = static_cast<const R *>(S.pb[kk & 1]);
    R *pn = static_cast<R *>(S.pb[(kk & 1) ^ 1]);
    // ---- F(kk) on the owned tile; arrival, decision and release ----
    R dnr = R(0), dpr = R(0);
    if (i < t.end) sweep_row<MX, CT>(S, i, pc, pn, om1, dnr, dpr);
    double dn, dp;
    tile_sums<MX>(dn, dp, sh, dnr, dpr);
    unsigned g0 = 0u;
    if (threadIdx.x == 0) {
      S.tile_part[2 * tt] = dn;
      S.tile_part[2 * tt + 1] = dp;
      g0 = *reinterpret_cast<volatile unsigned *>(gen + c);
      __threadfence();
      *shv = skip ? 0 : (atomicAdd(arrive + c, 1u) == unsigned(m - 1));
    }
    __syncthreads();
    const bool decider = *shv != 0;
    __syncthreads();
    if (decider) {
      __threadfence();
      const int stop_at = decide_case(S, c, kk, S.tile_part, sh, 2);
      if (threadIdx.x == 0) {
        arrive[c] = 0u;
        if (stop_at) {
          fin[c] = stop_at;
          __threadfence();
          done[c] = 1;
        }
        __threadfence();
        atomicAdd(gen + c, 1u);
        *shv = stop_at;
      }
    } else if (threadIdx.x == 0) {
      const bool ok = case_wait(S, gen + c, g0);
      __threadfence();
      *shv = ok ? __ldcg(fin + c) : -1;
    }
    __syncthreads();
    stop = *shv;
    __syncthreads();
    if (stop < 0) return false;
    skip = false;
    ++kk;
    // ---- W(kk): the case's wall rows, split over its owners (the final
    // wall update when the case has just stopped) ----
    R *pw = static_cast<R *>(S.pb[kk & 1]);
    for (int rr = q * T + threadIdx.x; rr < P.nw; rr += m * T) {
      const int r = P.wrow + rr;
      const int w = S.wall_at[r];
      pw[w] = wall_pressure<R, CT>(S, pw, r, w, c);
    }
    if (stop) break;
    if (P.nw > 0) {
      if (threadIdx.x == 0) {
        g0 = *reinterpret_cast<volatile unsigned *>(gen + c);
        __threadfence();
        bool ok = true;
        if (atomicAdd(wbar + c, 1u) == unsigned(m - 1)) {
          wbar[c] = 0u;
          __threadfence();
          atomicAdd(gen + c, 1u);
        } else {
          ok = case_wait(S, gen + c, g0);
        }
        __threadfence();
        *shv = ok ? 1 : 0;
      }
      __syncthreads();
      const bool ok = *shv != 0;
      __syncthreads();
      if (!ok) return false;
    }
    if (kk >= kcap) {
      if (threadIdx.x == 0) atomicOr(S.err, kErrNotConv);
      return true;
    }
  }
  // ---- publish what this block wrote last: its fluid rows (F(stop-1))
  // and its share of the wall rows (W(stop)), both in buffer stop & 1 ----
  if (i < t.end) publish_row<MX>(S, i, stop & 1);
  for (int rr = q * T + threadIdx.x; rr < P.nw; rr += m * T) publish_row<MX>(S, S.wall_at[P.wrow + rr], stop & 1);
  return true;
}

template <bool MX, int CH, bool TAIL>
__global__ void __launch_bounds__(256, sweep_blocks_per_sm(MX, CH)) k_sweeps(State S) {
  using R = SweepReal<MX>;
  __shared__ double sh[64];
  __shared__ int flag;
  __shared__ int apre[kBalCases + 1];
  __shared__ int wsum[33];
  __shared__ int tnext;
  const unsigned nb = gridDim.x;
  const int T = blockDim.x;
  const int nc = S.ncases;
  const R om1 = R(1.0 - S.omega);
  int *done = S.act;                 // [nc] case finished
  int *fin = S.act + nc;             // [nc] sweep count at which it finished
  unsigned *arrive = reinterpret_cast<unsigned *>(S.par + nc);  // [nc]
  bool skip = S.debug_skip_barrier && blockIdx.x == 1;
  bool alive = true, tail = false;
  // hard bound on the loop: every case stops at its max_iter at the latest
  int kcap = 0;
  for (int c = 0; c < nc; ++c) kcap = max(kcap, S.cases[c].max_iter);
  int k = 0;
  // tickets handed out before the current F phase: in every phase each tile
  // is claimed once and each block makes one claim past the end
  unsigned tbase = 0u;
  for (;;) {
    const int cur = k & 1;
    R *pc = static_cast<R *>(S.pb[cur]);
    // ---- W phase: wall extrapolation from p^k ----
    if (S.nw > 0) {
      // wall rows of the cases that take this phase, spread over the grid
      const bool bal = nc <= kBalCases;
      // (a case takes W phase k unless it stopped with fin < k sweeps)
      const int nrows = bal ? case_prefix(nc, apre, wsum, [&](int c) {
        const int f = __ldcg(fin + c);
        return (jacobi_case(S, c) && (k == 0 || f == 0 || f == k)) ? S.cases[c].nw : 0;
      }) : S.nw;
      for (int a = blockIdx.x * T + threadIdx.x; a < nrows; a += nb * T) {
        int r = a;
        if (bal) {
          const int c = case_of_index(apre, nc, a);
          r = S.cases[c].wrow + (a - apre[c]);
        }
        int w = S.wall_at[r];
        int c = S.case_of[w];
        if (!bal && (!jacobi_case(S, c) || (k > 0 && __ldcg(done + c) && __ldcg(fin + c) != k))) continue;
        pc[w] = wall_pressure<R, CH>(S, pc, r, w, c);
      }
      alive = grid_sync(S.bar, nb, S.barrier_budget, skip);
      skip = false;
      if (!alive) break;
    }
    // ---- any case left?  (a case without fluid has nothing to solve) ----
    int mine = 0;
    for (int c = threadIdx.x; c < nc; c += T)
      mine |= (__ldcg(done + c) == 0 && S.cases[c].nf > 0 && jacobi_case(S, c));
    if (!__syncthreads_or(mine)) break;
    if (k >= kcap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(S.err, kErrNotConv);
      break;
    }
    // ---- F phase: one damped-Jacobi sweep of the unfinished cases ----
    R *pn = static_cast<R *>(S.pb[cur ^ 1]);
    // fluid tiles of the unfinished cases, spread over the grid.  A case is
    // counted by its stop count alone, which is 0 until it stops and then
    // k + 1 if it stops in this very phase: every block, whenever it looks,
    // counts the same cases.
    const bool bal = nc <= kBalCases;
    const int ntiles = bal ? case_prefix(nc, apre, wsum, [&](int c) {
      const int f = __ldcg(fin + c);
      return (jacobi_case(S, c) && (f == 0 || f > k)) ? S.cases[c].nftile : 0;
    }) : S.nft;
    // fewer tiles than blocks: the tail (every block takes the same branch,
    // since all read the same stop counts after the grid barrier)
    if (TAIL && bal && ntiles < int(nb)) {
      alive = sweep_tail<MX, CH>(S, apre, ntiles, k, kcap, skip, sh, &flag);
      tail = true;
      break;
    }
    // Tiles are claimed from a grid-wide ticket counter, so a block that
    // finishes early takes more of them; thread 0 claims the next tile while
    // the block works on the current one.  Which block runs a tile changes
    // nothing: its sums are per tile and the decisions add them in tile order.
    if (threadIdx.x == 0) tnext = int(atomicAdd(&S.bar->ticket, 1u) - tbase);
    __syncthreads();
    int a = tnext;
    __syncthreads();
    while (a < ntiles) {
      int claim = 0;
      if (threadIdx.x == 0) claim = int(atomicAdd(&S.bar->ticket, 1u) - tbase);
      int tt = a;
      if (bal) {
        const int c = case_of_index(apre, nc, a);
        tt = S.cases[c].ftile + (a - apre[c]);
      }
      const Tile &t = S.ftiles[tt];
      if (!bal && (__ldcg(done + t.c) || !jacobi_case(S, t.c))) {
        if (threadIdx.x == 0) tnext = claim;
        __syncthreads();
        a = tnext;
        __syncthreads();
        continue;
      }
      int i = t.beg + threadIdx.x;
      R dnr = R(0), dpr = R(0);
      if (i < t.end) sweep_row<MX, CH>(S, i, pc, pn, om1, dnr, dpr);
      double dn, dp;
      tile_sums<MX>(dn, dp, sh, dnr, dpr);
      if (threadIdx.x == 0) {
        S.tile_part[2 * tt] = dn;
        S.tile_part[2 * tt + 1] = dp;
        __threadfence();
        const CaseDev &P = S.cases[t.c];
        flag = (atomicAdd(arrive + t.c, 1u) == unsigned(P.nftile - 1));
      }
      __syncthreads();
      if (flag) {
        __threadfence();
        const int c = t.c;
        const int stop_at = decide_case(S, c, k, S.tile_part, sh, 2);
        if (threadIdx.x == 0) {
          arrive[c] = 0u;
          if (stop_at) {
            fin[c] = stop_at;
            __threadfence();
            done[c] = 1;
          }
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) tnext = claim;
      __syncthreads();
      a = tnext;
      __syncthreads();
    }
    tbase += unsigned(ntiles) + nb;
    alive = grid_sync(S.bar, nb, S.barrier_budget, skip);
    skip = false;
    if (!alive) break;
    ++k;
  }
  if (!alive) return;
  // ---- publish the final pressure of every case (the tail has published
  // its cases itself) ----
  if (!tail)
    for (int i = blockIdx.x * T + threadIdx.x; i < S.n; i += nb * T) {
      const int c = S.case_of[i];
      if (jacobi_case(S, c)) publish_row<MX>(S, i, __ldcg(S.par + c));
    }
  if (blockIdx.x == 0) count_empty_solves(S);
}

// ---------------------------------------------------------------------------
// Persistent damped-Jacobi solve, point-to-point form: no grid barrier.
// Every tile (fluid tiles, then wall tiles, numbered 0..nft+nwt) counts its
// completed phases in a flag.  Phase W(k) of a wall tile needs F(k-1) done
// in the fluid tiles its rows read; phase F(k) of a fluid tile needs F(k-1)
// done in its fluid dependencies and W(k) done in its wall dependencies (the
// lists are built with the PPE rows; a tile whose list overflowed waits for
// every tile of its case).  Neighbourhoods are symmetric, so neighbouring
// tiles are never more than one phase apart.
// p^k lives in buffer k % 4.  The convergence decision after sweep k
// (decide_case) is awaited with a lag: W(k) and F(k) wait for the decision
// after sweep k - lag(k) (lag 2 for the first sweeps, 4 after), so tiles run
// ahead while the decision is being made.  A case that stopped with fin
// sweeps needs F(k) for k < fin and W(k) for k <= fin (W(fin) is the final
// wall update); a phase known to be unneeded is skipped, one not yet known
// runs and writes a buffer other than fin % 4 (the lag never exceeds the
// ring), so which phases run may depend on timing but the result does not:
// it equals the grid barrier form's bit for bit.  Needed phases wait only on
// needed phases; a waiting phase that learns it is unneeded gives up.  A
// block takes its tiles phase by phase (W tiles, then F tiles, for k = 0,
// 1, ...); every wait is for an earlier phase, so co-resident blocks always
// progress.  Waits are bounded: past the budget the kernel raises the
// timeout flag and every block returns.
// ---------------------------------------------------------------------------
constexpr int kRing = 4;

__device__ __forceinline__ int p2p_lag(int k) { return k < 4 ? 2 : kRing; }

__device__ __forceinline__ bool p2p_aborted(const State &S) {
  return *reinterpret_cast<volatile int *>(&S.bar->err) != 0;
}

// Whether phase k (wall: W(k), else F(k)) of case c is known to be unneeded.
__device__ __forceinline__ bool p2p_unneeded(const State &S, int c, int k, bool wall) {
  if (!*reinterpret_cast<volatile const int *>(S.act + c)) return false;
  __threadfence();
  const int fin = __ldcg(S.act + S.ncases + c);
  return wall ? fin <= k - 1 : fin <= k;
}

// Wait (one thread) until *f >= need.  1: reached; 0: the phase turned out
// unneeded; -1: timeout or abort.
__device__ __forceinline__ int p2p_wait(const State &S, const int *f, int need, int c, int k, bool wall) {
  volatile const int *vf = f;
  if (*vf >= need) return 1;
  const long long t0 = clock64();
  for (;;) {
    __nanosleep(32);
    if (*vf >= need) return 1;
    if (p2p_unneeded(S, c, k, wall)) return 0;
    if (p2p_aborted(S)) return -1;
    if (clock64() - t0 > S.barrier_budget) {
      atomicExch(&S.bar->err, kErrTimeout);
      return -1;
    }
  }
}

// Whether phase k of a tile of case c runs: waits for the decision after
// sweep k - lag(k), then skips the phase if it is known to be unneeded.
// 1 run, 0 skip, -1 timeout.  Block-uniform.
__device__ __forceinline__ int p2p_runs(const State &S, int c, int k, bool wall, int *shv) {
  if (threadIdx.x == 0) {
    int r = 1;
    const CaseDev &P = S.cases[c];
    if (!jacobi_case(S, c)) {
      r = 0;                                     // solved by BiCGStab
    } else if (P.nf == 0) {
      r = (wall && k == 0) ? 1 : 0;             // nothing to solve: W(0) only
    } else {
      const int need = k - p2p_lag(k) + 1;       // decisions made
      if (need > 0) r = p2p_wait(S, S.dsw + c, need, c, k, wall);
      if (r == 1 && p2p_unneeded(S, c, k, wall)) r = 0;
      if (r == 1) __threadfence();
    }
    *shv = r;
  }
  __syncthreads();
  const int r = *shv;
  __syncthreads();           // every thread has read it before it is reused
  return r;
}

// Wait for the dependencies of tile b before its phase k: fluid tiles must
// have completed need_f phases, wall tiles need_w.  1 run, 0 skip (the
// phase turned out unneeded), -1 timeout.  Block-uniform.
__device__ __forceinline__ int p2p_deps(const State &S, int b, int c, int k, bool wall, int need_f,
                                        int need_w) {
  const int nd = S.ndeps[b];
  int r = 1;
  if (nd >= 0) {
    for (int q = threadIdx.x; q < nd && r == 1; q += blockDim.x) {
      const int d = S.deps[(long long)b * kDepCap + q];
      r = p2p_wait(S, S.tflag + d, d < S.nft ? need_f : need_w, c, k, wall);
    }
  } else {
    // overflowed list: every tile of the case
    const CaseDev &P = S.cases[c];
    const int nt = P.nftile + (wall ? 0 : P.nwtile);
    for (int q = threadIdx.x; q < nt && r == 1; q += blockDim.x) {
      const int d = q < P.nftile ? P.ftile + q : S.nft + P.wtile + (q - P.nftile);
      r = p2p_wait(S, S.tflag + d, d < S.nft ? need_f : need_w, c, k, wall);
    }
  }
  if (r == 1) __threadfence();
  const int bad = __syncthreads_or(r < 0);
  const int skip = __syncthreads_or(r == 0);
  return bad ? -1 : (skip ? 0 : 1);
}

__device__ __forceinline__ void p2p_signal(const State &S, int b, int value) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *reinterpret_cast<volatile int *>(S.tflag + b) = value;
  }
}

// The decision block (the grid's last block, which owns no tile): for every
// case in turn it waits until all fluid tiles have added their sums of sweep
// dsw[c], applies Eq. convergence (decide_case) and publishes the decision.
// Tiles never wait for it except through the lag.  Returns false on timeout.
template <bool MX>
__device__ bool p2p_decide_loop(const State &S, double *sh, int *shv) {
  const int nc = S.ncases;
  unsigned *arrive = reinterpret_cast<unsigned *>(S.par + nc);   // [kRing][nc]
  long long t_last = clock64();
  for (;;) {
    bool progress = false, left = false;
    for (int c = 0; c < nc; ++c) {
      const CaseDev &P = S.cases[c];
      if (P.nf == 0 || !jacobi_case(S, c)) continue;
      if (threadIdx.x == 0) {
        int r = 0;       // 0: case done, 1: not ready, 2: decide sweep k
        if (!*reinterpret_cast<volatile const int *>(S.act + c)) {
          const int k = *reinterpret_cast<volatile const int *>(S.dsw + c);
          const unsigned got = *reinterpret_cast<volatile const unsigned *>(arrive + (k % kRing) * nc + c);
          r = got >= unsigned(P.nftile) ? 2 : 1;
        }
        *shv = r;
      }
      __syncthreads();
      const int r = *shv;
      __syncthreads();
      if (r == 0) continue;
      left = true;
      if (r == 1) continue;
      __threadfence();
      const int k = __ldcg(S.dsw + c);
      const int cur = k % kRing;
      const int stop_at = decide_case(S, c, k, S.tile_part + size_t(2) * S.nft * cur, sh, kRing);
      if (threadIdx.x == 0) {
        arrive[cur * nc + c] = 0u;
        if (stop_at) {
          S.act[nc + c] = stop_at;
          __threadfence();
          *reinterpret_cast<volatile int *>(S.act + c) = 1;
        }
        __threadfence();
        *reinterpret_cast<volatile int *>(S.dsw + c) = k + 1;
      }
      __syncthreads();
      progress = true;
    }
    if (!left) return true;
    if (progress) {
      t_last = clock64();
      continue;
    }
    if (threadIdx.x == 0) {
      int bad = p2p_aborted(S) ? 1 : 0;
      if (!bad && clock64() - t_last > S.barrier_budget) {
        atomicExch(&S.bar->err, kErrTimeout);
        bad = 1;
      }
      *shv = bad;
      if (!bad) __nanosleep(64);
    }
    __syncthreads();
    const int bad = *shv;
    __syncthreads();
    if (bad) return false;
  }
}

template <bool MX>
__global__ void __launch_bounds__(256, MX ? 5 : 4) k_sweeps_p2p(State S) {
  using R = typename std::conditional<MX, float, double>::type;
  __shared__ double sh[64];
  __shared__ int shv;
  const int nb = gridDim.x - 1;      // tile blocks; the last block decides
  const int nc = S.ncases;
  if (int(blockIdx.x) == nb) {
    if (p2p_decide_loop<MX>(S, sh, &shv)) count_empty_solves(S);
    return;
  }
  const R om1 = R(1.0 - S.omega);
  const R *prhs = static_cast<const R *>(S.prhs);
  const R *pwd = static_cast<const R *>(S.pwd);
  unsigned *arrive = reinterpret_cast<unsigned *>(S.par + nc);   // [kRing][nc]
  // test hook: block 1 never signals a phase nor adds its sums, so every
  // wait on it runs out
  const bool skip = S.debug_skip_barrier && blockIdx.x == 1;
  bool alive = true;
  for (int k = 0; alive; ++k) {
    const int cur = k % kRing;
    R *pc = static_cast<R *>(S.pb[cur]);
    R *pn = static_cast<R *>(S.pb[(k + 1) % kRing]);
    bool ran = false;
    // ---- W(k) on this block's wall tiles ----
    for (int wt = blockIdx.x; wt < S.nwt && alive; wt += nb) {
      const Tile &t = S.wtiles[wt];
      int run = p2p_runs(S, t.c, k, true, &shv);
      if (run == 1) run = p2p_deps(S, S.nft + wt, t.c, k, true, k, 0);
      if (run < 0) { alive = false; break; }
      if (!run) continue;
      ran = true;
      const int w = t.beg + threadIdx.x;
      if (w < t.end) {
        const CaseDev &P = S.cases[t.c];
        const int r = P.wrow + (w - P.wbeg);
        pc[w] = wall_pressure<R>(S, pc, r, w, t.c);
      }
      if (skip) continue;
      p2p_signal(S, S.nft + wt, k + 1);
    }
    // ---- F(k) on this block's fluid tiles ----
    for (int tt = blockIdx.x; tt < S.nft && alive; tt += nb) {
      const Tile &t = S.ftiles[tt];
      int run = p2p_runs(S, t.c, k, false, &shv);
      if (run == 1) run = p2p_deps(S, tt, t.c, k, false, k, k + 1);
      if (run < 0) { alive = false; break; }
      if (!run) continue;
      ran = true;
      const int i = t.beg + threadIdx.x;
      R dnr = R(0), dpr = R(0);
      if (i < t.end) {
        R acc = jacobi_sum<R>(S, pc, i, prhs[i], S.pcnt[i]);
        R po = pc[i];
        R pnew = jacobi_update(pwd[i], acc, om1, po);
        pn[i] = pnew;
        dnr = fabs(pnew - po);
        dpr = fabs(pnew);
      }
      if (skip) continue;
      p2p_signal(S, tt, k + 1);
      double dn, dp;
      tile_sums<MX>(dn, dp, sh, dnr, dpr);
      if (threadIdx.x == 0) {
        double *part = S.tile_part + size_t(2) * S.nft * cur;
        part[2 * tt] = dn;
        part[2 * tt + 1] = dp;
        __threadfence();
        atomicAdd(arrive + cur * nc + t.c, 1u);
      }
    }
    if (!ran) break;
  }
  if (!alive) return;
  // ---- publish the final pressure of the tiles this block owns (the same
  // fluid and wall tiles as in the phases above: their last writes to the
  // final buffer were this block's own) ----
  for (int kind = 0; kind < 2; ++kind) {
    const int ntk = kind ? S.nwt : S.nft;
    for (int b = blockIdx.x; b < ntk; b += nb) {
      const Tile &t = kind ? S.wtiles[b] : S.ftiles[b];
      const int i = t.beg + threadIdx.x;
      if (i >= t.end || !jacobi_case(S, t.c)) continue;
      const R v = __ldcg(static_cast<const R *>(S.pb[__ldcg(S.par + t.c)]) + i);
      S.p[i] = double(v);
      if constexpr (MX) S.pf[i] = v;
    }
  }
}

cudaError_t launch_ppe_setup(const State &S, const Launch &L) {
  cudaMemsetAsync(S.inact, 0, sizeof(int) * size_t(S.ncases), L.stream);
  if (S.nft) {
    if (L.before) L.before(L.ctx, "ppe_setup");
    if (S.dim == 2) {
      if (S.mixed) k_setup_fluid<2, true><<<S.nft, S.T, 0, L.stream>>>(S);
      else k_setup_fluid<2, false><<<S.nft, S.T, 0, L.stream>>>(S);
    } else {
      if (S.mixed) k_setup_fluid<3, true><<<S.nft, S.T, 0, L.stream>>>(S);
      else k_setup_fluid<3, false><<<S.nft, S.T, 0, L.stream>>>(S);
    }
    if (L.after) L.after(L.ctx, "ppe_setup", double(S.nf), 1);
  }
  if (S.nwt) {
    if (L.before) L.before(L.ctx, "ppe_setup_wall");
    if (S.dim == 2) {
      if (S.mixed) k_setup_wall<2, true><<<S.nwt, S.T, 0, L.stream>>>(S);
      else k_setup_wall<2, false><<<S.nwt, S.T, 0, L.stream>>>(S);
    } else {
      if (S.mixed) k_setup_wall<3, true><<<S.nwt, S.T, 0, L.stream>>>(S);
      else k_setup_wall<3, false><<<S.nwt, S.T, 0, L.stream>>>(S);
    }
    if (L.after) L.after(L.ctx, "ppe_setup_wall", double(S.nw), 1);
  }
  return cudaGetLastError();
}

// The barrier-form kernel for the state's precision and dimension.
using SweepKernel = void (*)(State);
// The tail is compiled in for batches only: a single case's grid is sized to
// its own tiles, so a per-case barrier would be its grid barrier, and the
// tail's code costs the 3D kernel about 1 % of its sweep time.
SweepKernel sweep_kernel(const State &S) {
  const bool tail = S.ncases > 1;
  if (!S.mixed) return tail ? k_sweeps<false, 8, true> : k_sweeps<false, 8, false>;
  if (S.dim == 3) return tail ? k_sweeps<true, 16, true> : k_sweeps<true, 16, false>;
  return tail ? k_sweeps<true, 12, true> : k_sweeps<true, 12, false>;
}

int ppe_max_blocks_per_sm(const State &S, int block, bool p2p) {
  int nb = 0;
  if (p2p) {
    if (S.mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweeps_p2p<true>, block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweeps_p2p<false>, block, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel(S), block, 0);
  }
  return nb;
}

// Per-solve state shared by the BiCGStab and Jacobi launches (each touches
// only its own cases' entries).
cudaError_t launch_ppe_reset(const State &S, const Launch &L) {
  const size_t nc = size_t(S.ncases);
  // done[nc], fin[nc]; par[nc] and the arrival counters par[nc..5nc)
  cudaMemsetAsync(S.act, 0, 2 * sizeof(int) * nc, L.stream);
  cudaMemsetAsync(S.par, 0, (1 + kRing) * sizeof(int) * nc, L.stream);
  cudaMemsetAsync(S.iters, 0, sizeof(int) * nc, L.stream);
  cudaMemsetAsync(S.pstat, 0, sizeof(int) * nc, L.stream);
  return cudaGetLastError();
}

cudaError_t launch_ppe_sweeps(const State &S, const Launch &L, int grid) {
  const size_t nc = size_t(S.ncases);
  cudaMemsetAsync(S.bar, 0, sizeof(Barrier), L.stream);
  // point-to-point form when every block can own at most one fluid and one
  // wall tile (its per-tile waits would otherwise add up), unless forced; it
  // takes one more block, which makes the convergence decisions
  const int tiles = S.nft > S.nwt ? S.nft : S.nwt;
  const bool p2p = S.p2p != 0;
  if (p2p) grid = (tiles + 1 < S.grid_cap_p2p ? tiles + 1 : S.grid_cap_p2p);
  if (p2p && grid < 2) grid = 2;
  if (p2p) {
    cudaMemsetAsync(S.dsw, 0, sizeof(int) * nc, L.stream);
    cudaMemsetAsync(S.tflag, 0, sizeof(int) * size_t(S.nft + S.nwt > 0 ? S.nft + S.nwt : 1), L.stream);
  }
  if (L.before) L.before(L.ctx, "ppe_sweeps");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(S.T);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (p2p) {
    if (S.mixed) e = cudaLaunchKernelEx(&cfg, k_sweeps_p2p<true>, S);
    else e = cudaLaunchKernelEx(&cfg, k_sweeps_p2p<false>, S);
  } else {
    e = cudaLaunchKernelEx(&cfg, sweep_kernel(S), S);
  }
  if (L.after) L.after(L.ctx, "ppe_sweeps", 0.0, 1);
  return e;
}

}  // namespace sisph
