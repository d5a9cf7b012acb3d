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

namespace sisph {

template <typename R>
__device__ __forceinline__ void kahan_add(R &sum, R &comp, R v) {
  R y = v - comp;
  R t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// ---------------------------------------------------------------------------
// Fluid set-up: RHS_i = sum_j -(m_j/(rho_j dt)) u*_ij . grad_i W_ij and
// fac_ij = 4 m_j/(rho_i (rho_i+rho_j)) (r_ij . grad_i W_ij)/(r^2 + eta h^2),
// D_ii = sum_j fac_ij (Kahan-compensated in FP32 for the MIXED form).  A
// particle with D_ii = 0 or on the free surface (rho_i/rho0 < fs_ratio) is
// inactive: p = 0 for the whole solve.  Lambda = max |RHS_i/D_ii| per tile.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void k_setup_fluid(State S) {
  using R = typename std::conditional<MX, float, double>::type;
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  const CaseDev &P = S.cases[t.c];
  double lam = 0.0;
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
    R *coef = static_cast<R *>(S.coef);
    ROW_CHUNKS(S, i, {
      const int k = _q0 + _u;
      int j = int(e & kIdxMask);
      R fac = R(0);
      if (j != i) {
        R d[3], r2, rj, mj, uj[3];
        if constexpr (MX) {
          float4 pj = S.pf4[j];
          r2 = pair_f<DIM>(K.lc, pi4, pj, e >> kCodeShift, d);
          float4 v = S.vf4[j];
          rj = v.w; uj[0] = v.x; uj[1] = v.y; uj[2] = v.z;
          mj = pj.w;
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
        if (!valid) { src = R(0); fac = R(0); }
        if constexpr (MX) {
          kahan_add(rhs, rc, src);
          kahan_add(dg, dc, fac);
        } else {
          rhs += src;
          dg += fac;
        }
      }
      if (valid) coef[(long long)k * _n + i] = fac;
    })
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
  }
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
__global__ void k_setup_wall(State S) {
  using R = typename std::conditional<MX, float, double>::type;
  const Tile &t = S.wtiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
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
  const long long n = S.n, nw = S.nw;
  R *wc = static_cast<R *>(S.wcoef);
  for (int k = 0; k < cnti; ++k) {
    unsigned e = S.nbr[(long long)k * n + i];
    int j = int(e & kIdxMask);
    if (j >= fend) continue;
    R d[3], r2, rj;
    if constexpr (MX) {
      float4 pj = S.pf4[j];
      r2 = pair_f<DIM>(K.lc, pi4, pj, e >> kCodeShift, d);
      rj = S.vf4[j].w;
    } else {
      double dd[3];
      r2 = pair_d<DIM>(P, xi, S.x, j, dd);
      _Pragma("unroll") for (int q = 0; q < DIM; ++q) d[q] = dd[q];
      if (DIM == 2) d[2] = 0.0;
      rj = S.rho[j];
    }
    R w = K.sig * poly_w<R>(qof<R>(sqrt_r(r2), K.h, K.ih));
    S.widx[(long long)cnt * nw + r] = j;
    wc[(long long)cnt * nw + r] = w;
    ++cnt;
    sw += w;
    _Pragma("unroll") for (int q = 0; q < DIM; ++q) acc[q] += rj * d[q] * w;
  }
  R hw = R(0);
  _Pragma("unroll") for (int q = 0; q < DIM; ++q) hw += R(P.g[q]) * acc[q];
  S.wcnt[r] = cnt;
  static_cast<R *>(S.wsinv)[r] = sw > R(0) ? R(1) / sw : R(0);
  static_cast<R *>(S.wh)[r] = hw;
}

// ---------------------------------------------------------------------------
// Grid barrier with a bounded wait.  All blocks are co-resident (cooperative
// launch).  A wait that exceeds `budget` clock cycles, or that sees another
// block's error, marks the error word and returns false; the caller returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_sync(Barrier *b, unsigned nblocks, long long budget, bool skip_arrive) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *vgen = &b->gen;
    volatile int *verr = &b->err;
    unsigned g = *vgen;
    __threadfence();
    bool last = false;
    if (!skip_arrive) last = (atomicAdd(&b->count, 1u) == nblocks - 1);
    if (last) {
      b->count = 0;
      __threadfence();
      atomicExch(&b->gen, g + 1u);
    } else {
      long long t0 = clock64();
      while (*vgen == g) {
        if (*verr) { ok = 0; break; }
        if (clock64() - t0 > budget) {
          atomicExch(&b->err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void block_sum2f(float &a, float &b, double *sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float *shf = reinterpret_cast<float *>(sh);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { shf[w] = a; shf[32 + w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float sa = 0.f, sb = 0.f;
    for (int q = 0; q < nw; ++q) { sa += shf[q]; sb += shf[32 + q]; }
    a = sa;
    b = sb;
  }
}

__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { sh[w] = a; sh[32 + w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < nw; ++q) { sa += sh[q]; sb += sh[32 + q]; }
    a = sa;
    b = sb;
  }
}

// ---------------------------------------------------------------------------
// Persistent damped-Jacobi solve for all cases, one launch.
//   W phase k: every case that swept in F phase k-1 (or k = 0) extrapolates
//     its wall pressure from p^k (Eq. p-shepard, clamped at 0 for
//     free-surface flows); for a case that has just finished this is the
//     final wall update.  Skipped, with its barrier, when no case has walls.
//   F phase k: for every unfinished case
//       p^{k+1}_i = omega/D_ii (RHS_i + sum_j fac_ij p^k_j) + (1 - omega) p^k_i
//     with per-tile FP64 sums of |p^{k+1}-p^k| and |p^{k+1}|.  The block that
//     completes the last tile of a case (per-case arrival counter) adds that
//     case's tile sums in tile order -- the same order whoever arrives last --
//     and applies Eq. convergence: at least min_iter sweeps, at most max_iter.
//   grid barrier after each phase.
// p^k lives in buffer k&1.  Pressures written by other blocks are read with
// ordinary (L1-cached) loads: every grid barrier ends with an acquire fence
// in the block's master thread followed by a block barrier, which orders
// those reads after the other blocks' writes.  Flags and partial sums are
// read with ld.global.cg.
// ---------------------------------------------------------------------------
template <bool MX>
__global__ void __launch_bounds__(256, MX ? 8 : 4) k_sweeps(State S) {
  using R = typename std::conditional<MX, float, double>::type;
  __shared__ double sh[64];
  __shared__ int flag;
  const unsigned nb = gridDim.x;
  const int T = blockDim.x;
  const int nc = S.ncases;
  const R om1 = R(1.0 - S.omega);
  const R *coef = static_cast<const R *>(S.coef);
  const R *prhs = static_cast<const R *>(S.prhs);
  const R *pwd = static_cast<const R *>(S.pwd);
  const R *wc = static_cast<const R *>(S.wcoef);
  const R *wsinv = static_cast<const R *>(S.wsinv);
  const R *wh = static_cast<const R *>(S.wh);
  const long long n = S.n, nwl = S.nw;
  int *done = S.act;                 // [nc] case finished
  int *fin = S.act + nc;             // [nc] sweep count at which it finished
  unsigned *arrive = reinterpret_cast<unsigned *>(S.par + nc);  // [nc]
  bool skip = S.debug_skip_barrier && blockIdx.x == 1;
  bool alive = true;
  // hard bound on the loop: every case stops at its max_iter at the latest
  int kcap = 0;
  for (int c = 0; c < nc; ++c) kcap = max(kcap, S.cases[c].max_iter);
  int k = 0;
  for (;;) {
    const int cur = k & 1;
    R *pc = static_cast<R *>(S.pb[cur]);
    // ---- W phase: wall extrapolation from p^k ----
    if (S.nw > 0) {
      for (int r = blockIdx.x * T + threadIdx.x; r < S.nw; r += nb * T) {
        int w = S.wall_at[r];
        int c = S.case_of[w];
        if (k > 0 && __ldcg(done + c) && __ldcg(fin + c) != k) continue;
        R acc = wh[r];
        const int cnt = S.wcnt[r];
        for (int q0 = 0; q0 < cnt; q0 += 8) {
          int jj[8];
          R ww[8];
          _Pragma("unroll") for (int u = 0; u < 8; ++u) {
            const int q = q0 + u;
            const long long o = (long long)q * nwl + r;
            jj[u] = q < cnt ? S.widx[o] : w;
            ww[u] = q < cnt ? wc[o] : R(0);
          }
          R pv[8];
          _Pragma("unroll") for (int u = 0; u < 8; ++u) pv[u] = pc[jj[u]];
          _Pragma("unroll") for (int u = 0; u < 8; ++u) acc += ww[u] * pv[u];
        }
        R pw = acc * wsinv[r];
        if (S.cases[c].free_surface && pw < R(0)) pw = R(0);
        pc[w] = pw;
      }
      alive = grid_sync(S.bar, nb, S.barrier_budget, skip);
      skip = false;
      if (!alive) break;
    }
    // ---- any case left?  (a case without fluid has nothing to solve) ----
    int mine = 0;
    for (int c = threadIdx.x; c < nc; c += T) mine |= (__ldcg(done + c) == 0 && S.cases[c].nf > 0);
    if (!__syncthreads_or(mine)) break;
    if (k >= kcap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(S.err, kErrNotConv);
      break;
    }
    // ---- F phase: one damped-Jacobi sweep of the unfinished cases ----
    R *pn = static_cast<R *>(S.pb[cur ^ 1]);
    for (int tt = blockIdx.x; tt < S.nft; tt += nb) {
      const Tile &t = S.ftiles[tt];
      if (__ldcg(done + t.c)) continue;
      int i = t.beg + threadIdx.x;
      double dn = 0.0, dp = 0.0;
      R dnr = R(0), dpr = R(0);
      if (i < t.end) {
        R acc = prhs[i];
        const int cnt = S.ncnt[i];
        // chunks of 8 slots: 8 independent index/coefficient loads, then 8
        // independent gathers, so a row costs a few memory round trips
        for (int q0 = 0; q0 < cnt; q0 += 8) {
          unsigned e[8];
          R cf[8];
          _Pragma("unroll") for (int u = 0; u < 8; ++u) {
            const int q = q0 + u;
            const long long o = (long long)q * n + i;
            e[u] = q < cnt ? S.nbr[o] : unsigned(i);
            cf[u] = q < cnt ? coef[o] : R(0);
          }
          R pj[8];
          _Pragma("unroll") for (int u = 0; u < 8; ++u) pj[u] = pc[e[u] & kIdxMask];
          _Pragma("unroll") for (int u = 0; u < 8; ++u) acc += cf[u] * pj[u];
        }
        R po = pc[i];
        R pnew = pwd[i] * acc + om1 * po;
        pn[i] = pnew;
        dnr = fabs(pnew - po);
        dpr = fabs(pnew);
      }
      // tile sums in the sweep's precision (256 terms), the sum over tiles
      // and cases in FP64
      if constexpr (MX) {
        block_sum2f(dnr, dpr, sh);
        dn = double(dnr);
        dp = double(dpr);
      } else {
        dn = dnr;
        dp = dpr;
        block_sum2(dn, dp, sh);
      }
      if (threadIdx.x == 0) {
        S.tile_part[2 * tt] = dn;
        S.tile_part[2 * tt + 1] = dp;
        __threadfence();
        const CaseDev &P = S.cases[t.c];
        flag = (atomicAdd(arrive + t.c, 1u) == unsigned(P.nftile - 1));
      }
      __syncthreads();
      if (flag) {
        // last tile of this case: Eq. convergence over all of its tiles
        __threadfence();
        const int c = t.c;
        const CaseDev &P = S.cases[c];
        double num = 0.0, den = 0.0, lm = 0.0;
        for (int q = threadIdx.x; q < P.nftile; q += T) {
          num += __ldcg(S.tile_part + 2 * (P.ftile + q));
          den += __ldcg(S.tile_part + 2 * (P.ftile + q) + 1);
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
          arrive[c] = 0u;
          if (!go) {
            S.pstat[c] = st;
            S.par[c] = kk & 1;
            fin[c] = kk;
            __threadfence();
            done[c] = 1;
            if (st == SISPH_ENONFINITE) atomicOr(S.err, kErrNonFinite);
            if (st == SISPH_ENOTCONVERGED) atomicOr(S.err, kErrNotConv);
          }
        }
        __syncthreads();
      }
    }
    alive = grid_sync(S.bar, nb, S.barrier_budget, skip);
    skip = false;
    if (!alive) break;
    ++k;
  }
  if (!alive) return;
  // ---- publish the final pressure of every case ----
  for (int i = blockIdx.x * T + threadIdx.x; i < S.n; i += nb * T) {
    int c = S.case_of[i];
    R v = __ldcg(static_cast<const R *>(S.pb[__ldcg(S.par + c)]) + i);
    S.p[i] = double(v);
    if constexpr (MX) S.pf[i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int c = 0; c < nc; ++c) {
      S.iters_tot[c] += S.iters[c];
      S.solves[c] += 1;
    }
  }
}

cudaError_t launch_ppe_setup(const State &S, const Launch &L) {
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

int ppe_max_blocks_per_sm(const State &S, int block) {
  int nb = 0;
  if (S.mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweeps<true>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweeps<false>, block, 0);
  return nb;
}

cudaError_t launch_ppe_sweeps(const State &S, const Launch &L, int grid) {
  cudaMemsetAsync(S.bar, 0, sizeof(Barrier), L.stream);
  // done[nc], fin[nc] = 0; par[nc] and the arrival counters par[nc..2nc) = 0
  cudaMemsetAsync(S.act, 0, 2 * sizeof(int) * size_t(S.ncases), L.stream);
  cudaMemsetAsync(S.par, 0, 2 * sizeof(int) * size_t(S.ncases), L.stream);
  cudaMemsetAsync(S.iters, 0, sizeof(int) * size_t(S.ncases), L.stream);
  cudaMemsetAsync(S.pstat, 0, sizeof(int) * size_t(S.ncases), L.stream);
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
  if (S.mixed) e = cudaLaunchKernelEx(&cfg, k_sweeps<true>, S);
  else e = cudaLaunchKernelEx(&cfg, k_sweeps<false>, S);
  if (L.after) L.after(L.ctx, "ppe_sweeps", 0.0, 1);
  return e;
}

}  // namespace sisph
