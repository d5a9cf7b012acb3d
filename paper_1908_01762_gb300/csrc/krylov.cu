// BiCGStab (van der Vorst 1992) for the PPE: the Krylov alternative the paper
// mentions beside its damped Jacobi iterations (Sec. 3.1), on the same stored
// coefficients.  It solves the linear system the Jacobi sweeps converge to,
//   D_ii p_i - sum_j fac_ij p_j = RHS_i (active fluid i),  p_i = 0 (inactive),
// with each wall pressure replaced by its extrapolation (Eq. p-shepard),
//   p_w = (sum_f W_wf p_f + H_w) / S_w,
// whose affine part H_w / S_w moves to the right-hand side; the free-surface
// clamp p_w >= 0 is applied only in the final wall update.  Stopping rule:
// Eq. convergence on the update of each iteration (the Jacobi test), at least
// min_iter and at most max_iter iterations.  A case without a free-surface
// row has a singular system and is left to the Jacobi kernel.
//
// One persistent cooperative launch for all BiCGStab cases, phases separated
// by the bounded grid barrier:
//   init:  W: x_w = lin(x)            F: r = b - A x, r^ = r, rho = (r^, r)
//   iter:  F: p = r + beta (p - omega v)
//          W: p_w = lin(p)            F: v = A p,  alpha = rho / (r^, v)
//          W: s_w = lin(r - alpha v)  F: t = A s,  omega = (t, s) / (t, t)
//          F: x += alpha p + omega s, r = s - omega t, rho' = (r^, r), test
//   final: W: p_w from x with H_w and the clamp; publish.
// (lin: the linear part of the wall extrapolation; s = r - alpha v is formed
// where it is read.)  Dot products are per-tile FP64 sums added in tile order
// by the block that completes a case's last tile; vectors are in the sweep's
// precision (FP32 in the MIXED form).
#include "ppe_sync.cuh"

namespace sisph {

namespace {

// per-case scalars, kS doubles each
enum { kRho = 0, kRhoPrev, kAlpha, kOmega, kBeta, kPart0 };
constexpr int kS = 8;

__device__ __forceinline__ bool krylov_case(const State &S, int c) {
  return S.cases[c].solver == 1 && __ldcg(S.inact + c) > 0;
}

template <typename R>
struct Vecs {
  R *x, *r, *rh, *p, *v, *t, *sw;
};

template <typename R>
__device__ __forceinline__ Vecs<R> vecs(const State &S) {
  Vecs<R> V;
  V.x = static_cast<R *>(S.pb[0]);
  V.r = static_cast<R *>(S.kv[0]);
  V.rh = static_cast<R *>(S.kv[1]);
  V.p = static_cast<R *>(S.kv[2]);
  V.v = static_cast<R *>(S.kv[3]);
  V.t = static_cast<R *>(S.kv[4]);
  V.sw = static_cast<R *>(S.kv[5]);
  return V;
}

// Linear part of the wall extrapolation of a fluid vector (value of fluid j:
// a[j] - alpha * b[j] when b != null), for wall row r of wall w.
template <typename R>
__device__ __forceinline__ R wall_linear(const State &S, const R *a, const R *b, double alpha, int r, int w) {
  const R *wc = static_cast<const R *>(S.wcoef);
  const int cnt = S.wcnt[r];
  const R al = R(alpha);
  R acc = R(0);
  for (int q0 = 0; q0 < cnt; q0 += 8) {
    int jj[8];
    R ww[8];
    _Pragma("unroll") for (int u = 0; u < 8; ++u) {
      const int q = q0 + u;
      const long long o = ell_at(S.wcap, q, r);
      jj[u] = q < cnt ? S.widx[o] : w;
      ww[u] = q < cnt ? wc[o] : R(0);
      SISPH_CHECK_IDX(S, jj[u], w);
    }
    _Pragma("unroll") for (int u = 0; u < 8; ++u) {
      const R val = b ? a[jj[u]] - al * b[jj[u]] : a[jj[u]];
      acc += ww[u] * val;
    }
  }
  return acc * static_cast<const R *>(S.wsinv)[r];
}

// (A y)_i for fluid row i: D_ii y_i - sum_j fac_ij y_j on an active row, y_i
// on an inactive one.  The fluid values are a[j] - alpha b[j] (b != null) or
// a[j]; the wall values come from wv.  *bwall (when not null) receives
// sum_{walls j} fac_ij H_j / S_j, the affine part of the walls.
template <typename R>
__device__ __forceinline__ R apply_row(const State &S, const CaseDev &P, int i, bool active, const R *a,
                                       const R *b, double alpha, const R *wv, double *bwall) {
  const R al = R(alpha);
  const R yi = b ? a[i] - al * b[i] : a[i];
  if (!active) return yi;
  const long long sb = slot_base(S, i);
  const int cnt = S.pcnt[i];
  const int fend = P.fbeg + P.nf;
  R acc = R(S.diag_out[i]) * yi;
  double bw = 0.0;
  for (int q0 = 0; q0 < cnt; q0 += 8) {
    int jj[8];
    R cf[8];
    _Pragma("unroll") for (int u = 0; u < 8; ++u)
      load_coef<R>(S, sb, q0 + u, q0 + u < cnt, i, jj[u], cf[u]);
    _Pragma("unroll") for (int u = 0; u < 8; ++u) {
      const int j = jj[u];
      R yj;
      if (j >= fend) {
        yj = wv[j];
        if (bwall) {
          const int r = P.wrow + (j - P.wbeg);
          bw += double(cf[u]) * (double(static_cast<const R *>(S.wh)[r]) *
                                 double(static_cast<const R *>(S.wsinv)[r]));
        }
      } else {
        yj = b ? a[j] - al * b[j] : a[j];
      }
      acc -= cf[u] * yj;
    }
  }
  if (bwall) *bwall = bw;
  return acc;
}

}  // namespace

// Per-tile FP64 partial sums (up to 4 per tile) and the per-case reduction
// by the block that completes the case's last tile.  Returns, in every
// thread of that block, true; the sums (in tile order) are in out[0..nq).
__device__ __forceinline__ bool tile_reduce(const State &S, int tt, int c, int nq, double q[4], double *sh,
                                            int *flag, double out[4]) {
  // block sums of the nq quantities
  for (int a = 0; a < nq; a += 2) {
    double x = q[a], y = a + 1 < nq ? q[a + 1] : 0.0;
    block_sum2(x, y, sh);
    if (threadIdx.x == 0) {
      S.kpart[(size_t)4 * tt + a] = x;
      if (a + 1 < nq) S.kpart[(size_t)4 * tt + a + 1] = y;
    }
    __syncthreads();
  }
  unsigned *arrive = reinterpret_cast<unsigned *>(S.par + S.ncases);
  if (threadIdx.x == 0) {
    __threadfence();
    const CaseDev &P = S.cases[c];
    *flag = (atomicAdd(arrive + c, 1u) == unsigned(P.nftile - 1));
    if (*flag) arrive[c] = 0u;
  }
  __syncthreads();
  if (!*flag) return false;
  __threadfence();
  const CaseDev &P = S.cases[c];
  for (int a = 0; a < nq; a += 2) {
    double x = 0.0, y = 0.0;
    for (int k = threadIdx.x; k < P.nftile; k += blockDim.x) {
      x += __ldcg(S.kpart + (size_t)4 * (P.ftile + k) + a);
      if (a + 1 < nq) y += __ldcg(S.kpart + (size_t)4 * (P.ftile + k) + a + 1);
    }
    block_sum2(x, y, sh);
    if (threadIdx.x == 0) {
      out[a] = x;
      if (a + 1 < nq) out[a + 1] = y;
    }
    __syncthreads();
  }
  return true;
}

template <bool MX>
__global__ void __launch_bounds__(256, MX ? 4 : 3) k_bicgstab(State S) {
  using R = typename std::conditional<MX, float, double>::type;
  __shared__ double sh[64];
  __shared__ int flag;
  __shared__ int apre[kBalCases + 1];
  __shared__ int wsum[33];
  const unsigned nb = gridDim.x;
  const int T = blockDim.x;
  const int nc = S.ncases;
  int *done = S.act;                 // [nc] case finished
  int *fin = S.act + nc;             // [nc] iterations at which it finished
  double *ks = S.kscal;              // [nc][kS]
  const Vecs<R> V = vecs<R>(S);
  bool alive = true;
  // the work of the BiCGStab cases still iterating.  fin[c] is 0 while a
  // case iterates and it + 2 once it stopped during iteration it (it = -1:
  // the initial phase), so every block, whenever it looks during iteration
  // k, counts the same cases.
  auto running = [&](int c, int k) {
    if (!krylov_case(S, c)) return false;
    const int f = __ldcg(fin + c);
    return f == 0 || f > k + 1;
  };
  // ---- W phase helper: wall values of a vector for the cases in `sel` ----
  auto wall_phase = [&](auto sel, auto value) {
    const int nrows = case_prefix(nc, apre, wsum, [&](int c) { return sel(c) ? S.cases[c].nw : 0; });
    for (int a = blockIdx.x * T + threadIdx.x; a < nrows; a += nb * T) {
      const int c = case_of_index(apre, nc, a);
      const CaseDev &P = S.cases[c];
      const int r = P.wrow + (a - apre[c]);
      value(r, S.wall_at[r], c);
    }
    return grid_sync(S.bar, nb, S.barrier_budget, false);
  };
  // ---- F phase helper: fluid tiles of the cases in `sel` ----
  auto tiles = [&](auto sel, auto body) {
    const int ntiles = case_prefix(nc, apre, wsum, [&](int c) { return sel(c) ? S.cases[c].nftile : 0; });
    for (int a = blockIdx.x; a < ntiles; a += nb) {
      const int c = case_of_index(apre, nc, a);
      body(S.cases[c].ftile + (a - apre[c]), c);
    }
    return grid_sync(S.bar, nb, S.barrier_budget, false);
  };
  const R *pwd = static_cast<const R *>(S.pwd);
  const R *prhs = static_cast<const R *>(S.prhs);
  // thread 0 of the deciding block; `it` the current iteration (-1 initial)
  auto decide = [&](int c, int it, int kk, double res, int st, bool stop) {
    // thread 0 of the deciding block
    S.iters[c] = kk;
    S.resid[c] = res;
    if (stop) {
      S.pstat[c] = st;
      S.par[c] = 0;
      S.iters_tot[c] += kk;
      S.solves[c] += 1;
      if (st == SISPH_ENONFINITE) atomicOr(S.err, kErrNonFinite);
      if (st == SISPH_ENOTCONVERGED) atomicOr(S.err, kErrNotConv);
      fin[c] = it + 2;
      __threadfence();
      done[c] = 1;
    }
  };

  // ---- init: x_w = lin(x); r = b - A x; r^ = r; p = v = 0; rho = (r, r) ----
  alive = wall_phase([&](int c) { return krylov_case(S, c); },
                     [&](int r, int w, int c) { V.x[w] = wall_linear<R>(S, V.x, nullptr, 0.0, r, w); });
  if (alive) alive = tiles([&](int c) { return krylov_case(S, c); }, [&](int tt, int c) {
    const Tile &t = S.ftiles[tt];
    const CaseDev &P = S.cases[c];
    const int i = t.beg + threadIdx.x;
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < t.end) {
      const bool act = pwd[i] != R(0);
      double bw = 0.0;
      const R ax = apply_row<R>(S, P, i, act, V.x, nullptr, 0.0, V.x, &bw);
      const R b = act ? R(double(prhs[i]) + bw) : R(0);
      const R r = b - ax;
      V.r[i] = r;
      V.rh[i] = r;
      V.p[i] = R(0);
      V.v[i] = R(0);
      q[0] = double(r) * double(r);
    }
    double out[4];
    if (tile_reduce(S, tt, c, 1, q, sh, &flag, out)) {
      // Lambda = max_i |RHS_i / D_ii| of Eq. convergence, over the case's tiles
      double lm = 0.0;
      for (int q2 = threadIdx.x; q2 < P.nftile; q2 += T) lm = fmax(lm, __ldcg(S.tile_lam + P.ftile + q2));
      for (int o = 16; o > 0; o >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lm;
      __syncthreads();
      if (threadIdx.x == 0) {
        double m = sh[0];
        for (int w = 1; w < (T >> 5); ++w) m = fmax(m, sh[w]);
        S.lam[c] = m;
        ks[kS * c + kRho] = out[0];
        ks[kS * c + kRhoPrev] = 1.0;
        ks[kS * c + kAlpha] = 1.0;
        ks[kS * c + kOmega] = 1.0;
        if (out[0] == 0.0) decide(c, -1, 0, 0.0, SISPH_OK, true);     // x0 solves it
        else if (!isfinite(out[0])) decide(c, -1, 0, out[0], SISPH_ENONFINITE, true);
        else ks[kS * c + kBeta] = out[0];                             // p = r (p = v = 0)
      }
    }
    __syncthreads();
  });

  int k = 0;
  while (alive) {
    // any BiCGStab case left?
    int mine = 0;
    for (int c = threadIdx.x; c < nc; c += T) mine |= running(c, k) ? 1 : 0;
    if (!__syncthreads_or(mine)) break;
    auto run_k = [&](int c) { return running(c, k); };
    // ---- p = r + beta (p - omega v) ----
    alive = tiles(run_k, [&](int tt, int c) {
      const Tile &t = S.ftiles[tt];
      const int i = t.beg + threadIdx.x;
      if (i < t.end) {
        const R beta = R(ks[kS * c + kBeta]), om = R(ks[kS * c + kOmega]);
        V.p[i] = V.r[i] + beta * (V.p[i] - om * V.v[i]);
      }
    });
    if (!alive) break;
    // ---- p_w = lin(p); v = A p; alpha = rho / (r^, v) ----
    if (S.nw > 0) {
      alive = wall_phase(run_k, [&](int r, int w, int c) { V.p[w] = wall_linear<R>(S, V.p, nullptr, 0.0, r, w); });
      if (!alive) break;
    }
    alive = tiles(run_k, [&](int tt, int c) {
      const Tile &t = S.ftiles[tt];
      const CaseDev &P = S.cases[c];
      const int i = t.beg + threadIdx.x;
      double q[4] = {0.0, 0.0, 0.0, 0.0};
      if (i < t.end) {
        const R v = apply_row<R>(S, P, i, pwd[i] != R(0), V.p, nullptr, 0.0, V.p, nullptr);
        V.v[i] = v;
        q[0] = double(V.rh[i]) * double(v);
      }
      double out[4];
      if (tile_reduce(S, tt, c, 1, q, sh, &flag, out) && threadIdx.x == 0) {
        if (out[0] == 0.0 || !isfinite(out[0]))          // breakdown: stop with x
          decide(c, k, k, k ? __ldcg(S.resid + c) : 0.0,
                 isfinite(out[0]) ? SISPH_ENOTCONVERGED : SISPH_ENONFINITE, true);
        else
          ks[kS * c + kAlpha] = ks[kS * c + kRho] / out[0];
      }
      __syncthreads();
    });
    if (!alive) break;
    // ---- s = r - alpha v (formed where read); s_w = lin(s); t = A s ----
    if (S.nw > 0) {
      alive = wall_phase(run_k, [&](int r, int w, int c) {
        if (!__ldcg(done + c)) V.sw[w] = wall_linear<R>(S, V.r, V.v, ks[kS * c + kAlpha], r, w);
      });
      if (!alive) break;
    }
    alive = tiles(run_k, [&](int tt, int c) {
      if (__ldcg(done + c)) return;          // stopped at a breakdown this iteration
      const Tile &t = S.ftiles[tt];
      const CaseDev &P = S.cases[c];
      const int i = t.beg + threadIdx.x;
      const double al = ks[kS * c + kAlpha];
      double q[4] = {0.0, 0.0, 0.0, 0.0};
      if (i < t.end) {
        const R tv = apply_row<R>(S, P, i, pwd[i] != R(0), V.r, V.v, al, V.sw, nullptr);
        V.t[i] = tv;
        const R s = V.r[i] - R(al) * V.v[i];
        q[0] = double(tv) * double(s);
        q[1] = double(tv) * double(tv);
      }
      double out[4];
      if (tile_reduce(S, tt, c, 2, q, sh, &flag, out) && threadIdx.x == 0)
        ks[kS * c + kOmega] = out[1] > 0.0 ? out[0] / out[1] : 0.0;
      __syncthreads();
    });
    if (!alive) break;
    // ---- x += alpha p + omega s; r = s - omega t; rho' = (r^, r); test ----
    alive = tiles(run_k, [&](int tt, int c) {
      if (__ldcg(done + c)) return;
      const Tile &t = S.ftiles[tt];
      const int i = t.beg + threadIdx.x;
      const R al = R(ks[kS * c + kAlpha]), om = R(ks[kS * c + kOmega]);
      double q[4] = {0.0, 0.0, 0.0, 0.0};
      if (i < t.end) {
        const R s = V.r[i] - al * V.v[i];
        const R dx = al * V.p[i] + om * s;
        const R xn = V.x[i] + dx;
        V.x[i] = xn;
        const R r = s - om * V.t[i];
        V.r[i] = r;
        q[0] = double(V.rh[i]) * double(r);
        q[1] = double(r) * double(r);
        q[2] = fabs(double(dx));
        q[3] = fabs(double(xn));
      }
      double out[4];
      if (tile_reduce(S, tt, c, 4, q, sh, &flag, out) && threadIdx.x == 0) {
        const CaseDev &P = S.cases[c];
        const int kk = k + 1;
        const double lamc = S.lam[c];
        const double lam = S.residual_form == 1 ? double(P.nf) * lamc : lamc;
        const double dd = lam > out[3] ? lam : out[3];
        const double res = dd > 0.0 ? out[2] / dd : out[2];
        if (!isfinite(res)) decide(c, k, kk, res, SISPH_ENONFINITE, true);
        else if (kk >= S.min_iter && res < P.tol) decide(c, k, kk, res, SISPH_OK, true);
        else if (kk >= P.max_iter) decide(c, k, kk, res, SISPH_ENOTCONVERGED, true);
        else if (out[0] == 0.0)        // next rho vanishes: solved exactly, or a breakdown
          decide(c, k, kk, out[1] == 0.0 ? 0.0 : res, out[1] == 0.0 ? SISPH_OK : SISPH_ENOTCONVERGED, true);
        else {
          const double rho = ks[kS * c + kRho];
          ks[kS * c + kBeta] = (out[0] / rho) * (ks[kS * c + kAlpha] / ks[kS * c + kOmega]);
          ks[kS * c + kRhoPrev] = rho;
          ks[kS * c + kRho] = out[0];
          decide(c, k, kk, res, SISPH_OK, false);
        }
      }
      __syncthreads();
    });
    ++k;
  }
  if (!alive) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(S.err, kErrTimeout);
    return;
  }
  // ---- final wall update from x (with H_w and the clamp); publish ----
  alive = wall_phase([&](int c) { return krylov_case(S, c); },
                     [&](int r, int w, int c) { V.x[w] = wall_pressure<R>(S, V.x, r, w, c); });
  if (!alive) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(S.err, kErrTimeout);
    return;
  }
  for (int i = blockIdx.x * T + threadIdx.x; i < S.n; i += nb * T) {
    const int c = S.case_of[i];
    if (!krylov_case(S, c)) continue;
    const R v = __ldcg(V.x + i);
    S.p[i] = double(v);
    if constexpr (MX) S.pf[i] = v;
  }
}

int krylov_max_blocks_per_sm(const State &S, int block) {
  int nb = 0;
  if (S.mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab<true>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bicgstab<false>, block, 0);
  return nb;
}

cudaError_t launch_ppe_krylov(const State &S, const Launch &L, int grid) {
  cudaMemsetAsync(S.bar, 0, sizeof(Barrier), L.stream);
  if (L.before) L.before(L.ctx, "ppe_krylov");
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
  if (S.mixed) e = cudaLaunchKernelEx(&cfg, k_bicgstab<true>, S);
  else e = cudaLaunchKernelEx(&cfg, k_bicgstab<false>, S);
  if (L.after) L.after(L.ctx, "ppe_krylov", 0.0, 1);
  return e;
}

}  // namespace sisph
