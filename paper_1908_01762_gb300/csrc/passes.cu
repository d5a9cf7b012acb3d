// Neighbour passes of one SISPH time step (Algorithm 1) other than the PPE.
// One thread per particle, one thread block per tile; every pass reads its
// neighbours from the ELL lists built by nbr.cu.  Template parameter MX
// selects the MIXED form: FP32 sums over FP32 cell-relative positions, with
// the FP64 master state updated in FP64.
#include <math_constants.h>

#include "sisph_internal.h"

namespace sisph {

template <int DIM, bool MX>
struct Geo {
  using R = typename std::conditional<MX, float, double>::type;
  double xi[3];
  float4 pi;
  __device__ __forceinline__ void init(const State &S, int i) {
    if constexpr (MX) {
      pi = S.pf4[i];
    } else {
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) xi[k] = S.x[k][i];
    }
  }
  __device__ __forceinline__ R pair(const State &S, const CaseDev &P, const float lc[3], unsigned e,
                                    int &j, R d[3]) const {
    j = int(e & kIdxMask);
    if constexpr (MX) {
      float4 pj = S.pf4[j];
      return pair_f<DIM>(lc, pi, pj, e >> kCodeShift, d);
    } else {
      double dd[3];
      double r2 = pair_d<DIM>(P, xi, S.x, j, dd);
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) d[k] = dd[k];
      if (DIM == 2) d[2] = 0.0;
      return r2;
    }
  }
};

template <bool MX>
__device__ __forceinline__ auto mass(const State &S, int j) {
  if constexpr (MX) return fabsf(S.pf4[j].w);    // the sign holds the near-range test
  else return S.m[j];
}
template <bool MX>
__device__ __forceinline__ auto dens(const State &S, int j) {
  if constexpr (MX) return S.vf4[j].w;
  else return S.rho[j];
}
template <int DIM, bool MX, typename R>
__device__ __forceinline__ void vel(const State &S, int j, R u[3]) {
  if constexpr (MX) {
    float4 v = S.vf4[j];
    u[0] = v.x; u[1] = v.y; u[2] = v.z;
  } else {
    u[0] = S.u[0][j]; u[1] = S.u[1][j]; u[2] = DIM == 3 ? S.u[2][j] : 0.0;
  }
}
template <int DIM, bool MX, typename R>
__device__ __forceinline__ void tvel(const State &S, int j, R u[3]) {
  if constexpr (MX) {
    float4 v = S.utf4[j];
    u[0] = v.x; u[1] = v.y; u[2] = v.z;
  } else {
    u[0] = S.ut[0][j]; u[1] = S.ut[1][j]; u[2] = DIM == 3 ? S.ut[2][j] : 0.0;
  }
}

#define ROW_LOOP(S, i, ...) ROW_LOOP_FROM(S, i, 0, __VA_ARGS__)
#define ROW_LOOP_FROM(S, i, k0, ...)                          \
  {                                                            \
    const int _cnt = S.ncnt[i];                                \
    const long long _b = ell_base(S.cap, i);                   \
    _Pragma("unroll 4")                                        \
    for (int _k = (k0); _k < _cnt; ++_k) {                     \
      unsigned e = S.nbr[_b + (long long)_k * kEllBlock];      \
      SISPH_CHECK_ENTRY(S, e, unsigned(i));                    \
      __VA_ARGS__                                              \
    }                                                          \
  }

// ---------------------------------------------------------------------------
// Summation density, Eq. summation_density, for fluid particles.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void __launch_bounds__(256, MX ? 6 : 3) k_density(State S) {
  using R = typename Geo<DIM, MX>::R;
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  KC<R> K;
  K.set(P, P.h, P.inv_h, P.sig_h);
  Geo<DIM, MX> G;
  G.init(S, i);
  R acc = R(0);
  ROW_CHUNKS(S, i, {
    int j;
    R d[3];
    R r2 = G.pair(S, P, K.lc, e, j, d);
    R w = mass<MX>(S, j) * poly_w<R>(qof<R>(sqrt_x(r2), K.h, K.ih));
    acc += valid ? w : R(0);
  })
  acc *= K.sig;
  S.rho[i] = double(acc);
  if constexpr (MX) S.vf4[i].w = float(acc);
}

// ---------------------------------------------------------------------------
// Wall normals, Sec. 3.4.1 (computed once; walls never move), FP64:
//   n*_i = -sum_j (m_j/rho_j) grad W_ij over wall neighbours, zero if
//   |n*| < 1/(4h) else unit; n_i = sum_j (m_j/rho_j) n*_j W_ij, unit, or zero
//   when shorter than 1e-6 (a cancelled average of unit vectors).
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_normals(State S, int pass) {
  const Tile &t = S.wtiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  double xi[3] = {S.x[0][i], S.x[1][i], DIM == 3 ? S.x[2][i] : 0.0};
  double acc[3] = {0, 0, 0};
  const int wend = P.wbeg + P.nw;
  ROW_LOOP(S, i, {
    int j = int(e & kIdxMask);
    if (j >= P.wbeg && j < wend) {
      double d[3] = {0, 0, 0};
      double r2 = pair_d<DIM>(P, xi, S.x, j, d);
      double r = sqrt(r2);
      double vj = S.m[j] / S.rho[j];
      if (pass == 0) {
        double fr = r > 0.0 ? P.sig_h * P.inv_h * poly_dw<double>(r / P.h) / r : 0.0;
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) acc[k] -= vj * fr * d[k];
      } else {
        double w = vj * P.sig_h * poly_w<double>(r / P.h);
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) acc[k] += w * S.nstar[k][j];
      }
    }
  })
  double mag = sqrt(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
  double thr = pass == 0 ? 1.0 / (4.0 * P.h) : 1e-6;
  bool keep = pass == 0 ? !(mag < thr) : (mag > thr);
  _Pragma("unroll") for (int k = 0; k < 3; ++k) {
    double v = keep ? acc[k] / mag : 0.0;
    if (pass == 0) S.nstar[k][i] = v;
    else S.nrm[k][i] = v;
  }
}

// ---------------------------------------------------------------------------
// Wall ghost velocity, Sec. 3.4, Eqs. vf, vg-adami, vg-no-normal.
//  no-slip (stage 1): u~ = Shepard(u_f, h/2), u_w = 2 u_wall - u~, and the
//    component into the solid removed;  u~ = u_wall without fluid in range.
//  slip (stage 2, u* of the PPE source): u_w = Shepard(u*_f, h), the fluid's
//    own u* extended into the wall (u_wall without fluid in range).
// The result is written into the wall's velocity slot.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void k_ghost(State S, int slip_stage) {
  using R = typename Geo<DIM, MX>::R;
  const Tile &t = S.wtiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  const bool slip = slip_stage && P.ustar_slip;
  KC<R> K;
  if (slip) K.set(P, P.h, P.inv_h, P.sig_h);
  else K.set(P, P.h2, P.inv_h2, P.sig_h2);
  Geo<DIM, MX> G;
  G.init(S, i);
  R sw = R(0), su[3] = {R(0), R(0), R(0)};
  const int fend = P.fbeg + P.nf;
  // fluid neighbours only: they follow the row's wall head
  ROW_LOOP_FROM(S, i, S.wfin[i], {
    int j = int(e & kIdxMask);
    if (j < fend) {
      R d[3];
      R r2 = G.pair(S, P, K.lc, e, j, d);
      R w = poly_w<R>(qof<R>(sqrt_r(r2), K.h, K.ih));
      R uj[3];
      vel<DIM, MX>(S, j, uj);
      sw += w;
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) su[k] += uj[k] * w;
    }
  })
  double ug[3] = {0, 0, 0}, nn[3] = {0, 0, 0}, ut[3];
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    ut[k] = sw > R(0) ? double(su[k]) / double(sw) : S.uw[k][i];
    nn[k] = S.nrm[k][i];
  }
  if (slip) {
    _Pragma("unroll") for (int k = 0; k < DIM; ++k) ug[k] = ut[k];
  } else {
    _Pragma("unroll") for (int k = 0; k < DIM; ++k) ug[k] = 2.0 * S.uw[k][i] - ut[k];
    double un = ug[0] * nn[0] + ug[1] * nn[1] + ug[2] * nn[2];
    if (un < 0.0) {
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) ug[k] -= un * nn[k];
    }
  }
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) S.u[k][i] = ug[k];
  if constexpr (MX) {
    float4 v = S.vf4[i];
    v.x = float(ug[0]); v.y = float(ug[1]); v.z = float(ug[2]);
    S.vf4[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Stage 1, Eqs. int:rnp1 and int:vint:  r* = r^n + dt u~^n,
// u* = u^n + dt (f_visc + f_avisc + f_astress + g) with
//   f_visc   = sum_j m_j 4 nu/(rho_i+rho_j) (r_ij.gradW)/(r^2+eta h^2) u_ij
//   f_avisc  = -sum_j m_j Pi_ij gradW, Pi_ij = -alpha h c phi_ij/rho_bar for
//              u_ij.r_ij < 0, phi_ij = u_ij.r_ij/(r^2+eta h^2)
//   f_astress= sum_{j fluid} m_j (A_i/rho_i^2 + A_j/rho_j^2).gradW,
//              A = rho u (x) (u~ - u)
// Walls enter with their ghost velocity.  Writes r*, u* to the stage-1
// buffers (neighbours still read r^n, u^n).
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void k_stage1(State S) {
  using R = typename Geo<DIM, MX>::R;
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  KC<R> K;
  K.set(P, P.h, P.inv_h, P.sig_h);
  Geo<DIM, MX> G;
  G.init(S, i);
  const R nu4 = R(4.0 * P.nu), eh2 = R(P.eh2);
  const R avc = R(2.0 * P.alpha * P.h * P.c0);     // 2 alpha h c
  const int fend = P.fbeg + P.nf;
  R ui[3], uti[3];
  vel<DIM, MX>(S, i, ui);
  tvel<DIM, MX>(S, i, uti);
  const R ri = dens<MX>(S, i);
  const R iri = R(1) / ri;
  R dti[3];
  _Pragma("unroll") for (int k = 0; k < 3; ++k) dti[k] = uti[k] - ui[k];
  R f[3] = {R(0), R(0), R(0)};
  // the row loop is compiled with and without the artificial viscosity (a
  // per-case choice), so that neither carries the other's branch
  auto rows = [&](auto with_av) {
  constexpr bool av = decltype(with_av)::value;
  ROW_CHUNKS(S, i, {
    int j;
    R d[3];
    R r2 = G.pair(S, P, K.lc, e, j, d);
    // 3D: every slot runs the pair arithmetic and its contribution is masked
    // (the row itself and the padding add 0), without a branch; 2D rows keep
    // the branches, which measured faster there
    const bool on = valid && j != i;
    if (DIM == 3 || on) {
      R r = sqrt_r(r2);
      R dw = K.dsc * poly_dw<R>(qof<R>(r, K.h, K.ih));
      R fr = r > R(0) ? divr(dw, r) : R(0);
      R rj = dens<MX>(S, j), mj = mass<MX>(S, j);
      R uj[3];
      vel<DIM, MX>(S, j, uj);
      R uij[3] = {ui[0] - uj[0], ui[1] - uj[1], ui[2] - uj[2]};
      R rsum = ri + rj, reta = r2 + eh2;
      R visc = divr(mj * nu4 * fr * r2, rsum * reta);
      R coef = R(0);
      if (av) {
        R vr = uij[0] * d[0] + uij[1] * d[1] + (DIM == 3 ? uij[2] * d[2] : R(0));
        // -m_j Pi_ij = m_j alpha h c phi_ij / ((rho_i + rho_j)/2)
        if constexpr (DIM == 3) coef = vr < R(0) ? divr(mj * avc * vr, reta * rsum) : R(0);
        else if (vr < R(0)) coef = divr(mj * avc * vr, reta * rsum);
      }
      R ai = R(0), aj = R(0);
      if constexpr (DIM == 3) {
        // the transport-velocity terms of fluid neighbours, masked for walls
        const bool fl = j < fend;
        R utj[3];
        tvel<DIM, MX>(S, j, utj);
        R gi = R(0), gj = R(0);
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
          gi += dti[k] * d[k];
          gj += (utj[k] - uj[k]) * d[k];
        }
        ai = fl ? mj * fr * gi * iri : R(0);
        aj = fl ? divr(mj * fr * gj, rj) : R(0);
      } else if (j < fend) {
        R utj[3];
        tvel<DIM, MX>(S, j, utj);
        R gi = R(0), gj = R(0);
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
          gi += dti[k] * d[k];
          gj += (utj[k] - uj[k]) * d[k];
        }
        ai = mj * fr * gi * iri;
        aj = divr(mj * fr * gj, rj);
      }
      _Pragma("unroll") for (int k = 0; k < DIM; ++k)
        f[k] += on ? visc * uij[k] + coef * fr * d[k] + ui[k] * ai + uj[k] * aj : R(0);
    }
  })
  };
  if (P.alpha > 0.0) rows(std::true_type{});
  else rows(std::false_type{});
  const double dt = P.dt;
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    double fk = double(f[k]) + P.g[k];
    if (P.adaptive) S.fs1[k][i] = fk;
    S.us[k][i] = S.u[k][i] + dt * fk;
    double xk = __dadd_rn(S.x[k][i], __dmul_rn(dt, S.ut[k][i]));
    if (P.per[k]) {
      if (xk >= P.hi[k]) xk -= P.L[k];
      else if (xk < P.lo[k]) xk += P.L[k];
    }
    S.xs[k][i] = xk;
  }
}

// Walls do not move: their stage-1 outputs are their current state.
template <int DIM>
__global__ void k_stage1_walls(State S) {
  const Tile &t = S.wtiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
_Pragma("unroll")
  for (int k = 0; k < DIM; ++k) {
    S.xs[k][i] = S.x[k][i];
    S.us[k][i] = S.u[k][i];
  }
}

// ---------------------------------------------------------------------------
// Pressure gradient and correction, Eqs. mom:sph:press:symm / :pij, int:vnp1:
//   symm : f_p = -sum_j m_j (p_i/rho_i^2 + p_j/rho_j^2) gradW
//   asymm: f_p = -sum_j m_j/(rho_i rho_j) (p_j - p_i) gradW
//   u^{n+1} = u* + dt f_p
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void k_pgrad(State S) {
  using R = typename Geo<DIM, MX>::R;
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  KC<R> K;
  K.set(P, P.h, P.inv_h, P.sig_h);
  Geo<DIM, MX> G;
  G.init(S, i);
  const R ri = dens<MX>(S, i);
  R pi;
  if constexpr (MX) pi = S.pf[i];
  else pi = S.p[i];
  const R pri = divr(pi, ri * ri);
  const R iri = R(1) / ri;
  R f[3] = {R(0), R(0), R(0)};
  const bool symm = P.pgrad_symm != 0;
  ROW_LOOP(S, i, {
    int j;
    R d[3];
    R r2 = G.pair(S, P, K.lc, e, j, d);
    if (j != i) {
      R r = sqrt_r(r2);
      R fr = r > R(0) ? divr(K.dsc * poly_dw<R>(qof<R>(r, K.h, K.ih)), r) : R(0);
      R rj = dens<MX>(S, j), mj = mass<MX>(S, j);
      R pj;
      if constexpr (MX) pj = S.pf[j];
      else pj = S.p[j];
      R c = symm ? -mj * (pri + divr(pj, rj * rj)) : -divr(mj * (pj - pi), rj) * iri;
      c *= fr;
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) f[k] += c * d[k];
    }
  })
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    S.u[k][i] = S.u[k][i] + P.dt * double(f[k]);
    if (P.adaptive) S.fs1[k][i] += double(f[k]);     // total acceleration
  }
}

// p_ref = 2 max_i p_i after the first PPE solve (internal flows, Sec. 2.1);
// one block per case, only while the case's flag is unset.
__global__ void k_pref(State S) {
  int c = blockIdx.x;
  const CaseDev &P = S.cases[c];
  if (P.pref_mode != SISPH_PREF_TWICE_MAX_FIRST || S.pref_set[c]) return;
  double mx = -1e300;
  for (int i = P.fbeg + threadIdx.x; i < P.fbeg + P.nf; i += blockDim.x) mx = fmax(mx, S.p[i]);
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sh[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    S.pref[c] = P.nf > 0 ? 2.0 * m : 0.0;
    S.pref_set[c] = 1;
  }
}

// ---------------------------------------------------------------------------
// GTVF homogenisation, Eqs. mom:sph:gtvf, int:gtvf:pos, int:gtvf:vel:tmp:
//   f_i = -p0_i sum_j (m_j/rho_j^2) grad W(r_ij, h~), on the r* lists with
//   distances from the sub-step positions (r* + d), d^0 = 0, u~^0 = 0;
//   d^k = d^{k-1} + dtau u~^{k-1} + dtau^2/2 f,  u~^k = u~^{k-1} + dtau f.
//   p0_i = p_ref, or min(10|p_i|, p_ref) for external flows.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void k_gtvf(State S, int sub, int cur, int skip_k1) {
  using R = typename Geo<DIM, MX>::R;
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  if (sub >= P.K || (skip_k1 && P.K == 1)) return;
  KC<R> K;
  K.set(P, P.hg, P.inv_hg, P.sig_hg);
  Geo<DIM, MX> G;
  G.init(S, i);
  const int fend = P.fbeg + P.nf;
  R di[3] = {R(0), R(0), R(0)};
  if (sub > 0) {
    if constexpr (MX) {
      float4 v = S.dgf[cur][i];
      di[0] = v.x; di[1] = v.y; di[2] = v.z;
    } else {
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) di[k] = S.dg[cur][k][i];
    }
  }
  R acc[3] = {R(0), R(0), R(0)};
  ROW_LOOP(S, i, {
    int j;
    R d[3];
    G.pair(S, P, K.lc, e, j, d);
    if (j != i) {
      if (sub > 0 && j < fend) {
        R dj[3];
        if constexpr (MX) {
          float4 v = S.dgf[cur][j];
          dj[0] = v.x; dj[1] = v.y; dj[2] = v.z;
        } else {
          _Pragma("unroll") for (int k = 0; k < DIM; ++k) dj[k] = S.dg[cur][k][j];
        }
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) d[k] += di[k] - dj[k];
      }
      R r2 = d[0] * d[0] + d[1] * d[1] + (DIM == 3 ? d[2] * d[2] : R(0));
      R r = sqrt_r(r2);
      if (r > R(0)) {
        R fr = divr(K.dsc * poly_dw<R>(qof<R>(r, K.h, K.ih)), r);
        R rj = dens<MX>(S, j);
        R c = divr(mass<MX>(S, j), rj * rj) * fr;
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) acc[k] += c * d[k];
      }
    }
  })
  double pref = S.pref[t.c];
  double pi = S.p[i];
  double p0 = P.pref_mode == SISPH_PREF_EXTERNAL ? fmin(10.0 * fabs(pi), pref) : pref;
  const double dtau = P.dt / P.K;
  const int nxt = cur ^ 1;
  double dn[3] = {0, 0, 0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    double fk = -p0 * double(acc[k]);
    double vk = sub > 0 ? S.vgt[k][i] : 0.0;
    double dk = sub > 0 ? double(di[k]) : 0.0;
    dn[k] = dk + dtau * vk + 0.5 * dtau * dtau * fk;
    S.vgt[k][i] = vk + dtau * fk;
    if constexpr (!MX) S.dg[nxt][k][i] = dn[k];
  }
  if constexpr (MX) S.dgf[nxt][i] = make_float4(float(dn[0]), float(dn[1]), float(dn[2]), 0.f);
}

// ---------------------------------------------------------------------------
// MIXED form, one pass over the r* lists for a case with one GTVF sub-step:
// pressure gradient and correction (Eq. int:vnp1), the GTVF force at r*
// (Eq. mom:sph:gtvf) and, with K = 1, d = dt^2/2 f (Eq. int:gtvf:pos),
// then the transport velocity and position update (Eqs. int:vhatnp2,
// int:rnp2).  Neighbours are read only through the FP32 mirrors (positions,
// mass, density, pressure), which this pass does not write, so the in-place
// FP64 updates of u, u~ and r cannot race.  A tile of a case with K > 1 only
// takes the pressure gradient here; its GTVF and update run as separate passes.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256, 5) k_pgrad_gtvf1(State S) {
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  const bool fused = P.K == 1;
  KC<float> K, KG;
  K.set(P, P.h, P.inv_h, P.sig_h);
  KG.set(P, P.hg, P.inv_hg, P.sig_hg);
  const float4 pi4 = S.pf4[i];
  const float ri = S.vf4[i].w;
  const float pi = S.pf[i];
  const float pri = divr(pi, ri * ri);
  const float iri = 1.f / ri;
  float f[3] = {0.f, 0.f, 0.f}, acc[3] = {0.f, 0.f, 0.f};
  // the row loop is compiled for each gradient form and with or without the
  // GTVF sum (per-case choices), so that no pair carries their branches
  auto rows = [&](auto symm_form, auto with_gtvf) {
  constexpr bool symm = decltype(symm_form)::value, fused = decltype(with_gtvf)::value;
  ROW_CHUNKS(S, i, {
    const int j = int(e & kIdxMask);
    if (valid && j != i) {
      float4 pj4 = S.pf4[j];
      float d[3];
      float r2 = pair_f<DIM>(K.lc, pi4, pj4, e >> kCodeShift, d);
      float r = sqrt_r(r2);
      float rj = S.vf4[j].w, mj = fabsf(pj4.w), pj = S.pf[j];
      float fr = r > 0.f ? divr(K.dsc * poly_dw<float>(qof<float>(r, K.h, K.ih)), r) : 0.f;
      float c = symm ? -mj * (pri + divr(pj, rj * rj)) : -divr(mj * (pj - pi), rj) * iri;
      c *= fr;
      _Pragma("unroll") for (int k = 0; k < DIM; ++k) f[k] += c * d[k];
      if (fused && r > 0.f) {
        float frg = divr(KG.dsc * poly_dw<float>(qof<float>(r, KG.h, KG.ih)), r);
        float cg = divr(mj, rj * rj) * frg;
        _Pragma("unroll") for (int k = 0; k < DIM; ++k) acc[k] += cg * d[k];
      }
    }
  })
  };
  if (P.pgrad_symm != 0) {
    if (fused) rows(std::true_type{}, std::true_type{});
    else rows(std::true_type{}, std::false_type{});
  } else {
    if (fused) rows(std::false_type{}, std::true_type{});
    else rows(std::false_type{}, std::false_type{});
  }
  const double dt = P.dt;
  double unew[3] = {0, 0, 0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    unew[k] = S.u[k][i] + dt * double(f[k]);
    S.u[k][i] = unew[k];
    if (P.adaptive) S.fs1[k][i] += double(f[k]);     // total acceleration
  }
  if (!fused) return;
  const double pref = S.pref[t.c];
  const double p0 = P.pref_mode == SISPH_PREF_EXTERNAL ? fmin(10.0 * fabs(S.p[i]), pref) : pref;
  double dn[3] = {0, 0, 0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    double fk = -p0 * double(acc[k]);
    dn[k] = 0.5 * dt * dt * fk;
    S.vgt[k][i] = dt * fk;
    double old = S.ut[k][i];
    double nw = __dadd_rn(unew[k], __ddiv_rn(double(float(dn[k])), dt));
    double xk = __dadd_rn(S.xn[k][i], __dmul_rn(__dmul_rn(0.5, dt), __dadd_rn(nw, old)));
    if (P.per[k]) {
      if (xk >= P.hi[k]) xk -= P.L[k];
      else if (xk < P.lo[k]) xk += P.L[k];
    }
    S.x[k][i] = xk;
    S.ut[k][i] = nw;
  }
  S.dgf[1][i] = make_float4(float(dn[0]), float(dn[1]), float(dn[2]), 0.f);
}

// ---------------------------------------------------------------------------
// Eqs. int:vhatnp2, int:rnp2:  u~^{n+1} = u^{n+1} + (r^K - r^0)/dt,
//   r^{n+1} = r^n + dt (u~^{n+1} + u~^n)/2, wrapped into periodic boxes.
// ---------------------------------------------------------------------------
template <int DIM, bool MX>
__global__ void k_update(State S, int skip_k1) {
  const Tile &t = S.ftiles[blockIdx.x];
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  if (skip_k1 && P.K == 1) return;
  const int par = P.K > 0 ? (P.K & 1) : 0;
  const double dt = P.dt;
  float4 df = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (MX) df = S.dgf[par][i];
  const float dfa[3] = {df.x, df.y, df.z};
_Pragma("unroll")
  for (int k = 0; k < DIM; ++k) {
    double dk;
    if constexpr (MX) dk = double(dfa[k]);
    else dk = S.dg[par][k][i];
    double old = S.ut[k][i];
    double nw = __dadd_rn(S.u[k][i], __ddiv_rn(dk, dt));
    double xk = __dadd_rn(S.xn[k][i], __dmul_rn(__dmul_rn(0.5, dt), __dadd_rn(nw, old)));
    if (P.per[k]) {
      if (xk >= P.hi[k]) xk -= P.L[k];
      else if (xk < P.lo[k]) xk += P.L[k];
    }
    S.x[k][i] = xk;
    S.ut[k][i] = nw;
  }
}

// Refresh the FP32 mirrors of velocity / density / pressure (MIXED) after
// the FP64 master state was written from the host.
__global__ void k_refresh(State S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  double u2 = S.dim == 3 ? S.u[2][i] : 0.0, t2 = S.dim == 3 ? S.ut[2][i] : 0.0;
  S.vf4[i] = make_float4(float(S.u[0][i]), float(S.u[1][i]), float(u2), float(S.rho[i]));
  S.utf4[i] = make_float4(float(S.ut[0][i]), float(S.ut[1][i]), float(t2), 0.f);
  S.pf[i] = float(S.p[i]);
}

// out_user[uid[i]] = field[i]
__global__ void k_scatter_field(State S, const void *src, int is_float, int stride_f4, int comp,
                                double *dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  double v;
  if (stride_f4) v = double((&static_cast<const float4 *>(src)[i].x)[comp]);
  else if (is_float == 2) v = double(static_cast<const int *>(src)[i]);
  else if (is_float) v = double(static_cast<const float *>(src)[i]);
  else v = static_cast<const double *>(src)[i];
  dst[S.uid[i]] = v;
}

// positions (moved_walls): a wall whose coordinate changes forces the next
// refresh to rebuild every case (fluid moves are caught by the refresh's own
// displacement check against the rebuild positions)
__global__ void k_gather_field(State S, const double *src, double *dst, int moved_walls) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  const double v = src[S.uid[i]];
  if (moved_walls && __double_as_longlong(v) != __double_as_longlong(dst[i]) &&
      i >= S.cases[S.case_of[i]].wbeg)
    *S.force = 1;
  dst[i] = v;
}

// ---------------------------------------------------------------------------
// Adaptive time step (Sec. 3.2).  k_speed_max: per case the maximum over its
// fluid of |u|^2 (which 0, at the start of the step) or of |f|^2 (which 1,
// the step's total acceleration), the squares evaluated as u0 u0 + u1 u1 +
// u2 u2 without contraction; a block reduces its tile and raises the case's
// maximum with one 64-bit atomic (non-negative doubles order as integers).
// k_adapt_dt: dt^{n+1} = min(0.25 h/max|u|, 0.25 sqrt(h/max|f|), 0.25 h^2/nu),
// a limit with a zero denominator left out (dt kept if all are); the
// maxima are cleared for the next step and the simulated time advances.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_speed_max(State S, int which) {
  const Tile &t = S.ftiles[blockIdx.x];
  const CaseDev &P = S.cases[t.c];
  if (!P.adaptive) return;
  const int i = t.beg + threadIdx.x;
  double v = 0.0;
  if (i < t.end) {
    double a[3] = {0.0, 0.0, 0.0};
    _Pragma("unroll") for (int k = 0; k < DIM; ++k) a[k] = which ? S.fs1[k][i] : S.u[k][i];
    v = __dadd_rn(__dadd_rn(__dmul_rn(a[0], a[0]), __dmul_rn(a[1], a[1])), __dmul_rn(a[2], a[2]));
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sh[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    unsigned long long *dst = (which ? S.fmax2 : S.umax2) + t.c;
    atomicMax(dst, static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

__global__ void k_adapt_dt(State S) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.ncases) return;
  CaseDev &P = const_cast<CaseDev &>(S.cases[c]);
  S.tsim[c] += P.dt;
  if (!P.adaptive) return;
  const double umax = sqrt(__longlong_as_double(static_cast<long long>(S.umax2[c])));
  const double fmax = sqrt(__longlong_as_double(static_cast<long long>(S.fmax2[c])));
  double dt = CUDART_INF;
  if (umax > 0.0) dt = fmin(dt, 0.25 * P.h / umax);
  if (fmax > 0.0) dt = fmin(dt, 0.25 * sqrt(P.h / fmax));
  dt = fmin(dt, P.dt_visc);
  if (isfinite(dt)) P.dt = dt;
  S.umax2[c] = 0ull;
  S.fmax2[c] = 0ull;
}

cudaError_t launch_speed_max(const State &S, const Launch &L, int which) {
  if (S.nft == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "speed_max");
  if (S.dim == 2) k_speed_max<2><<<S.nft, S.T, 0, L.stream>>>(S, which);
  else k_speed_max<3><<<S.nft, S.T, 0, L.stream>>>(S, which);
  if (L.after) L.after(L.ctx, "speed_max", double(S.nf), 1);
  return cudaGetLastError();
}

cudaError_t launch_adapt_dt(const State &S, const Launch &L) {
  if (L.before) L.before(L.ctx, "adapt_dt");
  k_adapt_dt<<<(S.ncases + 127) / 128, 128, 0, L.stream>>>(S);
  if (L.after) L.after(L.ctx, "adapt_dt", double(S.ncases), 1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
#define DISPATCH(S, KERN, ...)                                    \
  do {                                                            \
    if (S.dim == 2) {                                             \
      if (S.mixed) KERN<2, true> __VA_ARGS__;                     \
      else KERN<2, false> __VA_ARGS__;                            \
    } else {                                                      \
      if (S.mixed) KERN<3, true> __VA_ARGS__;                     \
      else KERN<3, false> __VA_ARGS__;                            \
    }                                                             \
  } while (0)

cudaError_t launch_density(const State &S, const Launch &L) {
  if (S.nft == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "density");
  DISPATCH(S, k_density, <<<S.nft, S.T, 0, L.stream>>>(S));
  if (L.after) L.after(L.ctx, "density", double(S.nf), 1);
  return cudaGetLastError();
}

cudaError_t launch_normals(const State &S, const Launch &L) {
  if (S.nwt == 0) return cudaSuccess;
  for (int pass = 0; pass < 2; ++pass) {
    if (S.dim == 2) k_normals<2><<<S.nwt, S.T, 0, L.stream>>>(S, pass);
    else k_normals<3><<<S.nwt, S.T, 0, L.stream>>>(S, pass);
  }
  return cudaGetLastError();
}

cudaError_t launch_ghost(const State &S, const Launch &L, int slip_stage) {
  if (S.nwt == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "ghost");
  DISPATCH(S, k_ghost, <<<S.nwt, S.T, 0, L.stream>>>(S, slip_stage));
  if (L.after) L.after(L.ctx, "ghost", double(S.nw), 1);
  return cudaGetLastError();
}

cudaError_t launch_stage1(const State &S, const Launch &L) {
  if (S.nft) {
    if (L.before) L.before(L.ctx, "stage1");
    DISPATCH(S, k_stage1, <<<S.nft, S.T, 0, L.stream>>>(S));
    if (L.after) L.after(L.ctx, "stage1", double(S.nf), 1);
  }
  if (S.nwt) {
    if (L.before) L.before(L.ctx, "stage1_walls");
    if (S.dim == 2) k_stage1_walls<2><<<S.nwt, S.T, 0, L.stream>>>(S);
    else k_stage1_walls<3><<<S.nwt, S.T, 0, L.stream>>>(S);
    if (L.after) L.after(L.ctx, "stage1_walls", double(S.nw), 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_pgrad(const State &S, const Launch &L) {
  if (S.nft == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "pgrad");
  DISPATCH(S, k_pgrad, <<<S.nft, S.T, 0, L.stream>>>(S));
  if (L.after) L.after(L.ctx, "pgrad", double(S.nf), 1);
  return cudaGetLastError();
}

cudaError_t launch_pref(const State &S, const Launch &L) {
  if (L.before) L.before(L.ctx, "pref");
  k_pref<<<S.ncases, 256, 0, L.stream>>>(S);
  if (L.after) L.after(L.ctx, "pref", double(S.ncases), 1);
  return cudaGetLastError();
}

cudaError_t launch_gtvf(const State &S, const Launch &L, int kmax, int skip_k1) {
  if (S.nft == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "gtvf");
  for (int sub = 0; sub < kmax; ++sub)
    DISPATCH(S, k_gtvf, <<<S.nft, S.T, 0, L.stream>>>(S, sub, sub & 1, skip_k1));
  if (L.after) L.after(L.ctx, "gtvf", double(S.nf) * kmax, kmax);
  return cudaGetLastError();
}

cudaError_t launch_update(const State &S, const Launch &L, int skip_k1) {
  if (S.nft == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "update");
  DISPATCH(S, k_update, <<<S.nft, S.T, 0, L.stream>>>(S, skip_k1));
  if (L.after) L.after(L.ctx, "update", double(S.nf), 1);
  return cudaGetLastError();
}

cudaError_t launch_pgrad_gtvf1(const State &S, const Launch &L) {
  if (S.nft == 0) return cudaSuccess;
  if (L.before) L.before(L.ctx, "pgrad_gtvf");
  if (S.dim == 2) k_pgrad_gtvf1<2><<<S.nft, S.T, 0, L.stream>>>(S);
  else k_pgrad_gtvf1<3><<<S.nft, S.T, 0, L.stream>>>(S);
  if (L.after) L.after(L.ctx, "pgrad_gtvf", double(S.nf), 1);
  return cudaGetLastError();
}

cudaError_t launch_refresh_mirrors(const State &S, const Launch &L) {
  if (!S.mixed) return cudaSuccess;
  k_refresh<<<(S.n + 255) / 256, 256, 0, L.stream>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_scatter_field(const State &S, const Launch &L, const void *src, int is_float,
                                 int stride_f4, int comp, double *dst_user) {
  k_scatter_field<<<(S.n + 255) / 256, 256, 0, L.stream>>>(S, src, is_float, stride_f4, comp, dst_user);
  return cudaGetLastError();
}

// Final GTVF displacement (buffer K & 1 of each particle's case) in user order.
__global__ void k_scatter_disp(State S, int comp, double *dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  int c = S.case_of[i];
  const CaseDev &P = S.cases[c];
  double v = 0.0;
  bool fluid = i < P.fbeg + P.nf;
  if (fluid && comp < S.dim) {
    int par = P.K & 1;
    if (S.mixed) v = double((&S.dgf[par][i].x)[comp]);
    else v = S.dg[par][comp][i];
  }
  dst[S.uid[i]] = v;
}

cudaError_t launch_scatter_disp(const State &S, const Launch &L, int comp, double *dst_user) {
  k_scatter_disp<<<(S.n + 255) / 256, 256, 0, L.stream>>>(S, comp, dst_user);
  return cudaGetLastError();
}

cudaError_t launch_gather_field(const State &S, const Launch &L, const double *src_user, double *dst,
                                bool positions) {
  k_gather_field<<<(S.n + 255) / 256, 256, 0, L.stream>>>(S, src_user, dst, positions ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace sisph
