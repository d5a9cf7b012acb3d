// Cell-list neighbour search with Verlet skin lists.  The paper leaves the
// search to PySPH (Sec. 3.3); N(i) = {j : |r_ij|^2 < (3h)^2} with the minimum
// image in periodic directions, i itself included (support of the quintic
// spline, Sec. 2.1).
//
// One refresh of the lists at positions X (r^n, or r* after stage 1):
//  check    a case whose fluid moved more than s/2 since its last rebuild
//           (or every case, on a forced refresh) is marked for a rebuild;
//  rebuild  only when some case is marked (every kernel returns at once
//           otherwise): Morton-ordered counting sort of the particle set --
//           marked cases binned at X, the others at their last rebuild
//           positions, which leaves them where they are -- gather, copy back;
//           then, for the marked cases, the skin list: every j within 3h + s
//           of i at the rebuild positions;
//  finish   without a rebuild, the stage-1 outputs and FP32 mirrors are
//           committed in place; the FP32 relative positions are brought to X;
//           then N(i) is filtered exactly out of the skin list at X.
// The order of the particles and the skin lists are a function of the rebuild
// positions alone, so a state restored with them (force mode 2: rebuild every
// case at its stored rebuild positions) continues bit-identically.
// Between rebuilds no particle has moved more than s/2 from its rebuild
// position, so every pair now closer than 3h was closer than 3h + s then.
#include "sisph_internal.h"

namespace sisph {

__device__ __forceinline__ unsigned spread2(unsigned x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

__device__ __forceinline__ unsigned spread3(unsigned x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

template <int DIM>
__device__ __forceinline__ void cell_of(const CaseDev &P, const double xi[3], int c[3]) {
  c[2] = 0;
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    // cells are (3h + s)(1 + 1e-9) or wider, so a product with 1/L_c instead
    // of a quotient still leaves any pair closer than 3h + s in adjacent cells
    double t = floor((xi[k] - P.lo[k]) * P.inv_lc[k]);
    int ci;
    if (!(t >= 0.0)) ci = 0;                       // also catches NaN
    else if (t >= double(P.nc[k])) ci = P.nc[k] - 1;
    else ci = int(t);
    c[k] = ci;
  }
}

// Rebuild cell of a particle, 21 bits per axis.
__device__ __forceinline__ long long pack_cell(const int c[3]) {
  return (long long)c[0] | ((long long)c[1] << 21) | ((long long)c[2] << 42);
}
__device__ __forceinline__ void unpack_cell(long long v, int c[3]) {
  c[0] = int(v & 0x1fffff);
  c[1] = int((v >> 21) & 0x1fffff);
  c[2] = int((v >> 42) & 0x1fffff);
}

template <int DIM>
__device__ __forceinline__ long long cell_key(const CaseDev &P, const int c[3]) {
  if (P.morton) {
    if (DIM == 2) return (long long)(spread2(unsigned(c[0])) | (spread2(unsigned(c[1])) << 1));
    return (long long)(spread3(unsigned(c[0])) | (spread3(unsigned(c[1])) << 1) |
                       (spread3(unsigned(c[2])) << 2));
  }
  return ((long long)c[2] * P.nc[1] + c[1]) * P.nc[0] + c[0];
}

__device__ __forceinline__ const Tile &tile_of(const State &S, int b) {
  return b < S.nft ? S.ftiles[b] : S.wtiles[b - S.nft];
}

// FP32 pair tests on cell-relative coordinates are trusted while both
// coordinates lie within kNearCells cell widths of their cell's origin: every
// operand of r_ij = rel_i - rel_j - o lc is then below 17 lc in magnitude, so
// each component carries an absolute error below 34 * 2^-24 lc, and with lc
// at most 8h (a skin of 3h in a periodic box of three cells) |r_ij|^2 near
// the cutoff a relative error below 2e-5 of (3h)^2, inside the bands the
// tests use.  Only a
// particle that left a non-periodic box (clamped into an edge cell) can be
// farther; its pairs take the FP64 test.
constexpr float kNearCells = 8.0f;
template <int DIM>
__device__ __forceinline__ bool near_cell(const float4 &p, const float lc[3]) {
  bool ok = fabsf(p.x) <= kNearCells * lc[0] && fabsf(p.y) <= kNearCells * lc[1];
  if (DIM == 3) ok = ok && fabsf(p.z) <= kNearCells * lc[2];
  return ok;
}

// FP32 position relative to the origin of the particle's rebuild cell (the
// minimum image of it in periodic directions, since a particle may have
// wrapped since the rebuild), and its mass: the neighbour tests use it, and
// so do all MIXED neighbour sums.  The mass carries the near-range test in
// its sign (negative: outside the near range), so that a neighbour test
// reads it with one comparison; every sum takes its magnitude.
template <int DIM>
__device__ __forceinline__ float4 rel_pos(const CaseDev &P, const double xi[3], long long cell, double m) {
  int c[3];
  unpack_cell(cell, c);
  float rel[3] = {0.f, 0.f, 0.f};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    double d = xi[k] - (P.lo[k] + double(c[k]) * P.lc[k]);
    if (P.per[k]) {
      if (d > P.half[k]) d -= P.L[k];
      else if (d < -P.half[k]) d += P.L[k];
    }
    rel[k] = float(d);
  }
  const float4 p = make_float4(rel[0], rel[1], rel[2], float(m));
  const float lc[3] = {P.lcf[0], P.lcf[1], P.lcf[2]};
  return make_float4(p.x, p.y, p.z, near_cell<DIM>(p, lc) ? p.w : -p.w);
}

// The near-range test of a mirrored position (the sign of its mass).
__device__ __forceinline__ bool is_near(const float4 &p) { return p.w > 0.f; }

// ---------------------------------------------------------------------------
// check
// ---------------------------------------------------------------------------
// Mark case c for a rebuild; count the rebuilds per case and the refreshes
// that rebuild anything (last counter).
__device__ __forceinline__ void mark(const State &S, int c) {
  if (atomicOr(S.need + c, 1) == 0) atomicAdd(reinterpret_cast<unsigned long long *>(S.nreb + c), 1ull);
  if (atomicOr(S.anyneed, 1) == 0)
    atomicAdd(reinterpret_cast<unsigned long long *>(S.nreb + S.ncases), 1ull);
}

// Binned at the current positions X: a marked case, unless the refresh
// restores the stored rebuild positions.
__device__ __forceinline__ bool at_x(const State &S, int c) { return S.need[c] != 0 && *S.force != 2; }

template <int DIM>
__global__ void k_check(State S, const double *__restrict__ x0, const double *__restrict__ x1,
                        const double *__restrict__ x2) {
  const Tile &t = tile_of(S, blockIdx.x);
  const int c = t.c;
  if (*S.force) {
    if (threadIdx.x == 0) mark(S, c);
    return;
  }
  if (t.kind != 0) return;   // walls never move
  const int i = t.beg + threadIdx.x;
  bool moved = false;
  if (i < t.end) {
    const CaseDev &P = S.cases[c];
    const double X[3] = {x0[i], x1[i], DIM == 3 ? x2[i] : 0.0};
    double d2 = 0.0;
    _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
      double d = X[k] - S.xref[k][i];
      if (P.per[k]) {
        if (d > P.half[k]) d -= P.L[k];
        else if (d < -P.half[k]) d += P.L[k];
      }
      d2 += d * d;
    }
    moved = !(d2 <= P.skin_half2);   // also catches NaN
  }
  if (__syncthreads_or(moved) && threadIdx.x == 0) mark(S, c);
}

// ---------------------------------------------------------------------------
// rebuild: counting sort
// ---------------------------------------------------------------------------
__global__ void k_zero_hist(State S, int count_on_device) {
  if (!*S.anyneed) return;
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (count_on_device && q == 0) atomicAdd(reinterpret_cast<unsigned long long *>(S.nbody), 1ull);
  if (q <= S.K) S.hist[q] = 0u;
}

// Marked cases are binned at X, the others at their rebuild positions.
template <int DIM>
__global__ void k_keys(State S, const double *__restrict__ p0, const double *__restrict__ p1,
                       const double *__restrict__ p2) {
  if (!*S.anyneed) return;
  const Tile &t = tile_of(S, blockIdx.x);
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  const bool mv = at_x(S, t.c);
  double xi[3];
  xi[0] = mv ? p0[i] : S.xref[0][i];
  xi[1] = mv ? p1[i] : S.xref[1][i];
  xi[2] = DIM == 3 ? (mv ? p2[i] : S.xref[2][i]) : 0.0;
  int c[3];
  cell_of<DIM>(P, xi, c);
  long long key = P.key_base + (long long)t.kind * P.slots + cell_key<DIM>(P, c);
  S.key[i] = unsigned(key);
  S.slot[i] = atomicAdd(&S.hist[key], 1u);
}

// Exclusive scan of hist[0..K] (K+1 entries), three phases.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *sh, unsigned *total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
  _Pragma("unroll") for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned s = (lane < int(blockDim.x >> 5)) ? sh[lane] : 0u;
    _Pragma("unroll") for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  unsigned base = (w > 0) ? sh[w - 1] : 0u;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  return base + x - v;
}

__global__ void k_scan_chunks(const int *flag, unsigned *a, long long n, unsigned *bsum) {
  if (!*flag) return;
  __shared__ unsigned sh[32];
  long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  unsigned v[kScanItems];
  unsigned s = 0;
  _Pragma("unroll") for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0u;
    s += v[k];
  }
  unsigned tot;
  unsigned ex = block_excl_scan(s, sh, &tot);
  _Pragma("unroll") for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) a[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_single(const int *flag, unsigned *a, int n) {
  if (!*flag) return;
  __shared__ unsigned sh[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += kScanChunk) {
    int idx = base + threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
    _Pragma("unroll") for (int k = 0; k < kScanItems; ++k) {
      v[k] = (idx + k < n) ? a[idx + k] : 0u;
      s += v[k];
    }
    unsigned tot;
    unsigned ex = block_excl_scan(s, sh, &tot) + carry;
    _Pragma("unroll") for (int k = 0; k < kScanItems; ++k) {
      if (idx + k < n) a[idx + k] = ex;
      ex += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_add(const int *flag, unsigned *a, long long n, const unsigned *bsum) {
  if (!*flag) return;
  long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  unsigned add = bsum[blockIdx.x];
  _Pragma("unroll") for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) a[base + k] += add;
}

__global__ void k_scatter(State S) {
  if (!*S.anyneed) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  unsigned dst = S.hist[S.key[i]] + S.slot[i];
  S.perm[dst] = i;
}

// Order each cell by original particle index, so the sorted order (and with
// it every neighbour-sum order) is independent of atomic arrival order.
__global__ void k_cellsort(State S) {
  if (!*S.anyneed) return;
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S.K) return;
  unsigned beg = S.hist[q], end = S.hist[q + 1];
  if (end - beg < 2) return;
  for (unsigned a = beg + 1; a < end; ++a) {
    int pa = S.perm[a];
    int ka = S.uid[pa];
    unsigned b = a;
    while (b > beg) {
      int pb = S.perm[b - 1];
      if (S.uid[pb] <= ka) break;
      S.perm[b] = pb;
      --b;
    }
    S.perm[b] = pa;
  }
}

// Gather every per-particle stream into the new order (B buffers).  mode 0:
// positions from x (refresh at r^n); mode 1: positions from the stage-1
// output r*, the old positions become r^n and the velocity comes from u*.
// The rebuild position follows the particle; a marked case takes its
// current position as the new one.
// A case that is not rebuilt keeps its order (its particles are binned at
// their stored rebuild positions, in the cells and in-cell order they already
// have, and no other case's keys fall among theirs), so its particles are
// left where they are; k_sync commits them as in a refresh without rebuild.
template <int DIM>
__global__ void k_gather(State S, int mode, int gather_static) {
  if (!*S.anyneed) return;
  int dst = blockIdx.x * blockDim.x + threadIdx.x;
  if (dst >= S.n) return;
  const int c = S.case_of[dst];
  if (!gather_static && !S.need[c]) return;
  const int src = S.perm[dst];
  const bool mv = at_x(S, c);
  double uu[3] = {0, 0, 0}, tt[3] = {0, 0, 0}, xr[3] = {0, 0, 0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    double xnew;
    if (mode == 0) {
      xnew = S.x[k][src];
      S.bxn[k][dst] = S.xn[k][src];
      uu[k] = S.u[k][src];
    } else {
      xnew = S.xs[k][src];
      S.bxn[k][dst] = S.x[k][src];
      uu[k] = S.us[k][src];
    }
    S.bx[k][dst] = xnew;
    xr[k] = mv ? xnew : S.xref[k][src];
    S.bxref[k][dst] = xr[k];
    tt[k] = S.ut[k][src];
    S.bu[k][dst] = uu[k];
    S.but[k][dst] = tt[k];
  }
  const double r = S.rho[src];
  S.bm[dst] = S.m[src];
  S.brho[dst] = r;
  S.bp[dst] = S.p[src];
  S.buid[dst] = S.uid[src];
  int cc[3];
  cell_of<DIM>(S.cases[c], xr, cc);
  S.bcell[dst] = pack_cell(cc);
  if (gather_static) {
    // walls only move once, at the first sort: carry their prescribed velocity
    _Pragma("unroll") for (int k = 0; k < 3; ++k) S.nstar[k][dst] = S.uw[k][src];
  }
  if (S.mixed) {
    S.vf4[dst] = make_float4(float(uu[0]), float(uu[1]), float(uu[2]), float(r));
    S.utf4[dst] = make_float4(float(tt[0]), float(tt[1]), float(tt[2]), 0.f);
    S.pf[dst] = float(S.p[src]);
  }
}

// Copy the gathered streams back into the state; the FP32 relative
// positions are taken at the rebuild positions for the skin lists.
template <int DIM>
__global__ void k_copyback(State S, int gather_static) {
  if (!*S.anyneed) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  if (!gather_static && !S.need[S.case_of[i]]) return;   // not rebuilt: not gathered
  double xr[3] = {0.0, 0.0, 0.0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    xr[k] = S.bxref[k][i];
    S.x[k][i] = S.bx[k][i];
    S.xn[k][i] = S.bxn[k][i];
    S.u[k][i] = S.bu[k][i];
    S.ut[k][i] = S.but[k][i];
    S.xref[k][i] = xr[k];
  }
  const double m = S.bm[i];
  const long long cell = S.bcell[i];
  S.m[i] = m;
  S.rho[i] = S.brho[i];
  S.p[i] = S.bp[i];
  S.uid[i] = S.buid[i];
  S.cell[i] = cell;
  if (gather_static) {
    _Pragma("unroll") for (int k = 0; k < 3; ++k) S.uw[k][i] = S.nstar[k][i];
  }
  S.pf4[i] = rel_pos<DIM>(S.cases[S.case_of[i]], xr, cell, m);
}

// ---------------------------------------------------------------------------
// rebuild: skin lists of the marked cases, every j within 3h + s of i (FP32
// test on cell-relative coordinates with a relative margin of 2e-4 on the
// squared cutoff, which covers its rounding; FP64 for a pair with a particle
// outside the near range), all at the rebuild positions.  The list only has
// to contain N(i) at every later refresh before the next rebuild.
// Walls never move, so the wall-wall pairs of a wall row are final here: a
// wall row starts with its wall neighbours within 3h exactly (the filter's
// FP32 test with the FP64 decision inside the band), wfin[i] of them, built
// at forced rebuilds only, then its fluid skin candidates.  The refresh
// copies that head unchanged, and the wall passes, which sum over fluid
// neighbours only, start after it.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_skin(State S) {
  const Tile &t = tile_of(S, blockIdx.x);
  if (!S.need[t.c]) return;
  const int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  const bool wall_row = i >= P.wbeg;
  int c[3];
  unpack_cell(S.cell[i], c);
  const double xi[3] = {S.xref[0][i], S.xref[1][i], DIM == 3 ? S.xref[2][i] : 0.0};
  const float4 pi = S.pf4[i];
  const float lc[3] = {P.lcf[0], P.lcf[1], P.lcf[2]};
  const float lx = lc[0], ly = lc[1], lz = lc[2];
  const bool exact_all = !near_cell<DIM>(pi, lc);
  const float cut2f = float(P.cut_s2) * (1.0f + 2e-4f);
  const float cull2f = float(P.cut_s2) * (1.0f + 1e-3f);
  const double cut2d = P.cut_s2 * (1.0 + 2e-4);
  const float cutf = float(P.cut2);
  const float lo_band = cutf * (1.0f - 1e-4f), hi_band = cutf * (1.0f + 1e-4f);
  const int zr = (DIM == 3) ? 1 : 0;
  int cnt = 0;
  bool over = false;
  auto append = [&](unsigned entry) {
    // a fluid row's own entry is placed first, before the scan (below)
    if (!wall_row && (entry & kIdxMask) == unsigned(i)) return;
    if (cnt < S.scap) S.snbr[ell_at(S.scap, cnt, i)] = entry;
    else over = true;
    ++cnt;
  };
  // the same for a candidate that is kept or not (k), without a branch
  auto append_if = [&](bool k, unsigned entry) {
    k = k && (wall_row || (entry & kIdxMask) != unsigned(i));
    if (k && cnt < S.scap) S.snbr[ell_at(S.scap, cnt, i)] = entry;
    over = over || (k && cnt >= S.scap);
    cnt += k ? 1 : 0;
  };
  // candidates of the stencil cells in buckets k0..k1 (0 fluid, 1 walls);
  // exact: N(i) itself (3h, walls only), else the skin test (3h + s)
  auto scan = [&](int k0, int k1, bool exact) {
    const double cut_d = exact ? P.cut2 : cut2d;
    for (int oz = -zr; oz <= zr; ++oz) {
      for (int oy = -1; oy <= 1; ++oy) {
        for (int ox = -1; ox <= 1; ++ox) {
          const int o[3] = {ox, oy, oz};
          int cn[3] = {c[0], c[1], c[2]};
          bool skip = false;
          _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
            int v = c[k] + o[k];
            if (v < 0 || v >= P.nc[k]) {
              if (P.per[k]) v = (v + P.nc[k]) % P.nc[k];
              else skip = true;
            }
            cn[k] = v;
          }
          if (skip) continue;
          const unsigned code = stencil_code(ox, oy, oz) << kCodeShift;
          const float fx = pi.x - float(ox) * lx, fy = pi.y - float(oy) * ly, fz = pi.z - float(oz) * lz;
          if (!exact_all) {
            // the neighbour cell spans [o lc, (o + 1) lc) per axis around i's
            // cell origin: skip it when its nearest point is beyond the skin
            // radius (with a margin far above the FP32 rounding of pi)
            const float ex = ox < 0 ? pi.x : (ox > 0 ? lx - pi.x : 0.f);
            const float ey = oy < 0 ? pi.y : (oy > 0 ? ly - pi.y : 0.f);
            const float ez = DIM == 3 ? (oz < 0 ? pi.z : (oz > 0 ? lz - pi.z : 0.f)) : 0.f;
            const float e2 = fmaxf(ex, 0.f) * fmaxf(ex, 0.f) + fmaxf(ey, 0.f) * fmaxf(ey, 0.f) +
                             fmaxf(ez, 0.f) * fmaxf(ez, 0.f);
            if (e2 > cull2f) continue;
          }
          const long long m = cell_key<DIM>(P, cn);
          for (int kind = k0; kind <= k1; ++kind) {
            if (kind == 1 && P.nw == 0) break;
            const long long q = P.key_base + (long long)kind * P.slots + m;
            const unsigned beg = S.hist[q], end = S.hist[q + 1];
            if (exact_all) {
              for (unsigned j = beg; j < end; ++j) {
                double d[3];
                if (pair_d<DIM>(P, xi, S.xref, int(j), d) < cut_d) append(j | code);
              }
              continue;
            }
            // candidates 8 at a time: the loads go out together; slots past
            // the cell's end get a position inside the near range, four cells
            // away, and are rejected by their index
            for (unsigned j0 = beg; j0 < end; j0 += 8) {
              float4 pj[8];
              _Pragma("unroll") for (int u = 0; u < 8; ++u)
                pj[u] = j0 + u < end ? S.pf4[j0 + u] : make_float4(4.f * lx, 4.f * ly, 4.f * lz, 0.f);
              _Pragma("unroll") for (int u = 0; u < 8; ++u) {
                const unsigned j = j0 + u;
                const bool nr = near_cell<DIM>(pj[u], lc);
                float dx = fx - pj[u].x, dy = fy - pj[u].y;
                float r2f = dx * dx + dy * dy;
                if (DIM == 3) {
                  float dz = fz - pj[u].z;
                  r2f += dz * dz;
                }
                if (!exact) {
                  // the common case without a branch; a particle outside
                  // the near range (rare) takes the FP64 test
                  bool k = nr && r2f < cut2f && j < end;
                  if (!nr) {
                    double d[3];
                    k = j < end && pair_d<DIM>(P, xi, S.xref, int(j), d) < cut_d;
                  }
                  append_if(k, j | code);
                } else if (!nr) {
                  double d[3];
                  if (j < end && pair_d<DIM>(P, xi, S.xref, int(j), d) < cut_d) append(j | code);
                } else if (r2f < lo_band) {
                  append(j | code);
                } else if (r2f <= hi_band) {
                  double d[3];
                  if (pair_d<DIM>(P, xi, S.xref, int(j), d) < P.cut2) append(j | code);
                }
              }
            }
          }
        }
      }
    }
  };
  int head = 0;
  if (wall_row && *S.force == 0) {
    // walls keep their positions, cells and sorted order between rebuilds
    // that nothing forced (creation, a caller's sisph_set and a restore all
    // force one), so the head built last time is still in place
    head = cnt = S.wfin[i];
    scan(0, 0, false);
  } else if (wall_row) {
    scan(1, 1, true);
    head = cnt;
    scan(0, 0, false);
  } else {
    // a fluid row starts with i itself, so that its lists (and the MIXED PPE
    // slots, which leave i out) keep one layout across the warp's rows
    S.snbr[ell_at(S.scap, 0, i)] = unsigned(i) | (stencil_code(0, 0, 0) << kCodeShift);
    cnt = 1;
    scan(0, 1, false);
  }
  if (over) {
    atomicOr(S.err, kErrCapacity);
    cnt = S.scap;
    head = min(head, S.scap);
  }
  S.sncnt[i] = cnt;
  S.wfin[i] = head;
}

// ---------------------------------------------------------------------------
// finish
// ---------------------------------------------------------------------------
// Without a rebuild of the particle's case its order is unchanged: mode 1
// commits the stage-1 outputs in place (r^n <- r, r <- r*, u <- u*) and the
// FP32 mirrors are refreshed from the FP64 state, as the gather would have
// done.  Always: the FP32 relative positions at X.
template <int DIM>
__global__ void k_sync(State S, int mode) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  const int c = S.case_of[i];
  const CaseDev &P = S.cases[c];
  double xi[3] = {0, 0, 0};
  if (*S.anyneed && S.need[c]) {
    // rebuilt: the gather has committed the state in the new order
    _Pragma("unroll") for (int k = 0; k < DIM; ++k) xi[k] = S.x[k][i];
    S.pf4[i] = rel_pos<DIM>(P, xi, S.cell[i], S.m[i]);
    return;
  }
  double uu[3] = {0, 0, 0}, tt[3] = {0, 0, 0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) {
    if (mode == 1) {
      xi[k] = S.xs[k][i];
      S.xn[k][i] = S.x[k][i];
      S.x[k][i] = xi[k];
      uu[k] = S.us[k][i];
      S.u[k][i] = uu[k];
    } else {
      xi[k] = S.x[k][i];
      uu[k] = S.u[k][i];
    }
    tt[k] = S.ut[k][i];
  }
  if (S.mixed) {
    S.vf4[i] = make_float4(float(uu[0]), float(uu[1]), float(uu[2]), float(S.rho[i]));
    S.utf4[i] = make_float4(float(tt[0]), float(tt[1]), float(tt[2]), 0.f);
    S.pf[i] = float(S.p[i]);
  }
  S.pf4[i] = rel_pos<DIM>(P, xi, S.cell[i], S.m[i]);
}

// N(i) out of the skin list at the current positions: FP32 test on
// cell-relative coordinates (error below 2e-5 of (3h)^2).
//   EXACT (the lists the API shows): a pair within a relative band of 1e-4 of
//     the cutoff, or with a particle outside the near range, is set aside and
//     decided after the loop by the exact unfused FP64 test, so the set equals
//     the FP64 definition.  Lattice inputs put many pairs exactly on the
//     cutoff; their FP64 tests run from a register copy of the case's
//     periodic data, loaded once.
//   otherwise (the refreshes inside a step): fluid rows leave out the pairs
//     whose FP32 |r_ij|^2 is within a relative 4e-5 below the cutoff or
//     above it, so no FP64 test runs unless a particle is outside the near
//     range.  Every pair left out has |r_ij| > 3h (1 - 3e-5), where the
//     quintic's weight is below 1e-21 and its gradient below 1e-17 of their
//     largest values, so no sum of a fluid row changes above FP64 rounding.
//     Wall rows, whose Shepard sums are normalised, stay exact.
// A wall row's head (its wall neighbours, decided exactly at the rebuild) is
// copied first.  The order is deterministic: the skin list's order, the
// set-aside pairs last.
struct PeriodicBox {
  int per[3];
  double half[3], L[3];
};

// DENS (MIXED, in-step refresh at r^n): a fluid row also sums its summation
// density (Eq. summation_density) over the pairs it keeps, in the order they
// are kept, with the same FP32 pair vector as the density pass, so the step
// needs no separate density pass over N(i).
template <int DIM, bool EXACT, bool DENS = false>
__global__ void __launch_bounds__(256, 4) k_filter(State S) {
  constexpr int kBand = DIM == 3 ? 48 : 16;   // at most 64 (one bit each below)
  constexpr int kU = DIM == 3 ? 4 : 6;         // candidates whose loads go out together
  const Tile &t = tile_of(S, blockIdx.x);
  const int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  const float4 pi = S.pf4[i];
  const float lc[3] = {P.lcf[0], P.lcf[1], P.lcf[2]};
  const bool own_near = is_near(pi);
  const float cut2f = float(P.cut2);
  // wall rows stay exact: their Shepard sums are normalised, so a wall whose
  // only fluid neighbour sits on the rim takes that neighbour's value
  const bool ex = EXACT || blockIdx.x >= unsigned(S.nft);
  const float lo_band = cut2f * (ex ? 1.0f - 1e-4f : 1.0f - 4e-5f), hi_band = cut2f * (1.0f + 1e-4f);
  const int scnt = S.sncnt[i];
  const int head = S.wfin[i];
  const long long sb = ell_base(S.scap, i);
  // cnt counts every kept entry; one past the capacity is reported after
  // the loops
  int cnt = 0;
  unsigned band[kBand];
  int nband = 0;
  auto append = [&](unsigned entry) {
    if (cnt < S.cap) S.nbr[ell_at(S.cap, cnt, i)] = entry;
    ++cnt;
  };
  const bool dens = DENS && blockIdx.x < unsigned(S.nft);
  const float dih = float(P.inv_h);
  float rho = 0.f;
  // a candidate of the skin list, kept or not (k), without a branch: a kept
  // entry is stored while the row has room and, when the row sums its
  // density (sum, a compile-time flag of each loop), adds m_j W_ij to it; one
  // not kept adds 0.  (Under a branch the warp would run the kept path
  // whenever one lane keeps, which is almost always, and pay for the branch
  // on top.)
  auto keep_if = [&](auto sum, bool k, unsigned entry, float r2f, float mj) {
    if (k && cnt < S.cap) S.nbr[ell_at(S.cap, cnt, i)] = entry;
    cnt += k ? 1 : 0;
    if constexpr (decltype(sum)::value) {
      const float w = mj * poly_w<float>(sqrtf(r2f) * dih);
      rho += k ? w : 0.f;
    }
  };
  auto exact = [&](unsigned entry) {
    const double xi[3] = {S.x[0][i], S.x[1][i], DIM == 3 ? S.x[2][i] : 0.0};
    double d[3];
    return pair_d<DIM>(P, xi, S.x, int(entry & kIdxMask), d) < P.cut2;
  };
  // a wall row's head (its wall neighbours, decided at the rebuild) is final
  for (int q0 = 0; q0 < head; q0 += 4) {
    unsigned h4[4];
    _Pragma("unroll") for (int u = 0; u < 4; ++u)
      h4[u] = q0 + u < head ? S.snbr[sb + (long long)(q0 + u) * kEllBlock] : 0u;
    _Pragma("unroll") for (int u = 0; u < 4; ++u) {
      SISPH_CHECK_ENTRY(S, h4[u], unsigned(i));
      if (q0 + u < head) append(h4[u]);
    }
  }
  // the next chunk's entries are loaded while this chunk's positions are
  // gathered (a slot past the row's end reads the row itself).  The loop is
  // compiled twice, for exact rows and for the others (a block-uniform
  // choice), so that the others test only for a particle outside the near
  // range
  const unsigned self = unsigned(i) | (stencil_code(0, 0, 0) << kCodeShift);
  auto candidates = [&](auto exact_rows) {
    constexpr bool EX = decltype(exact_rows)::value;
    unsigned en[kU];
    _Pragma("unroll") for (int u = 0; u < kU; ++u)
      en[u] = head + u < scnt ? S.snbr[sb + (long long)(head + u) * kEllBlock] : self;
    for (int q0 = head; q0 < scnt; q0 += kU) {
      unsigned e[kU];
      float4 pj[kU];
      _Pragma("unroll") for (int u = 0; u < kU; ++u) {
        e[u] = en[u];
        SISPH_CHECK_ENTRY(S, e[u], self);
        pj[u] = S.pf4[e[u] & kIdxMask];
      }
      _Pragma("unroll") for (int u = 0; u < kU; ++u) {
        const int q = q0 + kU + u;
        en[u] = q < scnt ? S.snbr[sb + (long long)q * kEllBlock] : self;
      }
      _Pragma("unroll") for (int u = 0; u < kU; ++u) {
        const bool valid = q0 + u < scnt;
        float d[3];
        const float r2f = pair_f<DIM>(lc, pi, pj[u], e[u] >> kCodeShift, d);
        const bool near = own_near && is_near(pj[u]);
        bool k = valid && near && r2f < lo_band;
        // rare: a particle outside the near range, or (exact rows) a pair in
        // the band around the cutoff: set aside for the FP64 test after the
        // loop, or decided here by it (not exact rows, or a full band)
        if (valid && (!near || (EX && r2f >= lo_band && r2f <= hi_band))) {
          if (EX && nband < kBand) band[nband++] = e[u];
          else k = exact(e[u]);
        }
        // exact rows are wall rows or the API's lists: neither sums a density
        keep_if(std::integral_constant<bool, DENS && !EX>{}, k, e[u], r2f, fabsf(pj[u].w));
      }
    }
  };
  if (ex) candidates(std::true_type{});
  else candidates(std::false_type{});
  if (ex && nband) {
    PeriodicBox B;
    _Pragma("unroll") for (int k = 0; k < 3; ++k) {
      B.per[k] = P.per[k];
      B.half[k] = P.half[k];
      B.L[k] = P.L[k];
    }
    const double cut2 = P.cut2;
    const double xi[3] = {S.x[0][i], S.x[1][i], DIM == 3 ? S.x[2][i] : 0.0};
    // all tests first (no store between their loads), then the appends
    unsigned long long keep = 0ull;
    _Pragma("unroll 4") for (int b = 0; b < nband; ++b) {
      double d[3];
      keep |= (unsigned long long)(pair_d<DIM>(B, xi, S.x, int(band[b] & kIdxMask), d) < cut2) << b;
    }
    for (int b = 0; b < nband; ++b)
      if ((keep >> b) & 1ull) append(band[b]);
  }
  if (cnt > S.cap) {
    atomicOr(S.err, kErrCapacity);
    cnt = S.cap;
  }
  S.ncnt[i] = cnt;
  if (DENS && dens) {
    rho *= float(P.sig_h);
    S.rho[i] = double(rho);
    S.vf4[i].w = rho;
  }
}

// The rebuild group of a captured step sits in a conditional graph node whose
// condition is whether any case needs a rebuild.
__global__ void k_set_conditional(cudaGraphConditionalHandle h, const int *anyneed) {
  cudaGraphSetConditional(h, *anyneed ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_set_conditional(const State &S, const Launch &L, cudaGraphConditionalHandle h) {
  if (L.before) L.before(L.ctx, "setcond");
  k_set_conditional<<<1, 1, 0, L.stream>>>(h, S.anyneed);
  if (L.after) L.after(L.ctx, "setcond", 0.0, 1);
  return cudaGetLastError();
}

cudaError_t launch_refresh_check(const State &S, const Launch &L, int mode) {
  const int nt = S.nft + S.nwt;
  const double *const *pos = mode == 0 ? S.x : S.xs;
  cudaMemsetAsync(S.need, 0, sizeof(int) * size_t(S.ncases), L.stream);
  cudaMemsetAsync(S.anyneed, 0, sizeof(int), L.stream);
  if (L.before) L.before(L.ctx, "check");
  if (S.dim == 2) k_check<2><<<nt, S.T, 0, L.stream>>>(S, pos[0], pos[1], pos[2]);
  else k_check<3><<<nt, S.T, 0, L.stream>>>(S, pos[0], pos[1], pos[2]);
  if (L.after) L.after(L.ctx, "check", double(S.n), 1);
  return cudaGetLastError();
}

cudaError_t launch_refresh_rebuild(const State &S, const Launch &L, int mode, bool gather_static,
                                   bool count_on_device) {
  const int nt = S.nft + S.nwt;
  const int nb = (S.n + 255) / 256;
  const double *const *pos = mode == 0 ? S.x : S.xs;
  const int gs = gather_static ? 1 : 0;
  if (L.before) L.before(L.ctx, "sort");
  k_zero_hist<<<int((S.K + 1 + 255) / 256), 256, 0, L.stream>>>(S, count_on_device ? 1 : 0);
  if (S.dim == 2) k_keys<2><<<nt, S.T, 0, L.stream>>>(S, pos[0], pos[1], pos[2]);
  else k_keys<3><<<nt, S.T, 0, L.stream>>>(S, pos[0], pos[1], pos[2]);
  // block sums live after the K+1 histogram entries
  const long long nh = S.K + 1;
  const int ns = int((nh + kScanChunk - 1) / kScanChunk);
  unsigned *bsum = S.hist + nh;
  k_scan_chunks<<<ns, kScanThreads, 0, L.stream>>>(S.anyneed, S.hist, nh, bsum);
  k_scan_single<<<1, kScanThreads, 0, L.stream>>>(S.anyneed, bsum, ns);
  k_scan_add<<<ns, kScanThreads, 0, L.stream>>>(S.anyneed, S.hist, nh, bsum);
  k_scatter<<<nb, 256, 0, L.stream>>>(S);
  k_cellsort<<<int((S.K + 255) / 256), 256, 0, L.stream>>>(S);
  if (S.dim == 2) {
    k_gather<2><<<nb, 256, 0, L.stream>>>(S, mode, gs);
    k_copyback<2><<<nb, 256, 0, L.stream>>>(S, gs);
  } else {
    k_gather<3><<<nb, 256, 0, L.stream>>>(S, mode, gs);
    k_copyback<3><<<nb, 256, 0, L.stream>>>(S, gs);
  }
  if (L.after) L.after(L.ctx, "sort", double(S.n), 9);
  if (L.before) L.before(L.ctx, "build");
  if (S.dim == 2) k_skin<2><<<nt, S.T, 0, L.stream>>>(S);
  else k_skin<3><<<nt, S.T, 0, L.stream>>>(S);
  if (L.after) L.after(L.ctx, "build", double(S.n), 1);
  return cudaGetLastError();
}

cudaError_t launch_refresh_finish(const State &S, const Launch &L, int mode, bool exact, bool density) {
  const int nt = S.nft + S.nwt;
  const int nb = (S.n + 255) / 256;
  if (L.before) L.before(L.ctx, "sync");
  if (S.dim == 2) k_sync<2><<<nb, 256, 0, L.stream>>>(S, mode);
  else k_sync<3><<<nb, 256, 0, L.stream>>>(S, mode);
  if (L.after) L.after(L.ctx, "sync", double(S.n), 1);
  if (L.before) L.before(L.ctx, "filter");
  if (exact) {
    if (S.dim == 2) k_filter<2, true><<<nt, S.T, 0, L.stream>>>(S);
    else k_filter<3, true><<<nt, S.T, 0, L.stream>>>(S);
  } else if (density && S.mixed) {
    if (S.dim == 2) k_filter<2, false, true><<<nt, S.T, 0, L.stream>>>(S);
    else k_filter<3, false, true><<<nt, S.T, 0, L.stream>>>(S);
  } else {
    if (S.dim == 2) k_filter<2, false><<<nt, S.T, 0, L.stream>>>(S);
    else k_filter<3, false><<<nt, S.T, 0, L.stream>>>(S);
  }
  if (L.after) L.after(L.ctx, "filter", double(S.n), 1);
  cudaMemsetAsync(S.force, 0, sizeof(int), L.stream);
  return cudaGetLastError();
}

}  // namespace sisph
