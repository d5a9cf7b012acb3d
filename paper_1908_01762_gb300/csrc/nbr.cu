// Cell-list neighbour search: Morton-ordered counting sort of the particles
// and ELL neighbour lists.  The paper leaves the search to PySPH (Sec. 3.3);
// N(i) = {j : |r_ij|^2 < (3h)^2} with the minimum image in periodic
// directions, i itself included (support of the quintic spline, Sec. 2.1).
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
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    // cells are 3h (1 + 1e-9) or wider, so a product with 1/L_c instead of a
    // quotient still leaves any pair closer than 3h in adjacent cells
    double t = floor((xi[k] - P.lo[k]) * P.inv_lc[k]);
    int ci;
    if (!(t >= 0.0)) ci = 0;                       // also catches NaN
    else if (t >= double(P.nc[k])) ci = P.nc[k] - 1;
    else ci = int(t);
    c[k] = ci;
  }
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

template <int DIM>
__global__ void k_keys(State S, const double *__restrict__ p0, const double *__restrict__ p1,
                       const double *__restrict__ p2) {
  const Tile &t = tile_of(S, blockIdx.x);
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  double xi[3] = {p0[i], p1[i], DIM == 3 ? p2[i] : 0.0};
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
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned s = (lane < int(blockDim.x >> 5)) ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
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

__global__ void k_scan_chunks(unsigned *a, long long n, unsigned *bsum) {
  __shared__ unsigned sh[32];
  long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  unsigned v[kScanItems];
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0u;
    s += v[k];
  }
  unsigned tot;
  unsigned ex = block_excl_scan(s, sh, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) a[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_single(unsigned *a, int n) {
  __shared__ unsigned sh[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += kScanChunk) {
    int idx = base + threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = (idx + k < n) ? a[idx + k] : 0u;
      s += v[k];
    }
    unsigned tot;
    unsigned ex = block_excl_scan(s, sh, &tot) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (idx + k < n) a[idx + k] = ex;
      ex += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_add(unsigned *a, long long n, const unsigned *bsum) {
  long long base = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
  unsigned add = bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) a[base + k] += add;
}

__global__ void k_scatter(State S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
  unsigned dst = S.hist[S.key[i]] + S.slot[i];
  S.perm[dst] = i;
}

// Order each cell by original particle index, so the sorted order (and with
// it every neighbour-sum order) is independent of atomic arrival order.
__global__ void k_cellsort(State S, const int *__restrict__ uid) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S.K) return;
  unsigned beg = S.hist[q], end = S.hist[q + 1];
  if (end - beg < 2) return;
  for (unsigned a = beg + 1; a < end; ++a) {
    int pa = S.perm[a];
    int ka = uid[pa];
    unsigned b = a;
    while (b > beg) {
      int pb = S.perm[b - 1];
      if (uid[pb] <= ka) break;
      S.perm[b] = pb;
      --b;
    }
    S.perm[b] = pa;
  }
}

// Gather every per-particle stream into the new order.  mode 0: positions
// from x (build at r^n); mode 1: positions from the stage-1 output r*, the
// old positions become r^n and the velocity comes from u*.
template <int DIM>
__global__ void k_gather(State S, int mode, int gather_static) {
  int dst = blockIdx.x * blockDim.x + threadIdx.x;
  if (dst >= S.n) return;
  int src = S.perm[dst];
  double uu[3] = {0, 0, 0}, tt[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    if (mode == 0) {
      S.bx[k][dst] = S.x[k][src];
      S.bxn[k][dst] = S.xn[k][src];
      uu[k] = S.u[k][src];
    } else {
      S.bx[k][dst] = S.xs[k][src];
      S.bxn[k][dst] = S.x[k][src];
      uu[k] = S.us[k][src];
    }
    tt[k] = S.ut[k][src];
    S.bu[k][dst] = uu[k];
    S.but[k][dst] = tt[k];
  }
  double r = S.rho[src];
  S.bm[dst] = S.m[src];
  S.brho[dst] = r;
  S.bp[dst] = S.p[src];
  S.buid[dst] = S.uid[src];
  if (gather_static) {
    // walls only move once, at the first sort: carry their prescribed velocity
#pragma unroll
    for (int k = 0; k < 3; ++k) S.nstar[k][dst] = S.uw[k][src];
  }
  if (S.mixed) {
    S.vf4[dst] = make_float4(float(uu[0]), float(uu[1]), float(uu[2]), float(r));
    S.utf4[dst] = make_float4(float(tt[0]), float(tt[1]), float(tt[2]), 0.f);
    S.pf[dst] = float(S.p[src]);
  }
  // FP32 position relative to the particle's own cell, and its mass: the
  // neighbour build pre-tests pairs on it, the MIXED sums use it throughout
  const CaseDev &P = S.cases[S.case_of[dst]];
  double xi[3] = {0.0, 0.0, 0.0};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) xi[k] = S.bx[k][dst];
  int c[3];
  cell_of<DIM>(P, xi, c);
  float rel[3] = {0.f, 0.f, 0.f};
  _Pragma("unroll") for (int k = 0; k < DIM; ++k) rel[k] = float(xi[k] - (P.lo[k] + double(c[k]) * P.lc[k]));
  S.pf4[dst] = make_float4(rel[0], rel[1], rel[2], float(S.m[src]));
}

__global__ void k_copy_static(State S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) S.uw[k][i] = S.nstar[k][i];
}

// A cell on the edge of a non-periodic grid holds the particles that left
// the box (clamped into it), whose cell-relative coordinates can be large.
template <int DIM>
__device__ __forceinline__ bool edge_cell(const CaseDev &P, const int c[3]) {
  bool e = false;
  _Pragma("unroll") for (int k = 0; k < DIM; ++k)
    e |= !P.per[k] && (c[k] == 0 || c[k] == P.nc[k] - 1);
  return e;
}

// One thread per particle: scan the 3^d stencil of cells (fluid block, then
// wall block of each cell) and append every j with |r_ij|^2 < (3h)^2 to the
// ELL row.  Each candidate is first tested in FP32 on cell-relative
// coordinates (error below 1e-5 of (3h)^2); a pair within a relative band of
// 1e-4 around the cutoff is set aside and decided after the cell loop by the
// exact unfused FP64 test, so the set equals the FP64 definition and a warp
// pays for as many FP64 tests as its busiest lane (lattice inputs put many
// pairs exactly on the cutoff).  Edge cells of a non-periodic grid take the
// FP64 test directly.
template <int DIM>
__global__ void __launch_bounds__(256) k_build(State S) {
  constexpr int kBand = DIM == 3 ? 48 : 16;
  const Tile &t = tile_of(S, blockIdx.x);
  int i = t.beg + threadIdx.x;
  if (i >= t.end) return;
  const CaseDev &P = S.cases[t.c];
  double xi[3] = {S.x[0][i], S.x[1][i], DIM == 3 ? S.x[2][i] : 0.0};
  int c[3];
  cell_of<DIM>(P, xi, c);
  const bool own_edge = edge_cell<DIM>(P, c);
  const float4 pi = S.pf4[i];
  const float lx = P.lcf[0], ly = P.lcf[1], lz = P.lcf[2];
  const float cut2f = float(P.cut2);
  const float lo_band = cut2f * (1.0f - 1e-4f), hi_band = cut2f * (1.0f + 1e-4f);
  const int zr = (DIM == 3) ? 1 : 0;
  int cnt = 0;
  bool over = false;
  const long long nn = S.n;
  unsigned band[kBand];
  int nband = 0;
  auto append = [&](unsigned entry) {
    if (cnt < S.cap) S.nbr[(long long)cnt * nn + i] = entry;
    else over = true;
    ++cnt;
  };
  for (int oz = -zr; oz <= zr; ++oz) {
    for (int oy = -1; oy <= 1; ++oy) {
      for (int ox = -1; ox <= 1; ++ox) {
        int o[3] = {ox, oy, oz};
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
        const bool exact_all = own_edge || edge_cell<DIM>(P, cn);
        const unsigned code = stencil_code(ox, oy, oz) << kCodeShift;
        const float fx = pi.x - float(ox) * lx, fy = pi.y - float(oy) * ly, fz = pi.z - float(oz) * lz;
        long long m = cell_key<DIM>(P, cn);
        for (int kind = 0; kind < 2; ++kind) {
          if (kind == 1 && P.nw == 0) break;
          long long q = P.key_base + (long long)kind * P.slots + m;
          const unsigned beg = S.hist[q], end = S.hist[q + 1];
          if (exact_all) {
            for (unsigned j = beg; j < end; ++j) {
              double d[3];
              if (pair_d<DIM>(P, xi, S.x, int(j), d) < P.cut2) append(j | code);
            }
            continue;
          }
          // candidates 8 at a time: the loads go out together; slots past the
          // cell's end get a far-away position and are rejected by the test
          for (unsigned j0 = beg; j0 < end; j0 += 8) {
            float4 pj[8];
            _Pragma("unroll") for (int u = 0; u < 8; ++u)
              pj[u] = j0 + u < end ? S.pf4[j0 + u] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
            _Pragma("unroll") for (int u = 0; u < 8; ++u) {
              const unsigned j = j0 + u;
              float dx = fx - pj[u].x, dy = fy - pj[u].y;
              float r2f = dx * dx + dy * dy;
              if (DIM == 3) {
                float dz = fz - pj[u].z;
                r2f += dz * dz;
              }
              if (r2f < lo_band) {
                append(j | code);
              } else if (r2f <= hi_band) {
                if (nband < kBand) {
                  band[nband++] = j | code;
                } else {
                  double d[3];
                  if (pair_d<DIM>(P, xi, S.x, int(j), d) < P.cut2) append(j | code);
                }
              }
            }
          }
        }
      }
    }
  }
  for (int b = 0; b < nband; ++b) {
    double d[3];
    if (pair_d<DIM>(P, xi, S.x, int(band[b] & kIdxMask), d) < P.cut2) append(band[b]);
  }
  if (over) {
    atomicOr(S.err, kErrCapacity);
    cnt = S.cap;
  }
  S.ncnt[i] = cnt;
}

static cudaError_t scan(const State &S, const Launch &L, unsigned *bsum) {
  long long n = S.K + 1;
  int nb = int((n + kScanChunk - 1) / kScanChunk);
  k_scan_chunks<<<nb, kScanThreads, 0, L.stream>>>(S.hist, n, bsum);
  k_scan_single<<<1, kScanThreads, 0, L.stream>>>(bsum, nb);
  k_scan_add<<<nb, kScanThreads, 0, L.stream>>>(S.hist, n, bsum);
  return cudaGetLastError();
}

cudaError_t launch_sort(const State &S, const Launch &L, const double *const pos[3], int gather_mode,
                        bool gather_static) {
  int nt = S.nft + S.nwt;
  if (L.before) L.before(L.ctx, "sort");
  cudaMemsetAsync(S.hist, 0, sizeof(unsigned) * size_t(S.K + 1), L.stream);
  if (S.dim == 2) k_keys<2><<<nt, S.T, 0, L.stream>>>(S, pos[0], pos[1], pos[2]);
  else k_keys<3><<<nt, S.T, 0, L.stream>>>(S, pos[0], pos[1], pos[2]);
  // block sums live after the K+1 histogram entries
  unsigned *bsum = S.hist + (S.K + 1);
  cudaError_t e = scan(S, L, bsum);
  if (e != cudaSuccess) return e;
  int nb = (S.n + 255) / 256;
  k_scatter<<<nb, 256, 0, L.stream>>>(S);
  int kb = int((S.K + 255) / 256);
  k_cellsort<<<kb, 256, 0, L.stream>>>(S, S.uid);
  if (S.dim == 2) k_gather<2><<<nb, 256, 0, L.stream>>>(S, gather_mode, gather_static ? 1 : 0);
  else k_gather<3><<<nb, 256, 0, L.stream>>>(S, gather_mode, gather_static ? 1 : 0);
  if (L.after) L.after(L.ctx, "sort", double(S.n), 7);
  return cudaGetLastError();
}

cudaError_t launch_build(const State &S, const Launch &L) {
  int nt = S.nft + S.nwt;
  if (L.before) L.before(L.ctx, "build");
  if (S.dim == 2) k_build<2><<<nt, S.T, 0, L.stream>>>(S);
  else k_build<3><<<nt, S.T, 0, L.stream>>>(S);
  if (L.after) L.after(L.ctx, "build", double(S.n), 1);
  return cudaGetLastError();
}

cudaError_t launch_copy_static(const State &S, const Launch &L) {
  int nb = (S.n + 255) / 256;
  k_copy_static<<<nb, 256, 0, L.stream>>>(S);
  return cudaGetLastError();
}

}  // namespace sisph
