// Device-side synchronisation and reduction helpers of the persistent PPE
// kernels (damped Jacobi and BiCGStab): the bounded grid barrier, block sums
// in FP32/FP64, and the per-case prefix that spreads the unfinished cases'
// work over the blocks.
#pragma once
#include "sisph_internal.h"

namespace sisph {

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

// Exclusive prefix over the cases of a per-case count, in shared memory
// (pre[0..nc], pre[nc] = total); thread t handles a contiguous run of
// cases.  Returns the total.  Used to spread the work of the cases still
// iterating evenly over the blocks.
template <typename F>
__device__ __forceinline__ int case_prefix(int nc, int *pre, int *wsum, F count) {
  const int T = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = T >> 5;
  const int per = (nc + T - 1) / T;
  const int c0 = threadIdx.x * per;
  int sum = 0;
  for (int c = c0; c < c0 + per && c < nc; ++c) sum += count(c);
  int x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int q = 0; q < nw; ++q) {
      const int t = wsum[q];
      wsum[q] = a;
      a += t;
    }
    wsum[nw] = a;
  }
  __syncthreads();
  int ex = wsum[w] + x - sum;
  for (int c = c0; c < c0 + per && c < nc; ++c) {
    pre[c] = ex;
    ex += count(c);
  }
  if (threadIdx.x == 0) pre[nc] = wsum[nw];
  __syncthreads();
  const int total = pre[nc];
  __syncthreads();
  return total;
}

// The case c with pre[c] <= a < pre[c + 1] (pre non-decreasing).
__device__ __forceinline__ int case_of_index(const int *pre, int nc, int a) {
  int lo = 0, hi = nc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= a) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// The sweep's arithmetic written out: the sweep's forms (grid barrier, point
// to point) round alike only if each multiply-add is fused or not in the same
// places, which a compiler left to contract a*b + c*d on its own does not
// promise across kernels.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R fma_r(R a, R b, R c) {
  if constexpr (std::is_same<R, float>::value) return __fmaf_rn(a, b, c);
  else return __fma_rn(a, b, c);
}
template <typename R>
__device__ __forceinline__ R mul_r(R a, R b) {
  if constexpr (std::is_same<R, float>::value) return __fmul_rn(a, b);
  else return __dmul_rn(a, b);
}
// p^{k+1} = omega/D (RHS + sum fac p^k) + (1 - omega) p^k (Eq. p-sor)
template <typename R>
__device__ __forceinline__ R jacobi_update(R wd, R acc, R om1, R po) {
  return fma_r(wd, acc, mul_r(om1, po));
}

// ---------------------------------------------------------------------------
// Stored PPE coefficients, one per ELL slot.  MIXED: the neighbour index and
// the FP32 coefficient packed in 8 bytes, so that a sweep streams one array
// with one load per slot; FP64: the coefficient alone (the index comes from
// the neighbour list).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void store_coef(void *base, long long o, int j, R fac) {
  if constexpr (std::is_same<R, float>::value)
    static_cast<uint2 *>(base)[o] = make_uint2(unsigned(j), __float_as_uint(fac));
  else
    static_cast<double *>(base)[o] = fac;
}

// The slots share the neighbour lists' blocked layout (ell_at): a warp's rows
// stream one contiguous run of 256-byte slot rows.
__device__ __forceinline__ long long slot_base(const State &S, int i) { return ell_base(S.cap, i); }
__device__ __forceinline__ long long slot_at(const State &S, int q, int i) { return ell_at(S.cap, q, i); }

// Slot q of row i (base = slot_base(S, i)): neighbour j and coefficient (a
// slot past the row's end, in false, reads the row itself with a zero
// coefficient).
template <typename R>
__device__ __forceinline__ void load_coef(const State &S, long long base, int q, bool in, int i, int &j,
                                          R &cf) {
  const long long o = base + (long long)q * kEllBlock;
  if constexpr (std::is_same<R, float>::value) {
    const uint2 v = in ? static_cast<const uint2 *>(S.coef)[o] : make_uint2(unsigned(i), 0u);
    j = int(v.x);
    cf = __uint_as_float(v.y);
  } else {
    j = in ? int(S.nbr[o] & kIdxMask) : i;
    cf = in ? static_cast<const double *>(S.coef)[o] : 0.0;
  }
  SISPH_CHECK_IDX(S, j, i);
}

// ---------------------------------------------------------------------------
// One wall row of Eq. p-shepard: p_w = (sum_f p_f W_wf + H_w) / sum_f W_wf,
// clamped at 0 in free-surface flows.  Chunks of CH: the index and weight
// loads go out together, then the CH pressure gathers; the sum runs over the
// entries in order whatever CH is.
// ---------------------------------------------------------------------------
template <typename R, int CH = 8>
__device__ __forceinline__ R wall_pressure(const State &S, const R *pc, int r, int w, int c) {
  const R *wc = static_cast<const R *>(S.wcoef);
  R acc = static_cast<const R *>(S.wh)[r];
  const int cnt = S.wcnt[r];
  for (int q0 = 0; q0 < cnt; q0 += CH) {
    int jj[CH];
    R ww[CH];
    _Pragma("unroll") for (int u = 0; u < CH; ++u) {
      const int q = q0 + u;
      const long long o = ell_at(S.wcap, q, r);
      jj[u] = q < cnt ? S.widx[o] : w;
      ww[u] = q < cnt ? wc[o] : R(0);
      SISPH_CHECK_IDX(S, jj[u], w);
    }
    R pv[CH];
    _Pragma("unroll") for (int u = 0; u < CH; ++u) pv[u] = pc[jj[u]];
    _Pragma("unroll") for (int u = 0; u < CH; ++u) acc = fma_r(ww[u], pv[u], acc);
  }
  R pw = acc * static_cast<const R *>(S.wsinv)[r];
  if (S.cases[c].free_surface && pw < R(0)) pw = R(0);
  return pw;
}

// Up to this many cases the work of the cases still iterating is spread
// evenly over the blocks in every phase; beyond, blocks stride over all
// tiles and skip the finished ones.
constexpr int kBalCases = 1024;

// A case is solved by the damped Jacobi iteration unless it asks for
// BiCGStab and its system is nonsingular (it has a free-surface row).
__device__ __forceinline__ bool jacobi_case(const State &S, int c) {
  return S.cases[c].solver == 0 || __ldcg(S.inact + c) == 0;
}

}  // namespace sisph
