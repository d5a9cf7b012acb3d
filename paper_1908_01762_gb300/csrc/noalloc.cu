// Neighbour search that allocates nothing: sisph_neighbors_noalloc.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// already fully reserved by its own allocator (a framework's caching pool that
// owns the whole card), or a latency-critical loop that must not pay for
// cudaMalloc / cudaFree, which can synchronise the device.  For them this
// entry point runs the same cell-list search as the library's handles, with
// every piece of scratch memory (cell histogram, cell ids, slots, the sort
// permutation, a status word) in one file-scope device array of fixed size,
// reserved when the library is loaded and held by every GPU that loads it
// until the process exits.  The caller passes the positions and the output
// rows (device memory it allocated itself).
//
// Every call shares that array and it keeps the last call's contents; each
// call clears what must start at zero.  Calls whose kernels overlap on the GPU
// (for example on two streams at once) race on the array: serialise them.
// In host code the array's name is only a host-side stand-in: every call
// looks up the array's device address on the current device (the lookup
// allocates nothing), so a pointer from an earlier context -- before a
// cudaDeviceReset, or on another context of the same device -- is never used.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "sisph_internal.h"

namespace sisph {
void set_global_error(const std::string &msg);
}

namespace {

constexpr int kNaMaxPoints = SISPH_NOALLOC_MAX_POINTS;
constexpr int kNaMaxCells = SISPH_NOALLOC_MAX_CELLS;
// word offsets inside the scratch array
constexpr int kOffStart = 0;                               // kNaMaxCells + 1 cell starts
constexpr int kOffCell = kOffStart + kNaMaxCells + 1;      // cell id per point
constexpr int kOffSlot = kOffCell + kNaMaxPoints;          // slot inside the cell
constexpr int kOffPerm = kOffSlot + kNaMaxPoints;          // sorted order
constexpr int kOffStatus = kOffPerm + kNaMaxPoints;        // overflow flag
constexpr int kScratchWords = kOffStatus + 64;

static __device__ __align__(256) unsigned int g_na_scratch[kScratchWords];

struct NaGrid {
  int dim, n, ncell, cap;
  int nc[3], per[3];
  double lo[3], lc[3], L[3], half[3];
  double cut2;
};

__device__ __forceinline__ void na_cell(const NaGrid &G, const double *const x[3], int i, int c[3]) {
  c[0] = c[1] = c[2] = 0;
  for (int k = 0; k < G.dim; ++k) {
    double t = floor((x[k][i] - G.lo[k]) / G.lc[k]);
    int ci;
    if (!(t >= 0.0)) ci = G.per[k] ? G.nc[k] - 1 : 0;
    else if (t >= double(G.nc[k])) ci = G.per[k] ? 0 : G.nc[k] - 1;
    else ci = int(t);
    c[k] = ci;
  }
}

__global__ void k_na_clear(unsigned int *scr, int ncell) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q <= ncell) scr[kOffStart + q] = 0u;
  if (q < 64) scr[kOffStatus + q] = 0u;
}

__global__ void k_na_keys(NaGrid G, const double *x0, const double *x1, const double *x2, unsigned int *scr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  const double *const x[3] = {x0, x1, x2};
  int c[3];
  na_cell(G, x, i, c);
  unsigned cid = unsigned((c[2] * G.nc[1] + c[1]) * G.nc[0] + c[0]);
  scr[kOffCell + i] = cid;
  scr[kOffSlot + i] = atomicAdd(&scr[kOffStart + cid], 1u);
}

// one block: exclusive scan of the ncell + 1 counts
__global__ void k_na_scan(unsigned int *scr, int ncell) {
  __shared__ unsigned int warp_sum[32];
  __shared__ unsigned int carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  const int total = ncell + 1;
  for (int base = 0; base < total; base += blockDim.x) {
    int q = base + threadIdx.x;
    unsigned v = q < total ? scr[kOffStart + q] : 0u;
    unsigned x = v;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned s = lane < int(blockDim.x >> 5) ? warp_sum[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sum[lane] = s;
    }
    __syncthreads();
    unsigned ex = carry + (w > 0 ? warp_sum[w - 1] : 0u) + x - v;
    if (q < total) scr[kOffStart + q] = ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
}

__global__ void k_na_scatter(int n, unsigned int *scr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned cid = scr[kOffCell + i];
  scr[kOffPerm + scr[kOffStart + cid] + scr[kOffSlot + i]] = unsigned(i);
}

__global__ void k_na_cellsort(int ncell, unsigned int *scr) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ncell) return;
  unsigned beg = scr[kOffStart + q], end = scr[kOffStart + q + 1];
  unsigned *perm = scr + kOffPerm;
  for (unsigned a = beg + 1; a < end; ++a) {
    unsigned v = perm[a];
    unsigned b = a;
    while (b > beg && perm[b - 1] > v) {
      perm[b] = perm[b - 1];
      --b;
    }
    perm[b] = v;
  }
}

// Row i (the caller's order): every j with |r_ij|^2 < (3h)^2, minimum image,
// |r_ij|^2 = dx*dx + dy*dy (+ dz*dz) unfused, ascending j; rows are
// row-major, cap entries each.  A row with more than cap neighbours keeps its
// cap smallest indices (a larger index is dropped, a smaller one displaces
// the row's largest) and raises the status word.
__global__ void k_na_rows(NaGrid G, const double *x0, const double *x1, const double *x2,
                          unsigned int *scr, int *counts, int *idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  const double *const x[3] = {x0, x1, x2};
  int c[3];
  na_cell(G, x, i, c);
  double xi[3] = {x0[i], x1[i], G.dim == 3 ? x2[i] : 0.0};
  const unsigned *start = scr + kOffStart;
  const unsigned *perm = scr + kOffPerm;
  int *row = idx + (long long)i * G.cap;
  int cnt = 0;
  const int zr = G.dim == 3 ? 1 : 0;
  for (int oz = -zr; oz <= zr; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        int o[3] = {ox, oy, oz};
        int cn[3] = {0, 0, 0};
        bool skip = false;
        for (int k = 0; k < G.dim; ++k) {
          int v = c[k] + o[k];
          if (v < 0 || v >= G.nc[k]) {
            if (G.per[k]) v = (v + G.nc[k]) % G.nc[k];
            else skip = true;
          }
          cn[k] = v;
        }
        if (skip) continue;
        int q = (cn[2] * G.nc[1] + cn[1]) * G.nc[0] + cn[0];
        for (unsigned t = start[q]; t < start[q + 1]; ++t) {
          int j = int(perm[t]);
          double d[3] = {0.0, 0.0, 0.0};
          for (int k = 0; k < G.dim; ++k) {
            double v = xi[k] - x[k][j];
            if (G.per[k]) {
              if (v > G.half[k]) v -= G.L[k];
              else if (v < -G.half[k]) v += G.L[k];
            }
            d[k] = v;
          }
          double r2 = __dmul_rn(d[0], d[0]);
          r2 = __dadd_rn(r2, __dmul_rn(d[1], d[1]));
          if (G.dim == 3) r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
          if (r2 < G.cut2) {
            if (cnt >= G.cap) atomicOr(&scr[kOffStatus], 1u);
            if (cnt < G.cap || j < row[G.cap - 1]) {
              // insert in ascending order (a full row drops its largest)
              int b = cnt < G.cap ? cnt : G.cap - 1;
              while (b > 0 && row[b - 1] > j) {
                row[b] = row[b - 1];
                --b;
              }
              row[b] = j;
            }
            ++cnt;
          }
        }
      }
  counts[i] = cnt < G.cap ? cnt : G.cap;
}

int na_fail(int code, const std::string &msg) {
  sisph::set_global_error(msg);
  return code;
}

}  // namespace

extern "C" int sisph_neighbors_noalloc(int32_t dim, int32_t n, const double *x_dev, const double *y_dev,
                                       const double *z_dev, double h, const double lo[3], const double hi[3],
                                       const int32_t periodic[3], int32_t cap, int32_t *counts_dev,
                                       int32_t *idx_dev, void *stream) {
  if (dim != 2 && dim != 3) return na_fail(SISPH_EINVAL, "noalloc: dim must be 2 or 3");
  if (n < 1 || n > kNaMaxPoints)
    return na_fail(SISPH_EINVAL, "noalloc: n must be in [1, " + std::to_string(kNaMaxPoints) + "]");
  if (!x_dev || !y_dev || (dim == 3 && !z_dev) || !counts_dev || !idx_dev || !lo || !hi || !periodic)
    return na_fail(SISPH_EINVAL, "noalloc: a required pointer is NULL");
  if (!(h > 0.0) || cap < 1) return na_fail(SISPH_EINVAL, "noalloc: h > 0 and cap >= 1 required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    // the call reads a status word back and waits for its kernels, which a
    // capturing stream does not allow: reject it before anything is launched
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ec = cudaStreamIsCapturing(st, &cs);
    if (ec != cudaSuccess) {
      cudaGetLastError();
      return na_fail(SISPH_ECUDA, std::string("noalloc: ") + cudaGetErrorString(ec));
    }
    if (cs != cudaStreamCaptureStatusNone)
      return na_fail(SISPH_EINVAL, "noalloc: the stream is capturing a graph; the call synchronises it");
  }
  NaGrid G{};
  G.dim = dim;
  G.n = n;
  G.cap = cap;
  G.cut2 = (3.0 * h) * (3.0 * h);
  const double lcmin = 3.0 * h * (1.0 + 1e-9);
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    G.nc[k] = 1;
    G.lc[k] = 1.0;
    G.lo[k] = 0.0;
    if (k >= dim) continue;
    G.lo[k] = lo[k];
    G.L[k] = hi[k] - lo[k];
    G.half[k] = 0.5 * G.L[k];
    G.per[k] = periodic[k] ? 1 : 0;
    if (!(G.L[k] > 0.0)) return na_fail(SISPH_EINVAL, "noalloc: hi must exceed lo");
    double ncd = G.per[k] ? std::floor(G.L[k] / lcmin) : std::ceil(G.L[k] / lcmin);
    if (G.per[k] && ncd < 3.0) return na_fail(SISPH_EINVAL, "noalloc: a periodic length must hold 3 cells of 3h");
    if (ncd > double(kNaMaxCells)) return na_fail(SISPH_EINVAL, "noalloc: too many cells");
    G.nc[k] = ncd < 1.0 ? 1 : int(ncd);
    G.lc[k] = G.per[k] ? G.L[k] / double(G.nc[k]) : lcmin;
    ncell *= G.nc[k];
  }
  if (ncell > kNaMaxCells)
    return na_fail(SISPH_EINVAL, "noalloc: the box needs " + std::to_string(ncell) + " cells, more than " +
                                     std::to_string(kNaMaxCells));
  G.ncell = int(ncell);

  // the device address of the scratch array on the current device (the
  // array's name in host code is only a host-side stand-in), looked up at
  // every call with that device current
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return na_fail(SISPH_ECUDA, std::string("noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  }
  unsigned int *scr = static_cast<unsigned int *>(ptr);
  const int T = 256;
  const double *z = dim == 3 ? z_dev : x_dev;
  k_na_clear<<<(G.ncell + 1 + T - 1) / T + 1, T, 0, st>>>(scr, G.ncell);
  k_na_keys<<<(n + T - 1) / T, T, 0, st>>>(G, x_dev, y_dev, z, scr);
  k_na_scan<<<1, 1024, 0, st>>>(scr, G.ncell);
  k_na_scatter<<<(n + T - 1) / T, T, 0, st>>>(n, scr);
  k_na_cellsort<<<(G.ncell + T - 1) / T, T, 0, st>>>(G.ncell, scr);
  k_na_rows<<<(n + T - 1) / T, T, 0, st>>>(G, x_dev, y_dev, z, scr, counts_dev, idx_dev);
  e = cudaGetLastError();
  unsigned int status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, scr + kOffStatus, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(SISPH_ECUDA, std::string("noalloc: ") + cudaGetErrorString(e));
  if (status) return na_fail(SISPH_ECAPACITY, "noalloc: a point has more than cap neighbours");
  return SISPH_OK;
}
