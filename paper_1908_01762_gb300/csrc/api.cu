// Host runtime behind the C-ABI of include/sisph.h: validation, the static
// particle layout, device allocation, the order of the kernels in one time
// step (Algorithm 1), CUDA-graph capture and replay, event timing, field
// access in the caller's order, and checkpoints.  Every kernel site and API
// call is an NVTX range (header-only NVTX 3: inert unless a tool attaches).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "sisph_internal.h"

using namespace sisph;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace sisph {
// Error message of a call that has no handle (creation, the no-alloc search).
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace sisph

namespace {

struct Pending {
  std::string name;
  double units;
  int nk;
  cudaEvent_t a, b;
};

struct ProfRec {
  int64_t launches = 0;
  double ms = 0.0;
  double units = 0.0;
};

}  // namespace

struct sisph_s {
  std::string err;
  State S{};
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;     // captures the body of the rebuild node
  sisph_options opt{};
  std::vector<sisph_case_params> prm;
  std::vector<CaseDev> hc;
  std::vector<Tile> hft, hwt;
  std::vector<void *> allocs;
  int ncases = 0, dim = 2;
  int64_t n = 0, nf = 0, nw = 0;
  int kmax = 1;
  int grid = 1;
  bool adaptive = false;           // some case adapts its time step
  bool krylov = false;             // some case asks for BiCGStab
  int grid_k = 1;                  // BiCGStab kernel grid
  // the captured step
  cudaGraphExec_t gexec = nullptr;
  bool graph_failed = false;
  bool no_conditional = false;     // capture the rebuild group unconditionally
  int graph_kernels = 0;
  // profiling
  bool profiling = false;
  std::string prof_only;           // empty: every kernel, no graphs
  std::vector<std::string> prof_set;  // prof_only split at commas
  bool capturing = false;
  std::vector<Pending> gsites;     // event nodes inside the captured graph
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, ProfRec> prof;
  int64_t launches = 0;
  int counting = 1;
  double *d_tmp = nullptr, *d_tmp2 = nullptr;
  long long sweep_units_pending = 0;
  // sisph_get_many / sisph_set_many: one staging column of n doubles per
  // field and a copy stream of their own, so that each field's host copy
  // overlaps the reordering of the field before (or after) it
  double *d_stage = nullptr;
  int stage_fields = 0;
  cudaStream_t copy = nullptr;
  std::vector<cudaEvent_t> xev;
};

namespace {

int fail(sisph_t s, int code, const std::string &msg) {
  if (s) s->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(sisph_t s, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(s, SISPH_ECUDA, m);
}

template <typename T>
cudaError_t dalloc(sisph_t s, T **p, size_t count) {
  void *v = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e != cudaSuccess) return e;
  s->allocs.push_back(v);
  *p = static_cast<T *>(v);
  return cudaSuccess;
}

bool profiled(sisph_t s, const char *name) {
  if (!s->profiling) return false;
  if (s->prof_only.empty()) return true;
  for (const auto &q : s->prof_set)
    if (q == name) return true;
  return false;
}

// An NVTX range around one API call.
struct NvtxScope {
  explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope &) = delete;
  NvtxScope &operator=(const NvtxScope &) = delete;
};

void before_cb(void *ctx, const char *name) {
  sisph_t s = static_cast<sisph_t>(ctx);
  nvtxRangePushA(name);
  if (!profiled(s, name)) return;
  if (s->capturing) {
    // a dedicated pair per launch site, recorded as external event nodes
    Pending p;
    p.name = name;
    p.units = 0;
    p.nk = 0;
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecordWithFlags(p.a, s->stream, cudaEventRecordExternal);
    s->gsites.push_back(p);
    return;
  }
  Pending p;
  p.name = name;
  p.units = 0;
  p.nk = 0;
  if (s->pool.size() < 2) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    s->pool.push_back(a);
    s->pool.push_back(b);
  }
  p.a = s->pool.back();
  s->pool.pop_back();
  p.b = s->pool.back();
  s->pool.pop_back();
  cudaEventRecord(p.a, s->stream);
  s->pending.push_back(p);
}

void after_cb(void *ctx, const char *name, double units, int nk) {
  sisph_t s = static_cast<sisph_t>(ctx);
  nvtxRangePop();
  if (s->counting) s->launches += nk;
  if (!profiled(s, name)) return;
  if (s->capturing) {
    Pending &p = s->gsites.back();
    p.units = units;
    p.nk = nk;
    cudaEventRecordWithFlags(p.b, s->stream, cudaEventRecordExternal);
    return;
  }
  Pending &p = s->pending.back();
  p.units = units;
  p.nk = nk;
  cudaEventRecord(p.b, s->stream);
}

Launch mk_launch(sisph_t s) {
  Launch L;
  L.stream = s->stream;
  L.before = before_cb;
  L.after = after_cb;
  L.ctx = s;
  return L;
}

void drain_profile(sisph_t s) {
  if (s->pending.empty()) return;
  cudaStreamSynchronize(s->stream);
  for (auto &p : s->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    ProfRec &r = s->prof[p.name];
    r.launches += 1;
    r.ms += ms;
    r.units += p.units;
    if (p.nk >= 0) {
      s->pool.push_back(p.a);
      s->pool.push_back(p.b);
    }
  }
  s->pending.clear();
}

// After one replay of the captured step: read its event nodes.
void drain_graph_sites(sisph_t s) {
  if (s->gsites.empty()) return;
  cudaStreamSynchronize(s->stream);
  for (auto &p : s->gsites) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    ProfRec &r = s->prof[p.name];
    r.launches += 1;
    r.ms += ms;
    r.units += p.units;
  }
}

// Capture the rebuild group into the body of a conditional node of the step
// graph: the node runs its body only when the check marked some case.  Body
// kernels are counted on the device (k_zero_hist), not here.
cudaError_t capture_rebuild_conditional(sisph_t s, int mode, bool first) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s->stream, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e != cudaSuccess) return e;
  e = launch_set_conditional(s->S, mk_launch(s), h);
  if (e != cudaSuccess) return e;
  e = cudaStreamGetCaptureInfo(s->stream, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  // (the struct holds a union without a default constructor: zeroed storage)
  alignas(cudaGraphNodeParams) unsigned char cp_mem[sizeof(cudaGraphNodeParams)];
  memset(cp_mem, 0, sizeof(cp_mem));
  cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_mem);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamUpdateCaptureDependencies(s->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(s->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  Launch B = mk_launch(s);
  B.stream = s->side;
  B.before = nullptr;
  B.after = nullptr;
  cudaError_t eb = launch_refresh_rebuild(s->S, B, mode, first, true);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(s->side, &out);
  return eb != cudaSuccess ? eb : e;
}

// One refresh of the neighbour lists (mode 0 at x, mode 1 at r*).  The
// buffers never change places on the host, so one captured graph serves
// every step.  Whether the cell sort and skin lists are rebuilt is decided on
// the device: in a captured step by a conditional node (unless a profiled
// site lies in the group, whose kernels then return at once without a
// rebuild), in direct launches by reading the decision back.
cudaError_t do_refresh(sisph_t s, int mode, bool first, bool exact = false, bool density = false) {
  Launch L = mk_launch(s);
  cudaError_t e = launch_refresh_check(s->S, L, mode);
  if (e != cudaSuccess) return e;
  const bool prof_group =
      profiled(s, "sort") || profiled(s, "build");
  if (s->capturing && !prof_group && !s->no_conditional) {
    e = capture_rebuild_conditional(s, mode, first);
  } else if (s->capturing) {
    e = launch_refresh_rebuild(s->S, L, mode, first, false);
  } else {
    int any = 0;
    e = cudaMemcpyAsync(&any, s->S.anyneed, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess && any) e = launch_refresh_rebuild(s->S, L, mode, first, false);
  }
  if (e == cudaSuccess) e = launch_refresh_finish(s->S, L, mode, exact, density);
  return e;
}

// Next refresh rebuilds every case: mode 1 at the current positions, mode 2
// at the stored rebuild positions (the int is written as 0 then its low byte).
cudaError_t force_rebuild(sisph_t s, int mode = 1) {
  cudaError_t e = cudaMemsetAsync(s->S.force, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->S.force, mode, 1, s->stream);
  return e;
}

cudaError_t do_ppe(sisph_t s) {
  Launch L = mk_launch(s);
  cudaError_t e = launch_ghost(s->S, L, 1);
  if (e == cudaSuccess) e = launch_ppe_setup(s->S, L);
  if (e == cudaSuccess) e = launch_ppe_reset(s->S, L);
  if (e == cudaSuccess && s->krylov) e = launch_ppe_krylov(s->S, L, s->grid_k);   // BiCGStab cases
  if (e == cudaSuccess) e = launch_ppe_sweeps(s->S, L, s->grid);                   // the rest
  return e;
}

cudaError_t do_step(sisph_t s) {
  Launch L = mk_launch(s);
  // neighbours at r^n; in MIXED the same pass sums rho (Eq. summation_density)
  cudaError_t e = do_refresh(s, 0, false, false, s->S.mixed != 0);
  if (e == cudaSuccess && s->adaptive) e = launch_speed_max(s->S, L, 0);  // max|u^n| (Sec. 3.2)
  if (e == cudaSuccess && !s->S.mixed) e = launch_density(s->S, L);  // rho (Eq. summation_density)
  if (e == cudaSuccess) e = launch_ghost(s->S, L, 0); // no-slip ghost velocity
  if (e == cudaSuccess) e = launch_stage1(s->S, L);   // u*, r* (Eqs. int:vint, int:rnp1)
  if (e == cudaSuccess) e = do_refresh(s, 1, false);  // neighbours at r*
  if (e == cudaSuccess) e = do_ppe(s);                // Eqs. sph-ppe, p-sor, convergence
  if (e == cudaSuccess) e = launch_pref(s->S, L);     // p_ref after the first solve
  if (s->S.mixed) {
    // one pass for the cases with K = 1; separate GTVF sub-steps and update
    // only for cases with K > 1
    if (e == cudaSuccess) e = launch_pgrad_gtvf1(s->S, L);
    if (e == cudaSuccess && s->kmax > 1) e = launch_gtvf(s->S, L, s->kmax, 1);
    if (e == cudaSuccess && s->kmax > 1) e = launch_update(s->S, L, 1);
  } else {
    if (e == cudaSuccess) e = launch_pgrad(s->S, L);    // Eq. int:vnp1
    if (e == cudaSuccess) e = launch_gtvf(s->S, L, s->kmax, 0);  // Eqs. int:gtvf:*
    if (e == cudaSuccess) e = launch_update(s->S, L, 0);   // Eqs. int:vhatnp2, int:rnp2
  }
  // next time step (Sec. 3.2) and the simulated time
  if (e == cudaSuccess && s->adaptive) e = launch_speed_max(s->S, L, 1);
  if (e == cudaSuccess) e = launch_adapt_dt(s->S, L);
  return e;
}

int check_status(sisph_t s, bool sweeps_ran) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, s->S.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "kernel execution");
  int bar_err = 0;
  if (sweeps_ran) {
    e = cudaMemcpy(&bar_err, &s->S.bar->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "status read");
  }
  cudaMemsetAsync(s->S.err, 0, sizeof(int), s->stream);
  if (bar_err || (err & kErrTimeout))
    return fail(s, SISPH_ETIMEOUT, "persistent PPE kernel: grid barrier wait exceeded its budget");
  if (err & kErrCapacity)
    return fail(s, SISPH_ECAPACITY, "a particle has more neighbours than the neighbour capacity");
  if (err & kErrNonFinite) return fail(s, SISPH_ENONFINITE, "non-finite PPE residual");
  if (err & kErrInternal)
    return fail(s, SISPH_EINTERNAL, "checked build: a gathered neighbour index was out of range");
  if (err & kErrNotConv) return fail(s, SISPH_ENOTCONVERGED, "PPE reached max_iter before the tolerance");
  return SISPH_OK;
}

bool valid_handle(sisph_t s) { return s != nullptr && s->S.n > 0; }

void destroy_graphs(sisph_t s) {
  if (s->gexec) {
    cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
  }
  for (auto &q : s->gsites) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  s->gsites.clear();
}

int setup_case(sisph_t s, int c, const sisph_particles &P, const sisph_case_params &q, int64_t fbeg,
               int64_t nfc, int64_t nwc, int64_t wrow, long long key_base, CaseDev &D) {
  memset(&D, 0, sizeof(D));
  const int dim = P.dim;
  const double cut = 3.0 * q.h;
  // Verlet skin; a periodic box too small for three cells of 3h + s falls
  // back to rebuilding at every refresh (s = 0)
  double skin = s->opt.skin * cut;
  for (int k = 0; k < dim; ++k)
    if (P.periodic[k] && std::floor((P.hi[k] - P.lo[k]) / ((cut + skin) * (1.0 + 1e-9))) < 3.0) skin = 0.0;
  const double lcmin = (cut + skin) * (1.0 + 1e-9);
  D.skin = skin;
  D.cut_s2 = (cut + skin) * (cut + skin);
  D.skin_half2 = skin > 0.0 ? 0.25 * skin * skin : -1.0;
  int maxnc = 1;
  for (int k = 0; k < 3; ++k) {
    D.lo[k] = P.lo[k];
    D.hi[k] = P.hi[k];
    D.L[k] = P.hi[k] - P.lo[k];
    D.half[k] = 0.5 * D.L[k];
    D.per[k] = (k < dim) ? (P.periodic[k] ? 1 : 0) : 0;
    if (k >= dim) {
      D.nc[k] = 1;
      D.lc[k] = 1.0;
      D.inv_lc[k] = 1.0;
      D.lcf[k] = 1.f;
      continue;
    }
    if (!(D.L[k] > 0.0)) return fail(nullptr, SISPH_EINVAL, "case " + std::to_string(c) + ": hi <= lo");
    if (D.per[k]) {
      double ncd = std::floor(D.L[k] / lcmin);
      if (ncd < 3.0)
        return fail(nullptr, SISPH_EINVAL,
                    "case " + std::to_string(c) + ": periodic length must hold at least 3 cells of 3h");
      if (ncd > double(kMaxCellsPerAxis))
        return fail(nullptr, SISPH_EINVAL, "case " + std::to_string(c) + ": too many cells");
      D.nc[k] = int(ncd);
      D.lc[k] = D.L[k] / double(D.nc[k]);
    } else {
      // one margin cell on each side: particles inside [lo, hi) never sit in
      // an edge cell, which only collects particles that left the box
      D.lc[k] = lcmin;
      double ncd = std::ceil(D.L[k] / lcmin);
      if (ncd > double(kMaxCellsPerAxis - 2))
        return fail(nullptr, SISPH_EINVAL, "case " + std::to_string(c) + ": too many cells");
      D.nc[k] = std::max(1, int(ncd)) + 2;
      D.lo[k] = P.lo[k] - lcmin;
    }
    D.lcf[k] = float(D.lc[k]);
    D.inv_lc[k] = 1.0 / D.lc[k];
    maxnc = std::max(maxnc, D.nc[k]);
  }
  int bits = 0;
  while ((1 << bits) < maxnc) ++bits;
  long long mslots = 1LL << (dim * bits);
  long long dense = (long long)D.nc[0] * D.nc[1] * D.nc[2];
  if ((dim == 2 && bits <= 16 && mslots <= (1LL << 24)) || (dim == 3 && bits <= 10 && mslots <= (1LL << 24))) {
    D.morton = 1;
    D.bits = bits;
    D.slots = mslots;
  } else {
    D.morton = 0;
    D.slots = dense;
  }
  D.key_base = key_base;
  D.h = q.h;
  D.dt = q.dt;
  D.rho0 = q.rho0;
  D.nu = q.nu;
  for (int k = 0; k < 3; ++k) D.g[k] = (k < dim) ? q.g[k] : 0.0;
  D.alpha = q.alpha;
  D.c0 = q.c0;
  D.tol = q.tol;
  D.hfac = q.gtvf_hfac;
  D.max_iter = q.max_iter;
  D.pgrad_symm = q.pgrad_symm;
  D.free_surface = q.free_surface;
  D.ustar_slip = q.ustar_slip;
  D.pref_mode = q.pref_mode;
  D.K = q.gtvf_K;
  D.p_ref0 = q.p_ref;
  D.adaptive = q.adaptive_dt;
  D.solver = q.ppe_solver;
  D.dt_visc = q.nu > 0.0 ? 0.25 * q.h * q.h / q.nu : INFINITY;
  D.cut2 = (3.0 * q.h) * (3.0 * q.h);
  D.eh2 = s->opt.eta * q.h * q.h;
  D.inv_h = 1.0 / q.h;
  D.sig_h = quintic_sigma(q.h, dim);
  D.h2 = 0.5 * q.h;
  D.inv_h2 = 1.0 / D.h2;
  D.sig_h2 = quintic_sigma(D.h2, dim);
  double hg = q.gtvf_hfac * q.h;
  D.hg = hg;
  D.inv_hg = 1.0 / hg;
  D.sig_hg = quintic_sigma(hg, dim);
  D.fbeg = int(fbeg);
  D.nf = int(nfc);
  D.wbeg = int(fbeg + nfc);
  D.nw = int(nwc);
  D.wrow = int(wrow);
  return SISPH_OK;
}

}  // namespace

extern "C" {

void sisph_default_case(sisph_case_params *q) {
  if (!q) return;
  memset(q, 0, sizeof(*q));
  q->h = 0.0;
  q->dt = 0.0;
  q->rho0 = 1.0;
  q->tol = 1e-2;
  q->max_iter = 1000;
  q->pgrad_symm = 0;
  q->free_surface = 0;
  q->ustar_slip = 1;
  q->pref_mode = SISPH_PREF_FIXED;
  q->p_ref = 0.0;
  q->gtvf_hfac = 1.0;
  q->gtvf_K = 1;
}

void sisph_default_options(sisph_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = SISPH_FP64;
  o->omega = 0.5;
  o->min_iter = 2;
  o->eta = 0.01;
  o->fs_ratio = 0.8;
  o->residual_form = 0;
  o->nbr_capacity = 0;
  o->skin = 0.15;
  o->block = 256;
  o->use_graph = 1;
  o->barrier_timeout_ms = 2000.0;
  o->debug_skip_barrier = 0;
  o->ppe_sync = 0;
  sisph_default_case(&o->physics);
}

const char *sisph_version(void) { return "sisph-gb300 0.1 (sm_103a)"; }

const char *sisph_last_error(sisph_t s) { return s ? s->err.c_str() : g_create_error.c_str(); }

int sisph_batch_create(int32_t ncases, const sisph_particles *parts, const sisph_case_params *params,
                       const sisph_options *opt_in, sisph_t *out) {
  NvtxScope nvtx("sisph_batch_create");
  if (!out) return fail(nullptr, SISPH_EINVAL, "out is NULL");
  *out = nullptr;
  if (ncases <= 0 || !parts || !params) return fail(nullptr, SISPH_EINVAL, "no cases");
  sisph_options opt;
  if (opt_in) opt = *opt_in;
  else sisph_default_options(&opt);
  if (opt.block < 64 || opt.block > 1024 || (opt.block % 32) != 0 || opt.block > 256)
    return fail(nullptr, SISPH_EINVAL, "block must be a multiple of 32 in [64, 256]");
  if (opt.precision != SISPH_FP64 && opt.precision != SISPH_MIXED)
    return fail(nullptr, SISPH_EINVAL, "precision must be SISPH_FP64 or SISPH_MIXED");
  if (!(opt.omega > 0.0 && opt.omega <= 1.0)) return fail(nullptr, SISPH_EINVAL, "omega must be in (0, 1]");
  if (opt.min_iter < 1) return fail(nullptr, SISPH_EINVAL, "min_iter must be >= 1");
  if (!(opt.skin >= 0.0 && opt.skin <= 1.0)) return fail(nullptr, SISPH_EINVAL, "skin must be in [0, 1]");
  if (opt.ppe_sync < 0 || opt.ppe_sync > 2) return fail(nullptr, SISPH_EINVAL, "ppe_sync must be 0, 1 or 2");
  const int dim = parts[0].dim;
  if (dim != 2 && dim != 3) return fail(nullptr, SISPH_EINVAL, "dim must be 2 or 3");
  int64_t ntot = 0, nftot = 0;
  for (int c = 0; c < ncases; ++c) {
    const sisph_particles &P = parts[c];
    const sisph_case_params &q = params[c];
    std::string cs = "case " + std::to_string(c) + ": ";
    if (P.dim != dim) return fail(nullptr, SISPH_EINVAL, cs + "all cases must share dim");
    if (P.n <= 0) return fail(nullptr, SISPH_EINVAL, cs + "n must be positive");
    if (!P.x || !P.y || (dim == 3 && !P.z) || !P.u || !P.v || (dim == 3 && !P.w) || !P.m)
      return fail(nullptr, SISPH_EINVAL, cs + "x, y, u, v, m (and z, w in 3D) are required");
    if (!(q.h > 0.0) || !(q.dt > 0.0) || !(q.rho0 > 0.0) || !(q.nu >= 0.0))
      return fail(nullptr, SISPH_EINVAL, cs + "h, dt, rho0 must be > 0 and nu >= 0");
    if (q.max_iter < 1 || q.gtvf_K < 1 || q.gtvf_K > 64)
      return fail(nullptr, SISPH_EINVAL, cs + "max_iter >= 1 and 1 <= gtvf_K <= 64");
    if (q.pref_mode < 0 || q.pref_mode > 2) return fail(nullptr, SISPH_EINVAL, cs + "bad pref_mode");
    if (!(q.gtvf_hfac > 0.0)) return fail(nullptr, SISPH_EINVAL, cs + "gtvf_hfac must be > 0");
    if (q.adaptive_dt != 0 && q.adaptive_dt != 1) return fail(nullptr, SISPH_EINVAL, cs + "adaptive_dt must be 0 or 1");
    if (q.ppe_solver != 0 && q.ppe_solver != 1) return fail(nullptr, SISPH_EINVAL, cs + "ppe_solver must be 0 or 1");
    for (int64_t i = 0; i < P.n; ++i) {
      int kd = P.kind ? P.kind[i] : 0;
      if (kd != SISPH_KIND_FLUID && kd != SISPH_KIND_WALL) return fail(nullptr, SISPH_EINVAL, cs + "bad kind");
      if (kd == SISPH_KIND_FLUID) ++nftot;
      if (!(P.m[i] > 0.0)) return fail(nullptr, SISPH_EINVAL, cs + "mass must be positive");
    }
    ntot += P.n;
  }
  if (ntot > kMaxParticles) return fail(nullptr, SISPH_EINVAL, "too many particles (max 2^26 - 1)");

  sisph_t s = new sisph_s();
  s->opt = opt;
  s->ncases = ncases;
  s->dim = dim;
  s->n = ntot;
  s->nf = nftot;
  s->nw = ntot - nftot;
  s->prm.assign(params, params + ncases);
  s->hc.resize(ncases);
  State &S = s->S;
  S.dim = dim;
  S.ncases = ncases;
  S.mixed = opt.precision == SISPH_MIXED;
  S.T = opt.block;
  S.n = int(ntot);
  S.nf = int(nftot);
  S.nw = int(ntot - nftot);
  S.omega = opt.omega;
  S.fs_ratio = opt.fs_ratio;
  S.eta = opt.eta;
  S.min_iter = opt.min_iter;
  S.residual_form = opt.residual_form;
  S.debug_skip_barrier = opt.debug_skip_barrier;
  S.ppe_sync = opt.ppe_sync;

  // static layout: per case [fluid | walls]; tiles never straddle a block
  std::vector<int> order;  // layout position -> caller index (global)
  order.reserve(ntot);
  std::vector<int> case_of(ntot), wall_at;
  long long key_base = 0;
  int64_t pos = 0, wrow = 0, off = 0;
  const int T = opt.block;
  int capmax = 0, scapmax = 0;
  for (int c = 0; c < ncases; ++c) {
    const sisph_particles &P = parts[c];
    int64_t nfc = 0;
    for (int64_t i = 0; i < P.n; ++i)
      if (!P.kind || P.kind[i] == SISPH_KIND_FLUID) { order.push_back(int(off + i)); ++nfc; }
    for (int64_t i = 0; i < P.n; ++i)
      if (P.kind && P.kind[i] == SISPH_KIND_WALL) order.push_back(int(off + i));
    int64_t nwc = P.n - nfc;
    CaseDev &D = s->hc[c];
    int rc = setup_case(s, c, P, params[c], pos, nfc, nwc, wrow, key_base, D);
    if (rc) {
      delete s;
      return rc;
    }
    key_base += 2 * D.slots;
    D.ftile = int(s->hft.size());
    for (int64_t b = 0; b < nfc; b += T) s->hft.push_back(Tile{int(pos + b), int(pos + std::min<int64_t>(nfc, b + T)), c, 0});
    D.nftile = int(s->hft.size()) - D.ftile;
    D.wtile = int(s->hwt.size());
    for (int64_t b = 0; b < nwc; b += T)
      s->hwt.push_back(Tile{int(pos + nfc + b), int(pos + nfc + std::min<int64_t>(nwc, b + T)), c, 1});
    D.nwtile = int(s->hwt.size()) - D.wtile;
    for (int64_t i = 0; i < P.n; ++i) case_of[pos + i] = c;
    for (int64_t i = 0; i < nwc; ++i) wall_at.push_back(int(pos + nfc + i));
    // neighbour capacity from the lattice count of the 3h ball
    int cap = opt.nbr_capacity;
    if (cap <= 0) {
      double mfl = 0.0;
      for (int64_t i = 0; i < P.n; ++i)
        if (!P.kind || P.kind[i] == SISPH_KIND_FLUID) { mfl = P.m[i]; break; }
      if (mfl <= 0.0) mfl = P.m[0];
      double dx = std::pow(mfl / params[c].rho0, 1.0 / dim);
      double rr = 3.0 * params[c].h / dx;
      double lat = dim == 2 ? M_PI * rr * rr : 4.0 / 3.0 * M_PI * rr * rr * rr;
      cap = int(std::ceil(1.5 * lat + 8.0));
      cap = (cap + 3) & ~3;
      cap = std::min(cap, 1024);
    }
    capmax = std::max(capmax, cap);
    // skin lists: the same headroom over the (3h + s) ball
    const double grow = std::pow((3.0 * params[c].h + D.skin) / (3.0 * params[c].h), double(dim));
    int scap = int(std::ceil(double(cap) * grow));
    scap = (scap + 3) & ~3;
    scapmax = std::max(scapmax, scap);
    pos += P.n;
    wrow += nwc;
    off += P.n;
    s->kmax = std::max(s->kmax, params[c].gtvf_K);
    s->adaptive = s->adaptive || params[c].adaptive_dt != 0;
    s->krylov = s->krylov || params[c].ppe_solver == 1;
  }
  if (s->krylov && ncases > 1024) {
    delete s;
    return fail(nullptr, SISPH_EINVAL, "BiCGStab cases: at most 1024 cases per handle");
  }
  if (key_base >= (1LL << 31) || key_base > (1LL << 26)) {
    delete s;
    return fail(nullptr, SISPH_EINVAL, "cell-key space too large; enlarge h or shrink the box");
  }
  S.K = key_base;
  S.cap = capmax;
  S.wcap = capmax;
  S.scap = scapmax;
  S.nft = int(s->hft.size());
  S.nwt = int(s->hwt.size());

  // device allocations
  cudaError_t e = cudaSuccess;
  auto A = [&](auto **p, size_t cnt) {
    if (e == cudaSuccess) e = dalloc(s, p, cnt);
  };
  const size_t N = size_t(ntot);
  CaseDev *dcases = nullptr;
  Tile *dft = nullptr, *dwt = nullptr;
  int *dcase_of = nullptr, *dwall_at = nullptr;
  A(&dcases, ncases);
  A(&dft, std::max(1, S.nft));
  A(&dwt, std::max(1, S.nwt));
  A(&dcase_of, N);
  A(&dwall_at, std::max<size_t>(1, wall_at.size()));
  A(&S.key, N);
  A(&S.slot, N);
  long long nbs = (S.K + 1 + 4095) / 4096 + 1;
  A(&S.hist, size_t(S.K + 1 + nbs));
  A(&S.perm, N);
  for (int k = 0; k < 3; ++k) {
    A(&S.x[k], N); A(&S.xn[k], N); A(&S.u[k], N); A(&S.ut[k], N);
    A(&S.bx[k], N); A(&S.bxn[k], N); A(&S.bu[k], N); A(&S.but[k], N);
    A(&S.xs[k], N); A(&S.us[k], N); A(&S.uw[k], N); A(&S.nrm[k], N); A(&S.nstar[k], N);
    A(&S.xref[k], N); A(&S.bxref[k], N);
    A(&S.vgt[k], N);
    if (!S.mixed) { A(&S.dg[0][k], N); A(&S.dg[1][k], N); }
  }
  A(&S.m, N); A(&S.rho, N); A(&S.p, N); A(&S.uid, N);
  A(&S.bm, N); A(&S.brho, N); A(&S.bp, N); A(&S.buid, N);
  A(&S.pf4, N);
  if (S.mixed) {
    A(&S.vf4, N); A(&S.utf4, N); A(&S.pf, N);
    A(&S.dgf[0], N); A(&S.dgf[1], N);
  }
  A(&S.nbr, ell_size(S.cap, (long long)N));
  A(&S.ncnt, N);
  A(&S.snbr, ell_size(S.scap, (long long)N));
  A(&S.sncnt, N);
  A(&S.wfin, N);
  A(&S.cell, N);
  A(&S.bcell, N);
  A(&S.need, ncases);
  A(&S.anyneed, 1);
  A(&S.force, 1);
  A(&S.nreb, size_t(ncases) + 1);
  A(&S.nbody, 1);
  const size_t rb = S.mixed ? sizeof(float) : sizeof(double);
  auto AR = [&](void **p, size_t cnt) {
    if (e != cudaSuccess) return;
    char *q = nullptr;
    e = dalloc(s, &q, cnt * rb);
    *p = q;
  };
  // one 8-byte slot per ELL entry: packed index + FP32 coefficient, or FP64
  if (e == cudaSuccess) {
    char *q = nullptr;
    e = dalloc(s, &q, ell_size(S.cap, (long long)N) * 8);
    S.coef = q;
  }
  A(&S.pcnt, N);
  AR(&S.prhs, N);
  AR(&S.pwd, N);
  for (int q = 0; q < 4; ++q) AR(&S.pb[q], N);
  A(&S.rhs_out, N);
  A(&S.diag_out, N);
  size_t NW = std::max<size_t>(1, size_t(s->nw));
  A(&S.wcnt, NW);
  A(&S.widx, ell_size(S.wcap, (long long)NW));
  AR(&S.wcoef, ell_size(S.wcap, (long long)NW));
  AR(&S.wsinv, NW);
  AR(&S.wh, NW);
  A(&S.tile_part, 8 * size_t(std::max(1, S.nft)));   // four sweeps in flight
  A(&S.tile_lam, size_t(std::max(1, S.nft)));
  A(&S.act, 2 * size_t(ncases));
  A(&S.iters, ncases); A(&S.pstat, ncases); A(&S.par, 5 * size_t(ncases));
  A(&S.dsw, ncases);
  int *dtile_of;
  A(&dtile_of, N);
  const size_t NT = size_t(std::max(1, S.nft + S.nwt));
  A(&S.deps, NT * kDepCap);
  A(&S.ndeps, NT);
  A(&S.tflag, NT);
  A(&S.resid, ncases); A(&S.lam, ncases);
  A(&S.iters_tot, ncases); A(&S.solves, ncases);
  A(&S.pref, ncases); A(&S.pref_set, ncases);
  A(&S.bar, 1);
  A(&S.tsim, ncases);
  A(&S.inact, ncases);
  if (s->krylov) {
    for (int q = 0; q < 6; ++q) AR(&S.kv[q], N);
    A(&S.kpart, 4 * size_t(std::max(1, S.nft)));
    A(&S.kscal, 8 * size_t(ncases));
  }
  if (s->adaptive) {
    for (int k = 0; k < 3; ++k) A(&S.fs1[k], N);
    A(&S.umax2, ncases);
    A(&S.fmax2, ncases);
  }
  A(&S.err, 1);
  A(&s->d_tmp, N);
  A(&s->d_tmp2, N);
  if (e != cudaSuccess) {
    sisph_destroy(s);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? SISPH_ENOMEM : SISPH_ECUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  }
  S.cases = dcases;
  S.ftiles = dft;
  S.wtiles = dwt;
  S.case_of = dcase_of;
  S.wall_at = dwall_at;
  S.tile_of = dtile_of;

  e = cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    sisph_destroy(s);
    return cuda_fail(nullptr, e, "stream");
  }
  s->stream = s->own_stream;

  // host staging in layout order
  std::vector<double> hb(N);
  std::vector<int> hi(N);
  auto up = [&](double *dst, std::vector<double> &v) {
    if (e == cudaSuccess) e = cudaMemcpy(dst, v.data(), N * sizeof(double), cudaMemcpyHostToDevice);
  };
  std::vector<int64_t> coff(ncases + 1, 0);
  for (int c = 0; c < ncases; ++c) coff[c + 1] = coff[c] + parts[c].n;
  std::vector<int> gcase(ntot);
  for (int c = 0; c < ncases; ++c)
    for (int64_t i = coff[c]; i < coff[c + 1]; ++i) gcase[i] = c;
  auto field = [&](int which, int comp, std::vector<double> &v) {
    for (size_t t = 0; t < N; ++t) {
      int g = order[t];
      int c = gcase[g];
      int64_t i = g - coff[c];
      const sisph_particles &P = parts[c];
      const sisph_case_params &q = params[c];
      bool wall = P.kind && P.kind[i] == SISPH_KIND_WALL;
      double val = 0.0;
      if (which == 0) {  // position, wrapped into periodic boxes
        const double *a = comp == 0 ? P.x : comp == 1 ? P.y : P.z;
        val = (comp < dim && a) ? a[i] : 0.0;
        if (comp < dim && P.periodic[comp]) {
          double L = P.hi[comp] - P.lo[comp];
          if (val >= P.hi[comp]) val -= L;
          else if (val < P.lo[comp]) val += L;
        }
      } else if (which == 1) {  // velocity (walls: prescribed)
        const double *a = comp == 0 ? P.u : comp == 1 ? P.v : P.w;
        const double *b = comp == 0 ? P.wall_u : comp == 1 ? P.wall_v : P.wall_w;
        if (comp < dim) val = wall ? (b ? b[i] : 0.0) : (a ? a[i] : 0.0);
      } else if (which == 2) {
        const double *b = comp == 0 ? P.wall_u : comp == 1 ? P.wall_v : P.wall_w;
        val = (wall && comp < dim && b) ? b[i] : 0.0;
      } else if (which == 3) val = P.m[i];
      else if (which == 4) val = (wall || !P.rho) ? q.rho0 : P.rho[i];
      else if (which == 5) val = P.p ? P.p[i] : 0.0;
      v[t] = val;
    }
  };
  for (int k = 0; k < 3; ++k) {
    field(0, k, hb);
    for (size_t t = 0; t < N; ++t)
      if (k < dim && order.size() && parts[gcase[order[t]]].periodic[k]) {
        const sisph_particles &P = parts[gcase[order[t]]];
        if (hb[t] < P.lo[k] || hb[t] >= P.hi[k]) {
          sisph_destroy(s);
          return fail(nullptr, SISPH_EINVAL, "a position lies more than one box length outside a periodic box");
        }
      }
    up(S.x[k], hb);
    up(S.xn[k], hb);
    field(1, k, hb);
    up(S.u[k], hb);
    up(S.ut[k], hb);
    field(2, k, hb);
    up(S.uw[k], hb);
  }
  field(3, 0, hb);
  up(S.m, hb);
  field(4, 0, hb);
  up(S.rho, hb);
  field(5, 0, hb);
  up(S.p, hb);
  for (size_t t = 0; t < N; ++t) hi[t] = order[t];
  if (e == cudaSuccess) e = cudaMemcpy(S.uid, hi.data(), N * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dcase_of, case_of.data(), N * sizeof(int), cudaMemcpyHostToDevice);
  {
    std::vector<int> tof(N, 0);
    for (int b = 0; b < S.nft; ++b)
      for (int q = s->hft[b].beg; q < s->hft[b].end; ++q) tof[q] = b;
    for (int b = 0; b < S.nwt; ++b)
      for (int q = s->hwt[b].beg; q < s->hwt[b].end; ++q) tof[q] = S.nft + b;
    if (e == cudaSuccess) e = cudaMemcpy(dtile_of, tof.data(), N * sizeof(int), cudaMemcpyHostToDevice);
    // no lists yet: until a PPE set-up builds them, a tile waits for its whole case
    std::vector<int> nd(NT, -1);
    if (e == cudaSuccess) e = cudaMemcpy(S.ndeps, nd.data(), NT * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && !wall_at.empty())
    e = cudaMemcpy(dwall_at, wall_at.data(), wall_at.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dcases, s->hc.data(), ncases * sizeof(CaseDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && S.nft) e = cudaMemcpy(dft, s->hft.data(), S.nft * sizeof(Tile), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && S.nwt) e = cudaMemcpy(dwt, s->hwt.data(), S.nwt * sizeof(Tile), cudaMemcpyHostToDevice);
  std::vector<double> pr(ncases);
  std::vector<int> ps(ncases);
  for (int c = 0; c < ncases; ++c) {
    pr[c] = params[c].p_ref;
    ps[c] = params[c].pref_mode == SISPH_PREF_TWICE_MAX_FIRST ? 0 : 1;
  }
  if (e == cudaSuccess) e = cudaMemcpy(S.pref, pr.data(), ncases * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(S.pref_set, ps.data(), ncases * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(S.iters_tot, 0, ncases * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(S.solves, 0, ncases * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(S.nreb, 0, (ncases + 1) * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(S.nbody, 0, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(S.tsim, 0, ncases * sizeof(double));
  if (e == cudaSuccess && s->adaptive) {
    e = cudaMemset(S.umax2, 0, ncases * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(S.fmax2, 0, ncases * sizeof(unsigned long long));
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemset(S.fs1[k], 0, N * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMemset(S.iters, 0, ncases * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(S.resid, 0, ncases * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(S.lam, 0, ncases * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(S.pstat, 0, ncases * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(S.err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(S.bar, 0, sizeof(Barrier));
  if (e == cudaSuccess) e = cudaMemset(S.wfin, 0, sizeof(int) * N);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemset(S.vgt[k], 0, N * sizeof(double));
  for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
    if (S.mixed) e = cudaMemset(S.dgf[p], 0, N * sizeof(float4));
    else
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemset(S.dg[p][k], 0, N * sizeof(double));
  }
  if (e != cudaSuccess) {
    sisph_destroy(s);
    return cuda_fail(nullptr, e, "upload");
  }
  // persistent-kernel grid: co-resident blocks, no more than there is work
  int dev = 0, nsm = 1, clk = 2000000;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  int bps = ppe_max_blocks_per_sm(S, S.T, false);
  if (bps < 1) bps = 1;
  int bps2 = ppe_max_blocks_per_sm(S, S.T, true);
  if (bps2 < 1) bps2 = 1;
  S.grid_cap_p2p = bps2 * nsm;
  {
    const int tiles = std::max(S.nft, S.nwt);
    S.p2p = (S.ppe_sync == 2 || (S.ppe_sync == 0 && S.grid_cap_p2p >= tiles + 1)) ? 1 : 0;
  }
  int want = std::max({S.nft, int((s->nw + S.T - 1) / S.T), ncases, 1});
  s->grid = std::min(want, bps * nsm);
  if (s->krylov) {
    int bk = krylov_max_blocks_per_sm(S, S.T);
    s->grid_k = std::max(1, std::min(want, std::max(1, bk) * nsm));
  }
  S.barrier_budget = (long long)(opt.barrier_timeout_ms * double(clk > 0 ? clk : 2000000));

  // first sort (places the walls for good), neighbour lists, wall normals
  e = force_rebuild(s);
  if (e == cudaSuccess) e = do_refresh(s, 0, true, true);
  if (e == cudaSuccess) e = launch_normals(S, mk_launch(s));
  if (e != cudaSuccess) {
    int rc = cuda_fail(nullptr, e, "initial neighbour build");
    sisph_destroy(s);
    return rc;
  }
  int rc = check_status(s, false);
  if (rc != SISPH_OK) {
    g_create_error = s->err;
    sisph_destroy(s);
    return rc;
  }
  *out = s;
  return SISPH_OK;
}

int sisph_create(const sisph_particles *particles, double h, double dt, double rho0, double nu,
                 const double g[3], const sisph_options *opt, sisph_t *out) {
  if (!particles) return fail(nullptr, SISPH_EINVAL, "particles is NULL");
  sisph_options o;
  if (opt) o = *opt;
  else sisph_default_options(&o);
  sisph_case_params q = o.physics;
  q.h = h;
  q.dt = dt;
  q.rho0 = rho0;
  q.nu = nu;
  for (int k = 0; k < 3; ++k) q.g[k] = g ? g[k] : 0.0;
  return sisph_batch_create(1, particles, &q, &o, out);
}

void sisph_destroy(sisph_t s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  destroy_graphs(s);
  for (auto &p : s->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto ev : s->pool) cudaEventDestroy(ev);
  for (void *p : s->allocs) cudaFree(p);
  if (s->copy) cudaStreamSynchronize(s->copy);
  if (s->d_stage) cudaFree(s->d_stage);
  for (auto ev : s->xev) cudaEventDestroy(ev);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->own_stream) cudaStreamDestroy(s->own_stream);
  if (s->side) cudaStreamDestroy(s->side);
  delete s;
}

int sisph_build_neighbors(sisph_t s) {
  NvtxScope nvtx("sisph_build_neighbors");
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  cudaError_t e = do_refresh(s, 0, false, true);
  if (e != cudaSuccess) return cuda_fail(s, e, "build_neighbors");
  return check_status(s, false);
}

int sisph_compute_density(sisph_t s) {
  NvtxScope nvtx("sisph_compute_density");
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  cudaError_t e = launch_density(s->S, mk_launch(s));
  if (e != cudaSuccess) return cuda_fail(s, e, "density");
  return check_status(s, false);
}

int sisph_ppe_solve(sisph_t s, double tol, int32_t max_iter, int32_t *iters, double *residual) {
  NvtxScope nvtx("sisph_ppe_solve");
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  if (max_iter < 1 || !(tol >= 0.0)) return fail(s, SISPH_EINVAL, "max_iter >= 1 and tol >= 0 required");
  // the solve's tolerance and cap on top of the device copy of the cases
  // (which holds the current, possibly adapted, time steps)
  std::vector<CaseDev> cur(s->hc.size()), hc;
  cudaError_t e = cudaMemcpyAsync(cur.data(), s->S.cases, cur.size() * sizeof(CaseDev),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  hc = cur;
  for (auto &c : hc) {
    c.tol = tol;
    c.max_iter = max_iter;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)s->S.cases, hc.data(), hc.size() * sizeof(CaseDev),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = do_ppe(s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)s->S.cases, cur.data(), cur.size() * sizeof(CaseDev),
                        cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "ppe_solve");
  int rc = check_status(s, true);
  std::vector<int> it(s->ncases);
  std::vector<double> rs(s->ncases);
  cudaMemcpy(it.data(), s->S.iters, s->ncases * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(rs.data(), s->S.resid, s->ncases * sizeof(double), cudaMemcpyDeviceToHost);
  if (iters) std::copy(it.begin(), it.end(), iters);
  if (residual) std::copy(rs.begin(), rs.end(), residual);
  drain_profile(s);
  return rc;
}

int sisph_step(sisph_t s, int32_t nsteps) {
  NvtxScope nvtx("sisph_step");
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  if (nsteps < 0) return fail(s, SISPH_EINVAL, "nsteps must be >= 0");
  bool use_graph = s->opt.use_graph && !(s->profiling && s->prof_only.empty()) && !s->graph_failed;
  cudaError_t e = cudaSuccess;
  for (int st = 0; st < nsteps && e == cudaSuccess; ++st) {
    if (use_graph && !s->gexec) {
      // Capture one step (recorded, not run).
      const int64_t l0 = s->launches;
      cudaGraph_t g = nullptr;
      cudaError_t ec = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
      if (ec == cudaSuccess) {
        s->capturing = true;
        cudaError_t es = do_step(s);
        s->capturing = false;
        ec = cudaStreamEndCapture(s->stream, &g);
        if (es != cudaSuccess) ec = es;
      }
      if (ec == cudaSuccess) ec = cudaGraphInstantiate(&s->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      s->graph_kernels = int(s->launches - l0);
      s->launches = l0;
      if (ec != cudaSuccess && !s->no_conditional) {
        // no conditional nodes here: capture again with the rebuild group
        // launched unconditionally (its kernels return at once when idle)
        cudaGetLastError();
        s->gexec = nullptr;
        for (auto &q : s->gsites) {
          cudaEventDestroy(q.a);
          cudaEventDestroy(q.b);
        }
        s->gsites.clear();
        s->no_conditional = true;
        s->err = std::string("conditional graph nodes unavailable: ") + cudaGetErrorString(ec);
        --st;
        continue;
      }
      if (ec != cudaSuccess) {
        cudaGetLastError();
        s->gexec = nullptr;
        for (auto &q : s->gsites) {
          cudaEventDestroy(q.a);
          cudaEventDestroy(q.b);
        }
        s->gsites.clear();
        s->graph_failed = true;
        use_graph = false;
        s->err = std::string("CUDA graph capture unavailable, using direct launches: ") + cudaGetErrorString(ec);
      }
    }
    if (use_graph) {
      e = cudaGraphLaunch(s->gexec, s->stream);
      s->launches += s->graph_kernels;
      if (s->profiling) drain_graph_sites(s);
      continue;
    }
    e = do_step(s);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "step");
  int rc = check_status(s, true);
  drain_profile(s);
  return rc;
}

// Device source of a readable field (nullptr for the GTVF displacement,
// which is scattered from its own buffers); false for an unknown field.
static bool get_source(sisph_t s, int32_t field, const void **src) {
  State &S = s->S;
  *src = nullptr;
  switch (field) {
    case SISPH_F_X: case SISPH_F_Y: case SISPH_F_Z: *src = S.x[field - SISPH_F_X]; return true;
    case SISPH_F_U: case SISPH_F_V: case SISPH_F_W: *src = S.u[field - SISPH_F_U]; return true;
    case SISPH_F_UT: case SISPH_F_VT: case SISPH_F_WT: *src = S.ut[field - SISPH_F_UT]; return true;
    case SISPH_F_P: *src = S.p; return true;
    case SISPH_F_RHO: *src = S.rho; return true;
    case SISPH_F_M: *src = S.m; return true;
    case SISPH_F_NX: case SISPH_F_NY: case SISPH_F_NZ: *src = S.nrm[field - SISPH_F_NX]; return true;
    case SISPH_F_RHS: *src = S.rhs_out; return true;
    case SISPH_F_DIAG: *src = S.diag_out; return true;
    case SISPH_F_DX: case SISPH_F_DY: case SISPH_F_DZ: return true;
    case SISPH_F_NSKIN: *src = S.sncnt; return true;
    case SISPH_F_NCOUNT: *src = S.ncnt; return true;
    default: return false;
  }
}

// Scatter one field into caller order in tmp (n doubles) on the library's
// stream.
static cudaError_t queue_scatter(sisph_t s, int32_t field, const void *src, double *tmp) {
  State &S = s->S;
  Launch L = mk_launch(s);
  L.before = nullptr;
  L.after = nullptr;
  if (field >= SISPH_F_DX && field <= SISPH_F_DZ) return launch_scatter_disp(S, L, field - SISPH_F_DX, tmp);
  if (field == SISPH_F_NSKIN || field == SISPH_F_NCOUNT) return launch_scatter_field(S, L, src, 2, 0, 0, tmp);
  return launch_scatter_field(S, L, src, 0, 0, 0, tmp);
}

// Scatter one field into caller order in d_tmp and queue its copy to out.
static cudaError_t queue_get(sisph_t s, int32_t field, const void *src, double *out) {
  cudaError_t e = queue_scatter(s, field, src, s->d_tmp);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, s->d_tmp, size_t(s->n) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  return e;
}

// Staging for nf fields (grown on demand; the previous call has finished
// with it, since every get/set waits for its copies), the copy stream and
// nf + 1 ordering events.
static cudaError_t ensure_stage(sisph_t s, int nf) {
  cudaError_t e = cudaSuccess;
  if (!s->copy) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess && s->stage_fields < nf) {
    if (s->d_stage) cudaFree(s->d_stage);
    s->d_stage = nullptr;
    s->stage_fields = 0;
    e = cudaMalloc(&s->d_stage, size_t(nf) * size_t(s->n) * sizeof(double));
    if (e == cudaSuccess) s->stage_fields = nf;
  }
  while (e == cudaSuccess && int(s->xev.size()) < nf + 1) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) s->xev.push_back(ev);
  }
  return e;
}

int sisph_get(sisph_t s, int32_t field, double *out) {
  if (!valid_handle(s) || !out) return fail(s, SISPH_EINVAL, "invalid handle or output");
  const void *src = nullptr;
  if (!get_source(s, field, &src)) return fail(s, SISPH_EINVAL, "unknown field");
  cudaError_t e = queue_get(s, field, src, out);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "get");
  return SISPH_OK;
}

int sisph_get_many(sisph_t s, int32_t nfields, const int32_t *fields, double *const *out) {
  if (!valid_handle(s) || nfields < 0 || (nfields > 0 && (!fields || !out)))
    return fail(s, SISPH_EINVAL, "invalid handle, count or arrays");
  std::vector<const void *> src(size_t(std::max(nfields, 1)));
  for (int k = 0; k < nfields; ++k) {
    if (!out[k]) return fail(s, SISPH_EINVAL, "a NULL output array");
    if (!get_source(s, fields[k], &src[k])) return fail(s, SISPH_EINVAL, "unknown field");
  }
  // field k: scatter into its staging column on the library's stream, then
  // its copy to the host on the copy stream, which waits for that scatter
  // only, so the copy of field k overlaps the scatter of field k + 1
  cudaError_t e = nfields > 0 ? ensure_stage(s, nfields) : cudaSuccess;
  const size_t bytes = size_t(s->n) * sizeof(double);
  for (int k = 0; k < nfields && e == cudaSuccess; ++k) {
    double *st = s->d_stage + size_t(k) * size_t(s->n);
    e = queue_scatter(s, fields[k], src[k], st);
    if (e == cudaSuccess) e = cudaEventRecord(s->xev[k], s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy, s->xev[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out[k], st, bytes, cudaMemcpyDeviceToHost, s->copy);
  }
  if (e == cudaSuccess && nfields > 0) e = cudaStreamSynchronize(s->copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "get_many");
  return SISPH_OK;
}

// Device destination of a writable field; false for an unknown or read-only
// field or a third component in 2D.
static bool set_target(sisph_t s, int32_t field, double **dst) {
  State &S = s->S;
  *dst = nullptr;
  switch (field) {
    case SISPH_F_X: case SISPH_F_Y: case SISPH_F_Z: *dst = S.x[field - SISPH_F_X]; break;
    case SISPH_F_U: case SISPH_F_V: case SISPH_F_W: *dst = S.u[field - SISPH_F_U]; break;
    case SISPH_F_UT: case SISPH_F_VT: case SISPH_F_WT: *dst = S.ut[field - SISPH_F_UT]; break;
    case SISPH_F_P: *dst = S.p; break;
    case SISPH_F_RHO: *dst = S.rho; break;
    default: return false;
  }
  if ((field == SISPH_F_Z || field == SISPH_F_W || field == SISPH_F_WT) && s->dim == 2) return false;
  return true;
}

// Queue the copy of one field into d_tmp and its gather into the sorted
// order (the stream orders the next copy after this gather).
static cudaError_t queue_set(sisph_t s, int32_t field, double *dst, const double *in) {
  Launch L = mk_launch(s);
  L.before = nullptr;
  L.after = nullptr;
  cudaError_t e = cudaMemcpyAsync(s->d_tmp, in, size_t(s->n) * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  // positions: fluid that moved past half the skin is re-sorted by the next
  // refresh's own check; a wall that moved forces every case to be rebuilt
  if (e == cudaSuccess) e = launch_gather_field(s->S, L, s->d_tmp, dst, field <= SISPH_F_Z);
  return e;
}

int sisph_set(sisph_t s, int32_t field, const double *in) {
  if (!valid_handle(s) || !in) return fail(s, SISPH_EINVAL, "invalid handle or input");
  double *dst = nullptr;
  if (!set_target(s, field, &dst)) return fail(s, SISPH_EINVAL, "field is read-only, unknown or not in 2D");
  Launch L = mk_launch(s);
  L.before = nullptr;
  L.after = nullptr;
  cudaError_t e = queue_set(s, field, dst, in);
  if (e == cudaSuccess) e = launch_refresh_mirrors(s->S, L);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "set");
  return SISPH_OK;
}

int sisph_set_many(sisph_t s, int32_t nfields, const int32_t *fields, const double *const *in) {
  if (!valid_handle(s) || nfields < 0 || (nfields > 0 && (!fields || !in)))
    return fail(s, SISPH_EINVAL, "invalid handle, count or arrays");
  std::vector<double *> dst(size_t(std::max(nfields, 1)));
  for (int k = 0; k < nfields; ++k) {
    if (!in[k]) return fail(s, SISPH_EINVAL, "a NULL input array");
    if (!set_target(s, fields[k], &dst[k]))
      return fail(s, SISPH_EINVAL, "field is read-only, unknown or not in 2D");
  }
  Launch L = mk_launch(s);
  L.before = nullptr;
  L.after = nullptr;
  // field k: its copy into its staging column on the copy stream (after the
  // work already queued on the library's stream), then its gather into the
  // sorted order on the library's stream, which waits for that copy only, so
  // the gather of field k overlaps the copy of field k + 1
  cudaError_t e = nfields > 0 ? ensure_stage(s, nfields) : cudaSuccess;
  const size_t bytes = size_t(s->n) * sizeof(double);
  if (e == cudaSuccess && nfields > 0) e = cudaEventRecord(s->xev[nfields], s->stream);
  if (e == cudaSuccess && nfields > 0) e = cudaStreamWaitEvent(s->copy, s->xev[nfields], 0);
  for (int k = 0; k < nfields && e == cudaSuccess; ++k) {
    double *st = s->d_stage + size_t(k) * size_t(s->n);
    e = cudaMemcpyAsync(st, in[k], bytes, cudaMemcpyHostToDevice, s->copy);
    if (e == cudaSuccess) e = cudaEventRecord(s->xev[k], s->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->xev[k], 0);
    // positions: a wall that moved forces every case to be rebuilt
    if (e == cudaSuccess) e = launch_gather_field(s->S, L, st, dst[k], fields[k] <= SISPH_F_Z);
  }
  if (e == cudaSuccess && nfields > 0) e = launch_refresh_mirrors(s->S, L);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "set_many");
  return SISPH_OK;
}

int sisph_neighbors(sisph_t s, int32_t *counts, int32_t *idx, int64_t idx_cap, int64_t *total) {
  if (!valid_handle(s) || !counts) return fail(s, SISPH_EINVAL, "invalid handle or counts");
  const size_t N = size_t(s->n);
  std::vector<int> cnt(N), uid(N);
  std::vector<unsigned> nbr(ell_size(s->S.cap, (long long)N));
  // the exact lists at the current positions (a step's own refreshes leave
  // out the pairs at the rim of the support)
  cudaError_t e = do_refresh(s, 0, false, true);
  if (e != cudaSuccess) return cuda_fail(s, e, "neighbors");
  const int rc = check_status(s, false);
  if (rc != SISPH_OK) return rc;
  e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), s->S.ncnt, N * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(uid.data(), s->S.uid, N * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && idx)
    e = cudaMemcpy(nbr.data(), s->S.nbr, nbr.size() * sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(s, e, "neighbors");
  std::vector<int> at(N);
  int64_t tot = 0;
  for (size_t i = 0; i < N; ++i) {
    counts[uid[i]] = cnt[i];
    at[uid[i]] = int(i);
    tot += cnt[i];
  }
  if (total) *total = tot;
  if (!idx) return SISPH_OK;
  if (tot > idx_cap) return fail(s, SISPH_EINVAL, "idx_cap too small");
  int64_t pos = 0;
  std::vector<int> row;
  for (size_t u = 0; u < N; ++u) {
    int i = at[u];
    row.clear();
    for (int k = 0; k < cnt[i]; ++k) row.push_back(uid[nbr[ell_at(s->S.cap, k, i)] & kIdxMask]);
    std::sort(row.begin(), row.end());
    for (int v : row) idx[pos++] = v;
  }
  return SISPH_OK;
}

int sisph_batch_step(sisph_t s, int32_t nsteps, int32_t *iters_per_case) {
  NvtxScope nvtx("sisph_batch_step");
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  const int nc = s->ncases;
  std::vector<long long> t0(nc), t1(nc);
  if (iters_per_case) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMemcpy(t0.data(), s->S.iters_tot, nc * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "batch_step");
  }
  const int rc = sisph_step(s, nsteps);
  if (rc != SISPH_OK && rc != SISPH_ENOTCONVERGED) return rc;
  if (iters_per_case) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMemcpy(t1.data(), s->S.iters_tot, nc * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "batch_step");
    for (int c = 0; c < nc; ++c) iters_per_case[c] = int32_t(t1[c] - t0[c]);
  }
  return rc;
}

int sisph_stats(sisph_t s, sisph_case_stats *st) {
  if (!valid_handle(s) || !st) return fail(s, SISPH_EINVAL, "invalid handle or stats");
  int nc = s->ncases;
  std::vector<int> it(nc), ps(nc);
  std::vector<double> rs(nc), lm(nc), pr(nc);
  std::vector<long long> tot(nc), sv(nc), rb(nc);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  const State &S = s->S;
  if (e == cudaSuccess) e = cudaMemcpy(it.data(), S.iters, nc * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ps.data(), S.pstat, nc * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(rs.data(), S.resid, nc * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(lm.data(), S.lam, nc * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(pr.data(), S.pref, nc * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(tot.data(), S.iters_tot, nc * sizeof(long long), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(sv.data(), S.solves, nc * sizeof(long long), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(rb.data(), S.nreb, nc * sizeof(long long), cudaMemcpyDeviceToHost);
  std::vector<CaseDev> cd(nc);
  std::vector<double> ts(nc);
  if (e == cudaSuccess) e = cudaMemcpy(cd.data(), S.cases, nc * sizeof(CaseDev), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(ts.data(), S.tsim, nc * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(s, e, "stats");
  for (int c = 0; c < nc; ++c) {
    st[c].iters = it[c];
    st[c].status = ps[c];
    st[c].residual = rs[c];
    st[c].lambda = lm[c];
    st[c].p_ref = pr[c];
    st[c].total_iters = tot[c];
    st[c].solves = sv[c];
    st[c].rebuilds = rb[c];
    st[c].dt = cd[c].dt;
    st[c].time = ts[c];
  }
  return SISPH_OK;
}

int sisph_info(sisph_t s, int64_t *n, int64_t *n_fluid, int32_t *ncases, int32_t *cap) {
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  if (n) *n = s->n;
  if (n_fluid) *n_fluid = s->nf;
  if (ncases) *ncases = s->ncases;
  if (cap) *cap = s->S.cap;
  return SISPH_OK;
}

int sisph_set_stream(sisph_t s, void *cuda_stream) {
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  cudaStreamSynchronize(s->stream);
  destroy_graphs(s);
  s->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : s->own_stream;
  return SISPH_OK;
}

int sisph_profile_enable(sisph_t s, int32_t on, const char *only) {
  if (!valid_handle(s)) return fail(s, SISPH_EINVAL, "invalid handle");
  drain_profile(s);
  std::string o = (on && only) ? std::string(only) : std::string();
  if (o != s->prof_only || (on != 0) != s->profiling) destroy_graphs(s);  // recapture
  s->profiling = on != 0;
  s->prof_only = o;
  s->prof_set.clear();
  for (size_t a = 0; a <= o.size() && !o.empty();) {
    size_t b = o.find(',', a);
    if (b == std::string::npos) b = o.size();
    if (b > a) s->prof_set.push_back(o.substr(a, b - a));
    a = b + 1;
  }
  if (on) s->prof.clear();
  return SISPH_OK;
}

int sisph_profile_get(sisph_t s, const char *kernel, int64_t *launches, double *total_ms, double *units) {
  if (!valid_handle(s) || !kernel) return fail(s, SISPH_EINVAL, "invalid handle or name");
  drain_profile(s);
  auto it = s->prof.find(kernel);
  ProfRec r;
  if (it != s->prof.end()) r = it->second;
  if (launches) *launches = r.launches;
  if (total_ms) *total_ms = r.ms;
  if (units) *units = r.units;
  return SISPH_OK;
}

int64_t sisph_launch_count(sisph_t s) {
  if (!valid_handle(s)) return 0;
  // kernels launched from the host, plus the rebuild groups that ran inside
  // conditional nodes of replayed step graphs (counted on the device)
  long long body = 0;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
      cudaMemcpy(&body, s->S.nbody, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    body = 0;
  }
  return s->launches + int64_t(kRebuildKernels) * body;
}

static const int kCkptFields[] = {SISPH_F_X, SISPH_F_Y, SISPH_F_Z, SISPH_F_U, SISPH_F_V, SISPH_F_W,
                                  SISPH_F_UT, SISPH_F_VT, SISPH_F_WT, SISPH_F_P, SISPH_F_RHO};

// A checkpoint holds the state in the caller's order, the background
// pressures and, so that a resumed run sorts and sums exactly as the saved
// one would have, the rebuild positions of the skin lists and whether a
// forced rebuild was pending.
static int copy_out(sisph_t s, const double *src, double *host) {
  Launch L = mk_launch(s);
  L.before = nullptr;
  L.after = nullptr;
  cudaError_t e = launch_scatter_field(s->S, L, src, 0, 0, 0, s->d_tmp);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, s->d_tmp, size_t(s->n) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? SISPH_OK : cuda_fail(s, e, "checkpoint read");
}

static int copy_in(sisph_t s, const double *host, double *dst) {
  Launch L = mk_launch(s);
  L.before = nullptr;
  L.after = nullptr;
  cudaError_t e = cudaMemcpyAsync(s->d_tmp, host, size_t(s->n) * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = launch_gather_field(s->S, L, s->d_tmp, dst, false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? SISPH_OK : cuda_fail(s, e, "checkpoint write");
}

int sisph_save(sisph_t s, const char *path) {
  NvtxScope nvtx("sisph_save");
  if (!valid_handle(s) || !path) return fail(s, SISPH_EINVAL, "invalid handle or path");
  FILE *f = fopen(path, "wb");
  if (!f) return fail(s, SISPH_EINVAL, std::string("cannot open ") + path);
  const char magic[8] = {'S', 'I', 'S', 'P', 'H', 'C', 'K', '3'};
  int64_t hdr[3] = {s->n, s->ncases, s->dim};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1;
  std::vector<double> buf(size_t(s->n));
  for (int fld : kCkptFields) {
    if (s->dim == 2 && (fld == SISPH_F_Z || fld == SISPH_F_W || fld == SISPH_F_WT)) continue;
    int rc = sisph_get(s, fld, buf.data());
    if (rc) { fclose(f); return rc; }
    ok = ok && fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  }
  for (int k = 0; k < s->dim; ++k) {
    int rc = copy_out(s, s->S.xref[k], buf.data());
    if (rc) { fclose(f); return rc; }
    ok = ok && fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  }
  std::vector<double> pr(s->ncases);
  std::vector<int> ps(s->ncases);
  int force = 0;
  cudaMemcpy(pr.data(), s->S.pref, s->ncases * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(ps.data(), s->S.pref_set, s->ncases * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&force, s->S.force, sizeof(int), cudaMemcpyDeviceToHost);
  int32_t pending = force != 0;
  // per case: the next time step (adaptive) and the simulated time
  std::vector<CaseDev> cd(s->ncases);
  std::vector<double> dts(s->ncases), ts(s->ncases);
  cudaMemcpy(cd.data(), s->S.cases, s->ncases * sizeof(CaseDev), cudaMemcpyDeviceToHost);
  cudaMemcpy(ts.data(), s->S.tsim, s->ncases * sizeof(double), cudaMemcpyDeviceToHost);
  for (int c = 0; c < s->ncases; ++c) dts[c] = cd[c].dt;
  ok = ok && fwrite(pr.data(), sizeof(double), pr.size(), f) == pr.size();
  ok = ok && fwrite(ps.data(), sizeof(int), ps.size(), f) == ps.size();
  ok = ok && fwrite(&pending, sizeof(pending), 1, f) == 1;
  ok = ok && fwrite(dts.data(), sizeof(double), dts.size(), f) == dts.size();
  ok = ok && fwrite(ts.data(), sizeof(double), ts.size(), f) == ts.size();
  fclose(f);
  return ok ? SISPH_OK : fail(s, SISPH_EINVAL, "write failed");
}

int sisph_load(sisph_t s, const char *path) {
  NvtxScope nvtx("sisph_load");
  if (!valid_handle(s) || !path) return fail(s, SISPH_EINVAL, "invalid handle or path");
  FILE *f = fopen(path, "rb");
  if (!f) return fail(s, SISPH_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int64_t hdr[3];
  bool ok = fread(magic, 1, 8, f) == 8 && fread(hdr, sizeof(hdr), 1, f) == 1;
  if (!ok || memcmp(magic, "SISPHCK3", 8) != 0 || hdr[0] != s->n || hdr[1] != s->ncases || hdr[2] != s->dim) {
    fclose(f);
    return fail(s, SISPH_EINVAL, "checkpoint does not match this handle");
  }
  std::vector<double> buf(size_t(s->n));
  for (int fld : kCkptFields) {
    if (s->dim == 2 && (fld == SISPH_F_Z || fld == SISPH_F_W || fld == SISPH_F_WT)) continue;
    if (fread(buf.data(), sizeof(double), buf.size(), f) != buf.size()) { fclose(f); return fail(s, SISPH_EINVAL, "short checkpoint"); }
    int rc = sisph_set(s, fld, buf.data());
    if (rc) { fclose(f); return rc; }
  }
  for (int k = 0; k < s->dim; ++k) {
    if (fread(buf.data(), sizeof(double), buf.size(), f) != buf.size()) { fclose(f); return fail(s, SISPH_EINVAL, "short checkpoint"); }
    int rc = copy_in(s, buf.data(), s->S.xref[k]);
    if (rc) { fclose(f); return rc; }
  }
  std::vector<double> pr(s->ncases);
  std::vector<int> ps(s->ncases);
  int32_t pending = 0;
  std::vector<double> dts(s->ncases), ts(s->ncases);
  ok = fread(pr.data(), sizeof(double), pr.size(), f) == pr.size() &&
       fread(ps.data(), sizeof(int), ps.size(), f) == ps.size() && fread(&pending, sizeof(pending), 1, f) == 1 &&
       fread(dts.data(), sizeof(double), dts.size(), f) == dts.size() &&
       fread(ts.data(), sizeof(double), ts.size(), f) == ts.size();
  fclose(f);
  if (!ok) return fail(s, SISPH_EINVAL, "short checkpoint");
  cudaError_t e = cudaMemcpy(s->S.pref, pr.data(), s->ncases * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->S.pref_set, ps.data(), s->ncases * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->S.tsim, ts.data(), s->ncases * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    std::vector<CaseDev> cd(s->ncases);
    e = cudaMemcpy(cd.data(), s->S.cases, s->ncases * sizeof(CaseDev), cudaMemcpyDeviceToHost);
    for (int c = 0; c < s->ncases; ++c) cd[c].dt = dts[c];
    if (e == cudaSuccess) e = cudaMemcpy((void *)s->S.cases, cd.data(), s->ncases * sizeof(CaseDev), cudaMemcpyHostToDevice);
  }
  // sort and skin lists as they were at the saved rebuild positions (or at
  // the current ones if a rebuild was pending), then the refresh the saved
  // run would have made next
  if (e == cudaSuccess) e = force_rebuild(s, pending ? 1 : 2);
  if (e == cudaSuccess) e = do_refresh(s, 0, false);
  if (e == cudaSuccess) e = do_refresh(s, 0, false);
  if (e != cudaSuccess) return cuda_fail(s, e, "load");
  return check_status(s, false);
}

}  // extern "C"
