// C ABI of include/sqsm.h: argument validation, plans (per batch layout),
// workspaces (per plan, dtype and nx) and captured graphs, all owned by the
// context.  Host code only builds index tables and enqueues kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <initializer_list>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sqsm.h"
#include "dispatch.h"

using namespace sqsm;

namespace {

struct Alloc {
  std::vector<void*> ptrs;
  ~Alloc() {
    for (void* p : ptrs) cudaFree(p);
  }
  void* get(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
};

struct Workspace {
  Alloc mem;
  ScanBuffers filt, smth;
  double* partial = nullptr;
  void* mf = nullptr;        // filter outputs when the caller wants none / IPLS
  void* Nf = nullptr;
  void* gamma = nullptr;     // IPLS linearised model, PRec<5, 2> records per step
  void* frows = nullptr;     // IPLS filter output, packed rows
  void* nrows = nullptr;     // IPLS nominal trajectory, packed rows
  int* tol_words = nullptr;  // tolerance mode: [0] iterations run, [1] continue flag,
                             // [2] largest change of the nominal means (float bits)
  void* params = nullptr;    // IPLS model constants
  void* dm0 = nullptr;       // IPLS prior mean in deviation coordinates
  void* n0fac = nullptr;     // prior factors chol(P0) when N0 arguments are covariances
  void* prevrows = nullptr;  // refinement: nominal rows before the last smoother pass
  double* partial2 = nullptr;   // refinement passes' log-likelihood partials
  void* etab = nullptr;      // refinement: E_k of every state row (mean-only passes)
  void* ftab = nullptr;      // refinement: the filter's stored combine factors (mean-only
                             // upper levels; null where the plan has none)
  bool ipls_ready = false;
  // NLL + gradient
  AdjArgs adj{};
  ScanBuffers adj_scan;
  bool adj_ready = false;
};

struct Plan {
  Alloc mem;
  int B = 0;
  int L0 = 0, R = 0;
  std::vector<int64_t> offsets;
  int64_t* d_offsets = nullptr;
  LevelSet filt, smth;
  std::map<std::pair<int, int>, std::unique_ptr<Workspace>> ws;   // (dtype, nx)
};

struct GraphKey {
  const Plan* plan;
  int dtype, lin, M, prof, adj;     // adj: adjoint iterations + 1 (0 = smoother only)
  const void *y, *m0, *N0, *ims, *iNs, *ms, *Ns, *ll;
  double tol = -1.0;                // tolerance mode (M = iteration cap), else -1
  const void* iters = nullptr;
  int kind = SQSM_MODEL_CT_BEARINGS;
  const void *grad = nullptr, *change = nullptr;   // NLL + gradient outputs
  const void* ichange = nullptr;
  int prior_cov = 0;                // N0 holds prior covariances
  bool operator<(const GraphKey& o) const {
    return std::tie(plan, dtype, lin, M, prof, adj, y, m0, N0, ims, iNs, ms, Ns, ll, tol, iters,
                    kind, grad, change, ichange, prior_cov) <
           std::tie(o.plan, o.dtype, o.lin, o.M, o.prof, o.adj, o.y, o.m0, o.N0, o.ims, o.iNs,
                    o.ms, o.Ns, o.ll, o.tol, o.iters, o.kind, o.grad, o.change, o.ichange,
                    o.prior_cov);
  }
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  std::unique_ptr<Prof> prof;   // events recorded by the instrumented graph
};

}  // namespace

// Workload shape an autotuned scan shape is stored for.
struct TuneKey {
  int dtype, lin;
  int64_t batch;
  int lg_total, lg_max;   // floor(log2) of the total and of the longest length
  bool operator<(const TuneKey& o) const {
    return std::tie(dtype, lin, batch, lg_total, lg_max) <
           std::tie(o.dtype, o.lin, o.batch, o.lg_total, o.lg_max);
  }
};

struct sqsm_ctx {
  int device = 0;
  int sm_count = 152;
  std::map<TuneKey, std::pair<int, int>> tuned;   // autotuned (leaf_chunk, radix)
  sqsm_options opt{};
  std::string err;
  int* d_status = nullptr;
  double* d_group = nullptr;      // one group's nll, grad[4], changes (grouped nll_grad)
  cudaStream_t capture_stream = nullptr;   // graphs are recorded here
  cudaStream_t body_stream = nullptr;      // bodies of conditional graph nodes
  std::vector<std::unique_ptr<Plan>> plans;
  std::map<GraphKey, GraphEntry> graphs;
  bool prof_on = false;
  Prof call_prof;                 // events of the last non-graph call
  Prof* last_prof = nullptr;      // events of the last profiled call
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int fail(sqsm_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(sqsm_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, SQSM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Adaptive plans fold a level with more items than this (4 per thread)
// rather than chunk-scanning it: its folds alone give > 40k threads, enough
// to fill the GPU.
constexpr int64_t kFoldAboveItems = 160000;

// Levels of a segmented scan whose level-0 items are `counts[b]` per
// sequence: chunks of L0 items at the leaf, then chunks of R items (or, for
// R == 0, of 4 or 32 items chosen per level) until each sequence has one item.

bool build_levels(Plan& p, const std::vector<int64_t>& counts0, LevelSet& L) {
  std::vector<int64_t> counts = counts0;
  L.B = (int)counts0.size();
  int level = 0;
  int64_t total = 0;
  for (int64_t v : counts) total += v;
  L.n_items.push_back(total);
  L.cs.assign(1, 0);
  for (;;) {
    int64_t size = level == 0 ? p.L0 : p.R;
    if (level > 0) {
      bool cs = false;
      if (p.R == 0) {                       // adaptive: see get_plan
        int64_t items = 0;
        for (int64_t v : counts) items += v;
        cs = items <= kFoldAboveItems;
        size = cs ? kChunkScan : 4;
      }
      L.cs.push_back(cs ? 1 : 0);
    }
    std::vector<int64_t> first;
    std::vector<int32_t> count, seq;
    std::vector<int64_t> next(counts.size());
    int64_t item_off = 0;
    bool all_one = true;
    for (size_t b = 0; b < counts.size(); ++b) {
      const int64_t nch = (counts[b] + size - 1) / size;
      for (int64_t j = 0; j < nch; ++j) {
        first.push_back(item_off + j * size);
        count.push_back((int32_t)std::min<int64_t>(size, counts[b] - j * size));
        seq.push_back((int32_t)b);
      }
      next[b] = nch;
      if (nch != 1) all_one = false;
      item_off += counts[b];
    }
    DevLevel d;
    d.n_chunks = (int64_t)first.size();
    int64_t* df = (int64_t*)p.mem.get(sizeof(int64_t) * first.size());
    int32_t* dc = (int32_t*)p.mem.get(sizeof(int32_t) * count.size());
    int32_t* ds = (int32_t*)p.mem.get(sizeof(int32_t) * seq.size());
    if (!df || !dc || !ds) return false;
    cudaMemcpy(df, first.data(), sizeof(int64_t) * first.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(dc, count.data(), sizeof(int32_t) * count.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(ds, seq.data(), sizeof(int32_t) * seq.size(), cudaMemcpyHostToDevice);
    d.first = df;
    d.count = dc;
    d.seq = ds;
    L.lv.push_back(d);
    L.n_items.push_back(d.n_chunks);
    // items of level+1 per sequence = chunks per sequence at this level
    {
      std::vector<int64_t> so(counts.size() + 1, 0);
      int64_t mx = 0;
      for (size_t b = 0; b < counts.size(); ++b) {
        so[b + 1] = so[b] + next[b];
        mx = std::max<int64_t>(mx, next[b]);
      }
      int64_t* dso = (int64_t*)p.mem.get(sizeof(int64_t) * so.size());
      if (!dso) return false;
      cudaMemcpy(dso, so.data(), sizeof(int64_t) * so.size(), cudaMemcpyHostToDevice);
      if (L.seq_item_off.empty()) {   // index 0 (steps) is not used
        L.seq_item_off.push_back(nullptr);
        L.max_seq_items.push_back(0);
      }
      L.seq_item_off.push_back(dso);
      L.max_seq_items.push_back(mx);
    }
    if (level == 0) {
      std::vector<int64_t> lco(counts.size() + 1, 0);
      for (size_t b = 0; b < counts.size(); ++b) lco[b + 1] = lco[b] + next[b];
      L.leaf_chunk_off = (int64_t*)p.mem.get(sizeof(int64_t) * lco.size());
      if (!L.leaf_chunk_off) return false;
      cudaMemcpy(L.leaf_chunk_off, lco.data(), sizeof(int64_t) * lco.size(),
                 cudaMemcpyHostToDevice);
    }
    counts = next;
    ++level;
    if (all_one) break;
  }
  return true;
}

// Scan shape from the options, else the default: leaf 3 steps per thread
// while the leaf chunks fit one wave of the leaf kernels (256 threads per SM
// at their register use), so that the latency-bound leaf chains are short, 4
// above that (fewer upper items); radix 0: a level with many items is folded
// 4 items per thread (enough threads to fill the GPU, least work), a level
// with few items is scanned in one-warp Kogge-Stone chunks of 32 (shortest
// chain of dependent combines).  An explicit radix folds that many items per
// thread at every level.
void default_shape(const sqsm_ctx* ctx, const int64_t* offsets, int64_t batch, int* L0, int* R) {
  const int64_t steps = offsets[batch] - offsets[0];
  *L0 = ctx->opt.leaf_chunk > 0 ? ctx->opt.leaf_chunk
        : steps <= 3 * int64_t(256) * ctx->sm_count ? 3 : 4;
  *R = ctx->opt.radix <= 1 ? 0 : ctx->opt.radix;
}

Plan* find_plan(sqsm_ctx* ctx, const int64_t* offsets, int64_t batch, int L0, int R) {
  for (auto& p : ctx->plans)
    if (p->B == batch && p->L0 == L0 && p->R == R &&
        std::memcmp(p->offsets.data(), offsets, sizeof(int64_t) * (batch + 1)) == 0)
      return p.get();
  return nullptr;
}

// Free a plan, its workspaces and the graphs that replay its buffers.
void drop_plan(sqsm_ctx* ctx, const Plan* victim) {
  for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
    if (it->first.plan == victim) {
      if (ctx->last_prof == it->second.prof.get()) ctx->last_prof = nullptr;
      cudaGraphExecDestroy(it->second.exec);
      it = ctx->graphs.erase(it);
    } else {
      ++it;
    }
  }
  cudaDeviceSynchronize();
  for (auto it = ctx->plans.begin(); it != ctx->plans.end(); ++it)
    if (it->get() == victim) {
      ctx->plans.erase(it);
      break;
    }
}

Plan* get_plan(sqsm_ctx* ctx, const int64_t* offsets, int64_t batch, int L0, int R) {
  if (Plan* q = find_plan(ctx, offsets, batch, L0, R)) return q;
  auto p = std::make_unique<Plan>();
  p->B = (int)batch;
  p->L0 = L0;
  p->R = R;
  p->offsets.assign(offsets, offsets + batch + 1);
  p->d_offsets = (int64_t*)p->mem.get(sizeof(int64_t) * (batch + 1));
  if (!p->d_offsets) return nullptr;
  cudaMemcpy(p->d_offsets, offsets, sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice);
  std::vector<int64_t> nf(batch), ns(batch);
  for (int64_t b = 0; b < batch; ++b) {
    nf[b] = offsets[b + 1] - offsets[b];
    ns[b] = nf[b] + 1;
  }
  if (!build_levels(*p, nf, p->filt) || !build_levels(*p, ns, p->smth)) return nullptr;
  if (ctx->plans.size() >= 8) drop_plan(ctx, ctx->plans.front().get());
  ctx->plans.push_back(std::move(p));
  return ctx->plans.back().get();
}

Plan* get_plan(sqsm_ctx* ctx, const int64_t* offsets, int64_t batch) {
  int L0, R;
  default_shape(ctx, offsets, batch, &L0, &R);
  return get_plan(ctx, offsets, batch, L0, R);
}

bool alloc_scan(Alloc& mem, const LevelSet& L, ScanBuffers& W, size_t item_bytes,
                size_t carry_bytes) {
  const size_t Lc = L.lv.size();
  W.items.assign(Lc + 1, nullptr);
  W.carry.assign(Lc + 1, nullptr);
  W.flag.assign(Lc + 1, nullptr);
  for (size_t l = 1; l <= Lc; ++l) {
    const int64_t n = L.n_items[l];
    W.items[l] = mem.get(item_bytes * n);
    W.carry[l] = mem.get(carry_bytes * n);
    W.flag[l] = (int*)mem.get(sizeof(int) * n);
    if (!W.items[l] || !W.carry[l] || !W.flag[l]) return false;
    cudaMemset(W.carry[l], 0, carry_bytes * n);
  }
  return true;
}

Workspace* get_ws(Plan* p, int dtype, int nx) {
  auto key = std::make_pair(dtype, nx);
  auto it = p->ws.find(key);
  if (it != p->ws.end()) return it->second.get();
  auto w = std::make_unique<Workspace>();
  const size_t es = dtype == SQSM_F64 ? 8 : 4;
  // carries: the square-root scans' packed records (XRow) and the standard
  // form's vector + full covariance share the buffers
  const size_t frec = frec_size(nx), srec = srec_size(nx),
               crec = std::max(nx + nx * nx, xrow_size(nx));
  if (!alloc_scan(w->mem, p->filt, w->filt, es * frec, es * crec)) return nullptr;
  if (!alloc_scan(w->mem, p->smth, w->smth, es * srec, es * crec)) return nullptr;
  w->partial = (double*)w->mem.get(sizeof(double) * p->filt.lv[0].n_chunks);
  const int64_t rows = p->smth.n_items[0];
  w->mf = w->mem.get(es * nx * rows);
  w->Nf = w->mem.get(es * nx * nx * rows);
  if (!w->partial || !w->mf || !w->Nf) return nullptr;
  Workspace* r = w.get();
  p->ws[key] = std::move(w);
  return r;
}

bool ensure_ipls(Workspace* w, const Plan* p, int dtype, int nx = 5, int ny = 2) {
  if (w->ipls_ready) return true;
  const size_t es = dtype == SQSM_F64 ? 8 : 4;
  const int64_t n = p->filt.n_items[0];
  // the linearised model of every step as packed records
  w->gamma = w->mem.get(es * prec_size(nx, ny) * n);
  const int64_t rows = p->smth.n_items[0];
  w->frows = w->mem.get(es * xrow_size(nx) * rows);
  w->nrows = w->mem.get(es * xrow_size(nx) * rows);
  if (!w->gamma || !w->frows || !w->nrows) return false;
  w->params = w->mem.get(512);
  w->dm0 = w->mem.get(es * nx * p->B);
  w->tol_words = (int*)w->mem.get(4 * sizeof(int));
  w->prevrows = w->mem.get(es * xrow_size(nx) * rows);
  w->partial2 = (double*)w->mem.get(sizeof(double) * p->filt.lv[0].n_chunks);
  if (!w->params || !w->dm0 || !w->tol_words || !w->prevrows || !w->partial2) return false;
  w->ipls_ready = true;
  return true;
}

// The tables of the mean-only refinement passes, made when a context with
// refinement first uses the workspace: the smoother's per-row E_k and, where
// the plan's filter levels take the mean-only form (fmeans_layout), the
// filter's stored combine factors.
bool ensure_refine_tabs(Workspace* w, const Plan* p, int dtype, int nx) {
  const size_t es = dtype == SQSM_F64 ? 8 : 4;
  if (!w->etab) w->etab = w->mem.get(es * ((nx * nx + 3) / 4 * 4) * p->smth.n_items[0]);
  if (!w->etab) return false;
  if (w->ftab) return true;
  const FMeansLayout f = fmeans_layout(p->filt, es, nx);
  if (!f.on) return true;
  w->ftab = w->mem.get(es * f.size);
  return w->ftab != nullptr;
}

bool ensure_adj(Workspace* w, const Plan* p, int dtype) {
  if (w->adj_ready) return true;
  const size_t es = dtype == SQSM_F64 ? 8 : 4;
  const int64_t rows = p->smth.n_items[0], steps = p->filt.n_items[0];
  const int nx = 5, ny = 2, X = nx + nx * nx;
  const int grec = 2 * nx * nx + nx + ny * nx + ny + ny * ny;
  AdjArgs& g = w->adj;
  g.nom_m = w->mem.get(es * nx * rows);
  g.nom_N = w->mem.get(es * nx * nx * rows);
  g.ms2 = w->mem.get(es * nx * rows);
  g.Ns2 = w->mem.get(es * nx * nx * rows);
  g.dir = w->mem.get(es * X * rows);
  g.dfilt = w->mem.get(es * X * rows);
  g.lam_a = w->mem.get(es * X * rows);
  g.lam_b = w->mem.get(es * X * rows);
  g.gbar = w->mem.get(es * grec * steps);
  g.ktab = w->mem.get(es * KfTab<5, 2>::size * steps);
  g.rtab = w->mem.get(es * RtsTab<5>::size * steps);
  g.stab = w->mem.get(es * SlrTab<5, 2>::size * steps);
  // theta partial sums, one triple per block of the SLR VJP kernel
  g.th_partial = (double*)w->mem.get(
      sizeof(double) * 4 * std::max<int64_t>(1, grid_for(p->smth.lv[0].n_chunks * p->L0)));
  g.ll = (double*)w->mem.get(sizeof(double) * p->B);
  g.change_words = w->mem.get(4 * sizeof(unsigned));
  if (!g.change_words) return false;
  if (!g.nom_m || !g.nom_N || !g.ms2 || !g.Ns2 || !g.dir || !g.dfilt || !g.lam_a || !g.lam_b ||
      !g.gbar || !g.ktab || !g.rtab || !g.stab || !g.th_partial || !g.ll)
    return false;
  if (!alloc_scan(w->mem, p->filt, w->adj_scan, es * (2 * nx * nx + 2 * nx), es * X)) return false;
  w->adj_ready = true;
  return true;
}

DevSeqs seqs_of(const Plan* p) {
  DevSeqs s;
  s.B = p->B;
  s.offsets = p->d_offsets;
  s.leaf_chunk_off = p->filt.leaf_chunk_off;
  return s;
}

bool valid_offsets(const int64_t* off, int64_t batch) {
  if (!off || off[0] != 0) return false;
  for (int64_t b = 0; b < batch; ++b)
    if (off[b + 1] <= off[b]) return false;
  return true;
}

// Every non-null pointer is a multiple of `bytes` (the kernels access caller
// arrays element by element, so an element must not straddle its boundary).
bool aligned(size_t bytes, std::initializer_list<const void*> ptrs) {
  for (const void* q : ptrs)
    if (q && reinterpret_cast<uintptr_t>(q) % bytes != 0) return false;
  return true;
}

size_t elem_bytes(int dtype) { return dtype == SQSM_F64 ? 8 : 4; }

// With the prior_covariance option the N0 argument of a call holds prior
// covariances P0: the scans then read the FP64 Cholesky factors that
// enqueue_prior writes into the workspace (returned here; null if that
// buffer cannot be allocated), else the caller's N0 itself.
const void* prior_input(const sqsm_ctx* ctx, Workspace* w, const Plan* p, int dtype, int nx,
                        const void* N0) {
  if (!ctx->opt.prior_covariance) return N0;
  if (!w->n0fac) w->n0fac = w->mem.get(elem_bytes(dtype) * nx * nx * p->B);
  return w->n0fac;
}

void enqueue_prior(const sqsm_ctx* ctx, const Plan* p, const Workspace* w, int dtype, int nx,
                   const void* P0, cudaStream_t s) {
  if (ctx->opt.prior_covariance)
    enqueue_prior_cholesky(dtype == SQSM_F64, p->B, nx, P0, w->n0fac, ctx->d_status, s);
}

}  // namespace

extern "C" {

int sqsm_create(sqsm_ctx** out, int device, const sqsm_options* opt) {
  if (!out) return SQSM_ERR_INVALID_ARG;
  *out = nullptr;
  if (opt && (opt->refine < 0 || opt->refine > 2 || opt->max_group_steps < 0))
    return SQSM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return SQSM_ERR_CUDA;
  auto* ctx = new sqsm_ctx();
  ctx->device = device;
  if (opt) ctx->opt = *opt;
  DeviceGuard g(device);
  if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return SQSM_ERR_CUDA;
  }
  if (cudaMalloc(&ctx->d_group, 8 * sizeof(double)) != cudaSuccess) {
    cudaFree(ctx->d_status);
    delete ctx;
    return SQSM_ERR_CUDA;
  }
  cudaMemset(ctx->d_status, 0, sizeof(int));
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_group);
    delete ctx;
    return SQSM_ERR_CUDA;
  }
  *out = ctx;
  return SQSM_OK;
}

int sqsm_destroy(sqsm_ctx* ctx) {
  if (!ctx) return SQSM_OK;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
    ctx->plans.clear();
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_group);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
  }
  delete ctx;
  return SQSM_OK;
}

const char* sqsm_last_error(const sqsm_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int sqsm_get_status(sqsm_ctx* ctx, int* status) {
  if (!ctx || !status) return SQSM_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_get_status");
  int v = 0;
  e = cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_get_status");
  cudaMemset(ctx->d_status, 0, sizeof(int));
  *status = v;
  return SQSM_OK;
}

int sqsm_supported_shape(int nx, int ny) { return lgssm_shape_supported(nx, ny) ? 1 : 0; }

int sqsm_profile_enable(sqsm_ctx* ctx, int on) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  ctx->prof_on = on != 0;
  return SQSM_OK;
}

int sqsm_profile_read(sqsm_ctx* ctx, int nkinds, double* ms, int* launches, int* nfamilies) {
  if (!ctx || nkinds < 0 || (nkinds > 0 && (!ms || !launches))) return SQSM_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_profile_read");
  for (int k = 0; k < nkinds; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  if (nfamilies) *nfamilies = K_NUM_KINDS;
  if (!ctx->last_prof) return SQSM_OK;
  for (const auto& r : ctx->last_prof->rec) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventElapsedTime");
    if (r.kind < nkinds) {
      ms[r.kind] += t;
      launches[r.kind] += 1;
    }
  }
  return SQSM_OK;
}

const char* sqsm_kernel_name(int k) {
  static const char* names[K_NUM_KINDS] = {
      "ct_params", "broadcast_prior", "ct_slr", "filter_leaf_up", "filter_up", "filter_down",
      "filter_leaf_down", "smoother_leaf_up", "smoother_up", "smoother_down",
      "smoother_leaf_down", "loglik_reduce"};
  return (k >= 0 && k < K_NUM_KINDS) ? names[k] : "";
}

int sqsm_lgssm_smooth(sqsm_ctx* ctx, int dtype, int nx, int ny, int64_t n, const void* F,
                      int64_t sF, const void* c, int64_t sc, const void* SQ, int64_t sSQ,
                      const void* H, int64_t sH, const void* d, int64_t sd, const void* SR,
                      int64_t sSR, const void* m0, const void* N0, const void* y, void* mf,
                      void* Nf, void* ms, void* Ns, double* loglik, void* stream) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  if (dtype != SQSM_F32 && dtype != SQSM_F64)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "dtype must be SQSM_F32 or SQSM_F64");
  if (n < 1) return fail(ctx, SQSM_ERR_INVALID_ARG, "n must be >= 1");
  if (nx < 1 || ny < 1 || nx > 8 || ny > 8)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "nx, ny must be in 1..8");
  if (!lgssm_shape_supported(nx, ny))
    return fail(ctx, SQSM_ERR_UNSUPPORTED, "(nx, ny) pair not compiled in");
  if (!F || !c || !SQ || !H || !d || !SR || !m0 || !N0 || !y || !ms || !Ns)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "null input or smoother output pointer");
  if (sF < 0 || sc < 0 || sSQ < 0 || sH < 0 || sd < 0 || sSR < 0)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "negative stride");
  if (!aligned(elem_bytes(dtype), {F, c, SQ, H, d, SR, m0, N0, y, mf, Nf, ms, Ns}) ||
      !aligned(8, {loglik}))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "pointer not a multiple of its element size");
  DeviceGuard g(ctx->device);
  const int64_t offsets[2] = {0, n};
  Plan* p = get_plan(ctx, offsets, 1);
  if (!p) return fail(ctx, SQSM_ERR_NO_MEMORY, "plan allocation failed");
  Workspace* w = get_ws(p, dtype, nx);
  if (!w) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace allocation failed");
  const void* n0 = prior_input(ctx, w, p, dtype, nx, N0);
  if (!n0) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace allocation failed");
  Prof* prof = nullptr;
  if (ctx->prof_on) {
    ctx->call_prof.clear();
    prof = &ctx->call_prof;
    ctx->last_prof = prof;
  }
  LgssmArgs a{nx, ny, F, c, SQ, H, d, SR, sF, sc, sSQ, sH, sd, sSR, m0, n0, y,
              mf ? mf : w->mf, Nf ? Nf : w->Nf, ms, Ns, prof};
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();
  enqueue_prior(ctx, p, w, dtype, nx, N0, s);
  const DevSeqs sq = seqs_of(p);
  int rc = dtype == SQSM_F32
               ? lgssm_enqueue_f32(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial,
                                   ctx->d_status, s)
               : lgssm_enqueue_f64(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial,
                                   ctx->d_status, s);
  if (rc) return fail(ctx, rc, "(nx, ny) pair not compiled in");
  if (loglik) enqueue_loglik_reduce(sq, w->partial, loglik, ctx->d_status, s, prof);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_lgssm_smooth launch");
  return SQSM_OK;
}

namespace {

// theta into IplsArgs::theta[4]: the CT model with one noise level per
// sensor passes log sigma of the second sensor as its fourth entry; with one
// noise level for both sensors (and for the other models) entry 3 repeats
// entry 0.
void copy_theta(double* dst, const sqsm_model* model, const double* theta) {
  for (int i = 0; i < 3; ++i) dst[i] = theta[i];
  dst[3] = model->kind == SQSM_MODEL_CT_BEARINGS_R ? theta[3] : theta[0];
}

// Arguments of one IPLS enqueue on plan p's workspace w.
IplsArgs make_ipls_args(const Plan* p, const Workspace* w, const sqsm_model* model,
                        const double* theta, int lin, int M, const void* y, const void* m0,
                        const void* N0, const void* init_ms, const void* init_Ns, void* ms,
                        void* Ns, double* loglik) {
  IplsArgs a{};
  a.linearization = lin;
  a.leaf = p->L0;
  a.M = M;
  copy_theta(a.theta, model, theta);
  a.dt = model->dt;
  for (int i = 0; i < 4; ++i) a.sensors[i] = model->sensors[i];
  a.y = y; a.m0 = m0; a.N0 = N0; a.init_ms = init_ms; a.init_Ns = init_Ns;
  a.ms = ms; a.Ns = Ns; a.loglik = loglik;
  a.mf = w->mf; a.Nf = w->Nf;
  a.F = w->gamma;   // PRec records; c, SQ, H, d, SR unused
  a.frows = w->frows;
  a.nrows = w->nrows;
  a.params = w->params;
  a.dm0 = w->dm0;
  a.prevrows = w->prevrows;
  a.partial2 = w->partial2;
  a.etab = w->etab;
  a.ftab = w->ftab;
  return a;
}

IplsArgs ctx_ipls_args(const sqsm_ctx* ctx, const Plan* p, const Workspace* w,
                        const sqsm_model* model, const double* theta, int lin, int M,
                        const void* y, const void* m0, const void* N0, const void* init_ms,
                        const void* init_Ns, void* ms, void* Ns, double* loglik) {
  IplsArgs a = make_ipls_args(p, w, model, theta, lin, M, y, m0, N0, init_ms, init_Ns, ms, Ns,
                              loglik);
  a.centered = ctx->opt.absolute ? 0 : 1;
  a.refine = ctx->opt.refine;
  a.textbook = ctx->opt.textbook_slr ? 1 : 0;
  return a;
}

void enqueue_ipls(sqsm_ctx* ctx, int dtype, const Plan* p, const Workspace* w, const IplsArgs& a,
                  cudaStream_t st) {
  const DevSeqs sq = seqs_of(p);
  if (dtype == SQSM_F32)
    ipls_enqueue_f32(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, st);
  else
    ipls_enqueue_f64(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, st);
}

// The population model's params kernel and M-iteration enqueue.
void pop_params(int dtype, const IplsArgs& a, cudaStream_t s) {
  if (dtype == SQSM_F32) pop_params_f32(a, s); else pop_params_f64(a, s);
}

void pop_phase(int dtype, sqsm_ctx* ctx, const Plan* p, const Workspace* w, const IplsArgs& a,
               cudaStream_t st, int phase, unsigned* dmax) {
  const DevSeqs sq = seqs_of(p);
  if (dtype == SQSM_F32)
    pop_phase_f32(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, st, phase,
                  dmax);
  else
    pop_phase_f64(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, st, phase,
                  dmax);
}

void enqueue_pop(sqsm_ctx* ctx, int dtype, const Plan* p, const Workspace* w, const IplsArgs& a,
                 cudaStream_t st) {
  pop_phase(dtype, ctx, p, w, a, st, IPLS_PRE, nullptr);
  for (int it = 0; it < a.M; ++it) pop_phase(dtype, ctx, p, w, a, st, IPLS_ITER, nullptr);
  pop_phase(dtype, ctx, p, w, a, st, IPLS_POST, nullptr);
}

bool known_model(const sqsm_model* model) {
  return model && (model->kind == SQSM_MODEL_CT_BEARINGS || model->kind == SQSM_MODEL_POPULATION ||
                   model->kind == SQSM_MODEL_CT_BEARINGS_R);
}

bool is_ct(const sqsm_model* model) {
  return model->kind == SQSM_MODEL_CT_BEARINGS || model->kind == SQSM_MODEL_CT_BEARINGS_R;
}

// Number of theta entries the caller passes (and of gradient entries).
int n_theta(const sqsm_model* model) { return model->kind == SQSM_MODEL_CT_BEARINGS_R ? 4 : 3; }

bool theta_finite(const sqsm_model* model, const double* theta) {
  for (int i = 0; i < n_theta(model); ++i)
    if (!std::isfinite(theta[i])) return false;
  return true;
}

int floor_log2(int64_t v) {
  int l = 0;
  while (v > 1) {
    v >>= 1;
    ++l;
  }
  return l;
}

TuneKey tune_key(int dtype, int lin, int64_t batch, const int64_t* offsets) {
  int64_t longest = 0;
  for (int64_t b = 0; b < batch; ++b) longest = std::max(longest, offsets[b + 1] - offsets[b]);
  return TuneKey{dtype, lin, batch, floor_log2(offsets[batch] - offsets[0]), floor_log2(longest)};
}

// Candidate scan shapes (leaf_chunk, radix) the autotuner measures.
constexpr int kTuneShapes[][2] = {{2, 0}, {3, 0}, {4, 0}, {6, 0}, {8, 0}, {4, 4}};

// Scan shape of an IPLS call: the options' or the default, or with
// autotune the fastest candidate for the workload shape, measured once per
// context (one IPLS iteration per candidate on the call's inputs, best of two
// after a warm-up run) and stored.  Plans made only for the measurement are
// freed as soon as a faster candidate is found.
int choose_ipls_shape(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                      int lin, int64_t batch, const int64_t* offsets, const void* y,
                      const void* m0, const void* N0, const void* init_ms, const void* init_Ns,
                      void* ms, void* Ns, cudaStream_t s, int* L0, int* R) {
  default_shape(ctx, offsets, batch, L0, R);
  if (!ctx->opt.autotune || ctx->opt.leaf_chunk > 0 || ctx->opt.radix > 0) return SQSM_OK;
  const TuneKey key = tune_key(dtype, lin, batch, offsets);
  auto found = ctx->tuned.find(key);
  if (found != ctx->tuned.end()) {
    *L0 = found->second.first;
    *R = found->second.second;
    return SQSM_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(ctx, SQSM_ERR_CUDA, "autotune: cudaEventCreate failed");
  }
  float best = INFINITY;
  int bl = *L0, br = *R;
  bool best_made = false;   // the best plan was made only for the measurement
  int rc = SQSM_OK;
  for (const auto& c : kTuneShapes) {
    const bool existed = find_plan(ctx, offsets, batch, c[0], c[1]) != nullptr;
    Plan* p = get_plan(ctx, offsets, batch, c[0], c[1]);
    if (!p) continue;
    Workspace* w = get_ws(p, dtype, 5);
    const void* n0 = w && ensure_ipls(w, p, dtype) &&
                             (ctx->opt.refine == 0 || ensure_refine_tabs(w, p, dtype, 5))
                         ? prior_input(ctx, w, p, dtype, 5, N0)
                         : nullptr;
    if (!n0) {
      if (!existed) drop_plan(ctx, p);
      continue;
    }
    const IplsArgs a = ctx_ipls_args(ctx, p, w, model, theta, lin, 1, y, m0, n0, init_ms, init_Ns,
                                      ms, Ns, nullptr);
    enqueue_prior(ctx, p, w, dtype, 5, N0, s);
    if (dtype == SQSM_F32) ipls_params_f32(a, s); else ipls_params_f64(a, s);
    float t = INFINITY;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      enqueue_ipls(ctx, dtype, p, w, a, s);
      cudaEventRecord(e1, s);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = cuda_fail(ctx, e, "autotune");
        break;
      }
      float ms_ = 0.f;
      cudaEventElapsedTime(&ms_, e0, e1);
      if (rep > 0) t = std::min(t, ms_);
    }
    if (rc != SQSM_OK) break;
    if (t < best) {
      if (best_made) drop_plan(ctx, find_plan(ctx, offsets, batch, bl, br));
      best = t;
      bl = c[0];
      br = c[1];
      best_made = !existed;
    } else if (!existed) {
      drop_plan(ctx, p);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SQSM_OK) return rc;
  ctx->tuned[key] = {bl, br};
  *L0 = bl;
  *R = br;
  return SQSM_OK;
}

}  // namespace

extern "C" int sqsm_scan_shape(sqsm_ctx* ctx, int dtype, int linearization, int64_t batch,
                               const int64_t* offsets, int* leaf_chunk, int* radix) {
  if (!ctx || !leaf_chunk || !radix) return SQSM_ERR_INVALID_ARG;
  if (batch < 1 || batch > (1 << 30) || !valid_offsets(offsets, batch))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "offsets must start at 0 and increase strictly");
  default_shape(ctx, offsets, batch, leaf_chunk, radix);
  if (ctx->opt.autotune && ctx->opt.leaf_chunk <= 0 && ctx->opt.radix <= 0) {
    auto it = ctx->tuned.find(tune_key(dtype, linearization, batch, offsets));
    if (it != ctx->tuned.end()) {
      *leaf_chunk = it->second.first;
      *radix = it->second.second;
    }
  }
  return SQSM_OK;
}

int sqsm_ipls_smooth(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                     int linearization, int M, int64_t batch, const int64_t* offsets,
                     const void* y, const void* m0, const void* N0, const void* init_ms,
                     const void* init_Ns, void* ms, void* Ns, double* loglik, void* stream) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  if (dtype != SQSM_F32 && dtype != SQSM_F64)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "dtype must be SQSM_F32 or SQSM_F64");
  if (!known_model(model)) return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown model kind");
  const bool pop = model->kind == SQSM_MODEL_POPULATION;
  if (!pop && !(model->dt > 0)) return fail(ctx, SQSM_ERR_INVALID_ARG, "model dt must be > 0");
  if (pop && linearization != SQSM_CUBATURE && linearization != SQSM_EXTENDED)
    return fail(ctx, SQSM_ERR_UNSUPPORTED, "the population model takes cubature or extended SLR");
  if (!theta) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta is null");
  if (linearization < SQSM_CUBATURE || linearization > SQSM_GAUSS_HERMITE)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown linearization");
  if (M < 1) return fail(ctx, SQSM_ERR_INVALID_ARG, "M must be >= 1");
  if (batch < 1 || batch > (1 << 30)) return fail(ctx, SQSM_ERR_INVALID_ARG, "bad batch");
  if (!valid_offsets(offsets, batch))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "offsets must start at 0 and increase strictly");
  if (!y || !m0 || !N0 || !ms || !Ns)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "null input or output pointer");
  if ((init_ms == nullptr) != (init_Ns == nullptr))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "init_ms and init_Ns must both be set or both NULL");
  if (!theta_finite(model, theta)) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta not finite");
  if (!aligned(elem_bytes(dtype), {y, m0, N0, init_ms, init_Ns, ms, Ns}) || !aligned(8, {loglik}))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "pointer not a multiple of its element size");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();
  int L0 = 0, R = 0;
  if (pop) {
    default_shape(ctx, offsets, batch, &L0, &R);
  } else {
    const int trc = choose_ipls_shape(ctx, dtype, model, theta, linearization, batch, offsets, y,
                                      m0, N0, init_ms, init_Ns, ms, Ns, s, &L0, &R);
    if (trc != SQSM_OK) return trc;
  }
  Plan* p = get_plan(ctx, offsets, batch, L0, R);
  if (!p) return fail(ctx, SQSM_ERR_NO_MEMORY, "plan allocation failed");
  const int nx = pop ? 1 : 5, ny = pop ? 1 : 2;
  Workspace* w = get_ws(p, dtype, nx);
  if (!w || !ensure_ipls(w, p, dtype, nx, ny) ||
      (ctx->opt.refine > 0 && !ensure_refine_tabs(w, p, dtype, nx)))
    return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  const void* n0 = prior_input(ctx, w, p, dtype, nx, N0);
  if (!n0) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  IplsArgs a = ctx_ipls_args(ctx, p, w, model, theta, linearization, M, y, m0, n0, init_ms, init_Ns,
                              ms, Ns, loglik);
  // theta -> model constants, outside any graph so that theta is not baked in
  if (pop) pop_params(dtype, a, s);
  else if (dtype == SQSM_F32) ipls_params_f32(a, s);
  else ipls_params_f64(a, s);
  auto enqueue = [&](cudaStream_t st) {
    enqueue_prior(ctx, p, w, dtype, nx, N0, st);
    if (pop) enqueue_pop(ctx, dtype, p, w, a, st);
    else enqueue_ipls(ctx, dtype, p, w, a, st);
  };
  if (!ctx->opt.use_graph) {
    if (ctx->prof_on) {
      ctx->call_prof.clear();
      a.prof = &ctx->call_prof;
      ctx->last_prof = a.prof;
    }
    enqueue(s);
  } else {
    GraphKey key{p, dtype, linearization, M, ctx->prof_on ? 1 : 0, 0, y, m0, N0, init_ms, init_Ns,
                 ms, Ns, loglik};
    key.kind = model->kind;
    key.prior_cov = ctx->opt.prior_covariance;
    auto it = ctx->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != ctx->graphs.end()) {
      exec = it->second.exec;
      if (ctx->prof_on) ctx->last_prof = it->second.prof.get();
    } else {
      std::unique_ptr<Prof> gprof;
      if (ctx->prof_on) {
        gprof = std::make_unique<Prof>();
        a.prof = gprof.get();
      }
      // Recording executes nothing, so it happens on the context's own
      // stream (the legacy default stream cannot be captured); the graph is
      // then launched on the caller's stream.
      cudaGraph_t graph = nullptr;
      cudaStream_t cs = ctx->capture_stream;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
      enqueue(cs);
      e = cudaStreamEndCapture(cs, &graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
      if (ctx->graphs.size() >= 16) {
        if (ctx->last_prof == ctx->graphs.begin()->second.prof.get()) ctx->last_prof = nullptr;
        cudaGraphExecDestroy(ctx->graphs.begin()->second.exec);
        ctx->graphs.erase(ctx->graphs.begin());
      }
      GraphEntry& ge = ctx->graphs[key];
      ge.exec = exec;
      ge.prof = std::move(gprof);
      if (ctx->prof_on) ctx->last_prof = ge.prof.get();
    }
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ipls_smooth launch");
  return SQSM_OK;
}

int sqsm_ipls_smooth_tol(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                         int linearization, int max_iters, double tol, int64_t batch,
                         const int64_t* offsets, const void* y, const void* m0, const void* N0,
                         const void* init_ms, const void* init_Ns, void* ms, void* Ns,
                         double* loglik, int* iters_done, void* stream) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  if (dtype != SQSM_F32 && dtype != SQSM_F64)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "dtype must be SQSM_F32 or SQSM_F64");
  if (!known_model(model)) return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown model kind");
  const bool pop = model->kind == SQSM_MODEL_POPULATION;
  if (!pop && !(model->dt > 0)) return fail(ctx, SQSM_ERR_INVALID_ARG, "model dt must be > 0");
  if (pop && linearization != SQSM_CUBATURE && linearization != SQSM_EXTENDED)
    return fail(ctx, SQSM_ERR_UNSUPPORTED, "the population model takes cubature or extended SLR");
  if (!theta) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta is null");
  if (linearization < SQSM_CUBATURE || linearization > SQSM_GAUSS_HERMITE)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown linearization");
  if (max_iters < 1) return fail(ctx, SQSM_ERR_INVALID_ARG, "max_iters must be >= 1");
  if (!(tol >= 0.0) || !std::isfinite(tol))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (batch < 1 || batch > (1 << 30)) return fail(ctx, SQSM_ERR_INVALID_ARG, "bad batch");
  if (!valid_offsets(offsets, batch))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "offsets must start at 0 and increase strictly");
  if (!y || !m0 || !N0 || !ms || !Ns || !iters_done)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "null input or output pointer");
  if ((init_ms == nullptr) != (init_Ns == nullptr))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "init_ms and init_Ns must both be set or both NULL");
  if (!theta_finite(model, theta)) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta not finite");
  if (!aligned(elem_bytes(dtype), {y, m0, N0, init_ms, init_Ns, ms, Ns}) ||
      !aligned(8, {loglik}) || !aligned(4, {iters_done}))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "pointer not a multiple of its element size");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();
  int L0 = 0, R = 0;
  if (pop) {
    default_shape(ctx, offsets, batch, &L0, &R);
  } else {
    const int trc = choose_ipls_shape(ctx, dtype, model, theta, linearization, batch, offsets, y,
                                      m0, N0, init_ms, init_Ns, ms, Ns, s, &L0, &R);
    if (trc != SQSM_OK) return trc;
  }
  Plan* p = get_plan(ctx, offsets, batch, L0, R);
  if (!p) return fail(ctx, SQSM_ERR_NO_MEMORY, "plan allocation failed");
  const int nx = pop ? 1 : 5, ny = pop ? 1 : 2;
  Workspace* w = get_ws(p, dtype, nx);
  if (!w || !ensure_ipls(w, p, dtype, nx, ny) ||
      (ctx->opt.refine > 0 && !ensure_refine_tabs(w, p, dtype, nx)))
    return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  const void* n0 = prior_input(ctx, w, p, dtype, nx, N0);
  if (!n0) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  const IplsArgs a = ctx_ipls_args(ctx, p, w, model, theta, linearization, max_iters, y, m0, n0,
                                    init_ms, init_Ns, ms, Ns, loglik);
  int* iters = w->tol_words;
  int* go = w->tol_words + 1;
  unsigned* dmax = (unsigned*)(w->tol_words + 2);
  const DevSeqs sq = seqs_of(p);
  auto phase = [&](int ph, cudaStream_t st) {
    if (pop)
      pop_phase(dtype, ctx, p, w, a, st, ph, ph == IPLS_ITER ? dmax : nullptr);
    else if (dtype == SQSM_F32)
      ipls_phase_f32(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, st, ph,
                     ph == IPLS_ITER ? dmax : nullptr);
    else
      ipls_phase_f64(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, st, ph,
                     ph == IPLS_ITER ? dmax : nullptr);
  };
  if (pop) pop_params(dtype, a, s);
  else if (dtype == SQSM_F32) ipls_params_f32(a, s);
  else ipls_params_f64(a, s);
  if (!ctx->opt.use_graph) {
    // host-driven loop: one device-to-host read of the continue flag per iteration
    enqueue_prior(ctx, p, w, dtype, nx, N0, s);
    phase(IPLS_PRE, s);
    cudaMemsetAsync(w->tol_words, 0, 4 * sizeof(int), s);
    for (int it = 0; it < max_iters; ++it) {
      phase(IPLS_ITER, s);
      enqueue_tol_check(dmax, iters, max_iters, (float)tol, 0, 0, go, s);
      int more = 0;
      cudaMemcpyAsync(&more, go, sizeof(int), cudaMemcpyDeviceToHost, s);
      const cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ipls_smooth_tol");
      if (!more) break;
    }
    phase(IPLS_POST, s);
    cudaMemcpyAsync(iters_done, iters, sizeof(int), cudaMemcpyDeviceToDevice, s);
  } else {
    // one graph: the initial trajectory, a conditional WHILE node whose body is
    // one iteration followed by the check that sets the loop's condition, then
    // the result and the log-likelihood
    GraphKey key{p, dtype, linearization, max_iters, 0, 0, y, m0, N0, init_ms, init_Ns,
                 ms, Ns, loglik};
    key.tol = tol;
    key.iters = iters_done;
    key.kind = model->kind;
    key.prior_cov = ctx->opt.prior_covariance;
    auto it = ctx->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != ctx->graphs.end()) {
      exec = it->second.exec;
    } else {
      cudaStream_t cs = ctx->capture_stream;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
      enqueue_prior(ctx, p, w, dtype, nx, N0, cs);
      phase(IPLS_PRE, cs);
      cudaMemsetAsync(w->tol_words, 0, 4 * sizeof(int), cs);
      cudaStreamCaptureStatus cst;
      cudaGraph_t graph = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
      cudaGraphConditionalHandle handle = 0;
      if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode = nullptr;
      if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp);
      if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1,
                                                cudaStreamSetCaptureDependencies);
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(ctx->body_stream, cp.conditional.phGraph_out[0], nullptr,
                                          nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaGraph_t dead = nullptr;
        cudaStreamEndCapture(cs, &dead);
        if (dead) cudaGraphDestroy(dead);
        return cuda_fail(ctx, e, "conditional graph node");
      }
      phase(IPLS_ITER, ctx->body_stream);
      enqueue_tol_check(dmax, iters, max_iters, (float)tol, handle, 1, nullptr, ctx->body_stream);
      cudaGraph_t body = nullptr;
      e = cudaStreamEndCapture(ctx->body_stream, &body);
      if (e != cudaSuccess) {
        cudaGraph_t dead = nullptr;
        cudaStreamEndCapture(cs, &dead);
        if (dead) cudaGraphDestroy(dead);
        return cuda_fail(ctx, e, "conditional body capture");
      }
      phase(IPLS_POST, cs);
      cudaMemcpyAsync(iters_done, iters, sizeof(int), cudaMemcpyDeviceToDevice, cs);
      e = cudaStreamEndCapture(cs, &graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
      if (ctx->graphs.size() >= 16) {
        if (ctx->last_prof == ctx->graphs.begin()->second.prof.get()) ctx->last_prof = nullptr;
        cudaGraphExecDestroy(ctx->graphs.begin()->second.exec);
        ctx->graphs.erase(ctx->graphs.begin());
      }
      ctx->graphs[key].exec = exec;
    }
    const cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ipls_smooth_tol launch");
  return SQSM_OK;
}

int sqsm_ipls_smooth_std(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                         int linearization, int M, int64_t batch, const int64_t* offsets,
                         const void* y, const void* m0, const void* P0, void* ms, void* Ps,
                         double* loglik, void* stream) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  if (dtype != SQSM_F32 && dtype != SQSM_F64)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "dtype must be SQSM_F32 or SQSM_F64");
  if (!known_model(model)) return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown model kind");
  if (!is_ct(model))
    return fail(ctx, SQSM_ERR_UNSUPPORTED, "implemented for the CT bearings model");
  if (!(model->dt > 0)) return fail(ctx, SQSM_ERR_INVALID_ARG, "model dt must be > 0");
  if (!theta) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta is null");
  if (linearization != SQSM_CUBATURE && linearization != SQSM_EXTENDED)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown linearization");
  if (M < 1) return fail(ctx, SQSM_ERR_INVALID_ARG, "M must be >= 1");
  if (batch < 1 || batch > (1 << 30)) return fail(ctx, SQSM_ERR_INVALID_ARG, "bad batch");
  if (!valid_offsets(offsets, batch))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "offsets must start at 0 and increase strictly");
  if (!y || !m0 || !P0 || !ms || !Ps)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "null input or output pointer");
  if (!theta_finite(model, theta)) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta not finite");
  if (!aligned(elem_bytes(dtype), {y, m0, P0, ms, Ps}) || !aligned(8, {loglik}))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "pointer not a multiple of its element size");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();
  int L0 = 0, R = 0;
  default_shape(ctx, offsets, batch, &L0, &R);
  Plan* p = get_plan(ctx, offsets, batch, L0, 4);   // fold-only levels
  if (!p) return fail(ctx, SQSM_ERR_NO_MEMORY, "plan allocation failed");
  Workspace* w = get_ws(p, dtype, 5);
  if (!w || !ensure_ipls(w, p, dtype)) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  // a.N0 carries the prior covariances, a.Ns the covariance output
  const IplsArgs a = ctx_ipls_args(ctx, p, w, model, theta, linearization, M, y, m0, P0, nullptr,
                                    nullptr, ms, Ps, loglik);
  const DevSeqs sq = seqs_of(p);
  if (dtype == SQSM_F32) {
    ipls_params_f32(a, s);
    std_ipls_enqueue_f32(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, s);
  } else {
    ipls_params_f64(a, s);
    std_ipls_enqueue_f64(a, p->filt, w->filt, p->smth, w->smth, sq, w->partial, ctx->d_status, s);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ipls_smooth_std launch");
  return SQSM_OK;
}

// One NLL + gradient evaluation of a batch whose arguments were checked.
static int nll_grad_run(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                        int linearization, int M, int adj_iters, double tol, int64_t batch,
                        const int64_t* offsets, const void* y, const void* m0, const void* N0,
                        const void* init_ms, const void* init_Ns, void* ms, void* Ns,
                        double* nll, double* grad, double* adj_change, double* ipls_change,
                        cudaStream_t s, bool use_graph) {
  cudaGetLastError();
  int L0 = 0, R = 0;
  const int trc = choose_ipls_shape(ctx, dtype, model, theta, linearization, batch, offsets, y,
                                    m0, N0, init_ms, init_Ns, ms, Ns, s, &L0, &R);
  if (trc != SQSM_OK) return trc;
  Plan* p = get_plan(ctx, offsets, batch, L0, R);
  if (!p) return fail(ctx, SQSM_ERR_NO_MEMORY, "plan allocation failed");
  Workspace* w = get_ws(p, dtype, 5);
  if (!w || !ensure_ipls(w, p, dtype) || !ensure_adj(w, p, dtype) ||
      (ctx->opt.refine > 0 && !ensure_refine_tabs(w, p, dtype, 5)))
    return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  const void* n0 = prior_input(ctx, w, p, dtype, 5, N0);
  if (!n0) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  IplsArgs a = ctx_ipls_args(ctx, p, w, model, theta, linearization, M, y, m0, n0, init_ms, init_Ns,
                              ms, Ns, nullptr);
  AdjArgs adj = w->adj;
  adj.iters = adj_iters;
  adj.n_theta = n_theta(model);
  adj.nll = nll;
  adj.grad = grad;
  adj.change = adj_change;
  adj.ichange = ipls_change;
  adj.tol = tol;
  const DevSeqs sq = seqs_of(p);
  if (dtype == SQSM_F32) ipls_params_f32(a, s); else ipls_params_f64(a, s);
  auto enqueue = [&](cudaStream_t st) {
    enqueue_prior(ctx, p, w, dtype, 5, N0, st);
    if (dtype == SQSM_F32)
      adj_enqueue_f32(a, adj, p->filt, w->filt, p->smth, w->smth, w->adj_scan, sq, w->partial,
                      ctx->d_status, st);
    else
      adj_enqueue_f64(a, adj, p->filt, w->filt, p->smth, w->smth, w->adj_scan, sq, w->partial,
                      ctx->d_status, st);
  };
  if (!use_graph) {
    enqueue(s);
  } else {
    GraphKey key{p, dtype, linearization, M, 0, adj_iters + 1, y, m0, N0, init_ms, init_Ns,
                 ms, Ns, nll};
    key.kind = model->kind;
    key.grad = grad;          // every pointer the captured kernels write is
    key.change = adj_change;  // part of the key, and the tolerance the
    key.ichange = ipls_change;   // check kernel is given
    key.tol = tol;
    key.prior_cov = ctx->opt.prior_covariance;
    auto it = ctx->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != ctx->graphs.end()) {
      exec = it->second.exec;
    } else {
      cudaGraph_t graph = nullptr;
      cudaStream_t cs = ctx->capture_stream;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
      enqueue(cs);
      e = cudaStreamEndCapture(cs, &graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
      if (ctx->graphs.size() >= 16) {
        if (ctx->last_prof == ctx->graphs.begin()->second.prof.get()) ctx->last_prof = nullptr;
        cudaGraphExecDestroy(ctx->graphs.begin()->second.exec);
        ctx->graphs.erase(ctx->graphs.begin());
      }
      ctx->graphs[key].exec = exec;
    }
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ipls_nll_grad launch");
  return SQSM_OK;
}

int sqsm_ipls_nll_grad(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                       int linearization, int M, int adj_iters, double tol, int64_t batch,
                       const int64_t* offsets, const void* y, const void* m0, const void* N0,
                       const void* init_ms, const void* init_Ns, void* ms, void* Ns,
                       double* nll, double* grad, double* adj_change, double* ipls_change,
                       void* stream) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  if (dtype != SQSM_F32 && dtype != SQSM_F64)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "dtype must be SQSM_F32 or SQSM_F64");
  if (!known_model(model)) return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown model kind");
  if (!is_ct(model))
    return fail(ctx, SQSM_ERR_UNSUPPORTED, "implemented for the CT bearings model");
  if (!(model->dt > 0)) return fail(ctx, SQSM_ERR_INVALID_ARG, "model dt must be > 0");
  if (!theta) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta is null");
  if (linearization < SQSM_CUBATURE || linearization > SQSM_GAUSS_HERMITE)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown linearization");
  if (M < 0 || adj_iters < 0) return fail(ctx, SQSM_ERR_INVALID_ARG, "M, adj_iters must be >= 0");
  if (std::isnan(tol)) return fail(ctx, SQSM_ERR_INVALID_ARG, "tol is NaN");
  if (M == 0 && (!init_ms || !init_Ns))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "M = 0 needs an initial trajectory");
  if (batch < 1 || batch > (1 << 30)) return fail(ctx, SQSM_ERR_INVALID_ARG, "bad batch");
  if (!valid_offsets(offsets, batch))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "offsets must start at 0 and increase strictly");
  if (!y || !m0 || !N0 || !ms || !Ns || !nll || !grad)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "null input or output pointer");
  if ((init_ms == nullptr) != (init_Ns == nullptr))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "init_ms and init_Ns must both be set or both NULL");
  if (!theta_finite(model, theta)) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta not finite");
  if (!aligned(elem_bytes(dtype), {y, m0, N0, init_ms, init_Ns, ms, Ns}) ||
      !aligned(8, {nll, grad, adj_change, ipls_change}))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "pointer not a multiple of its element size");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t cap = ctx->opt.max_group_steps;
  if (cap <= 0 || offsets[batch] <= cap)
    return nll_grad_run(ctx, dtype, model, theta, linearization, M, adj_iters, tol, batch, offsets,
                        y, m0, N0, init_ms, init_Ns, ms, Ns, nll, grad, adj_change, ipls_change,
                        s, ctx->opt.use_graph != 0);
  for (int64_t b = 0; b < batch; ++b)
    if (offsets[b + 1] - offsets[b] > cap)
      return fail(ctx, SQSM_ERR_TOO_LARGE, "a sequence is longer than max_group_steps");
  // groups of consecutive sequences with at most cap steps each, evaluated
  // one after another; each group's plan and workspace are freed before the
  // next group's are made
  const size_t es = elem_bytes(dtype);
  constexpr int nx = 5, ny = 2;
  auto at = [es](const void* p, int64_t elems) -> void* {
    return p ? (void*)((const char*)p + elems * (int64_t)es) : nullptr;
  };
  std::vector<int64_t> sub;
  for (int64_t g0 = 0; g0 < batch;) {
    int64_t g1 = g0 + 1;
    while (g1 < batch && offsets[g1 + 1] - offsets[g0] <= cap) ++g1;
    sub.assign(offsets + g0, offsets + g1 + 1);
    for (auto& v : sub) v -= offsets[g0];
    const int64_t row0 = offsets[g0] + g0;   // the group's first state row
    std::vector<const Plan*> before;
    for (auto& q : ctx->plans) before.push_back(q.get());
    const int rc = nll_grad_run(
        ctx, dtype, model, theta, linearization, M, adj_iters, tol, g1 - g0, sub.data(),
        at(y, offsets[g0] * ny), at(m0, g0 * nx), at(N0, g0 * nx * nx), at(init_ms, row0 * nx),
        at(init_Ns, row0 * nx * nx), at(ms, row0 * nx), at(Ns, row0 * nx * nx), ctx->d_group,
        ctx->d_group + 1, ctx->d_group + 5, ctx->d_group + 6, s, false);
    if (rc != SQSM_OK) return rc;
    enqueue_nll_grad_group_add(g0 == 0 ? 1 : 0, n_theta(model), ctx->d_group, nll, grad,
                               adj_change, ipls_change, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ipls_nll_grad group");
    for (size_t k = ctx->plans.size(); k-- > 0;) {
      const Plan* q = ctx->plans[k].get();
      if (std::find(before.begin(), before.end(), q) == before.end()) drop_plan(ctx, q);
    }
    g0 = g1;
  }
  return SQSM_OK;
}

int sqsm_ct_linearize(sqsm_ctx* ctx, int dtype, const sqsm_model* model, const double* theta,
                      int linearization, int64_t batch, const int64_t* offsets, const void* y,
                      const void* ms, const void* Ns, void* F, void* c, void* SQ, void* H,
                      void* d, void* SR, void* stream) {
  if (!ctx) return SQSM_ERR_INVALID_ARG;
  if (dtype != SQSM_F32 && dtype != SQSM_F64)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "dtype must be SQSM_F32 or SQSM_F64");
  if (!known_model(model)) return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown model kind");
  if (!is_ct(model))
    return fail(ctx, SQSM_ERR_UNSUPPORTED, "implemented for the CT bearings model");
  if (!(model->dt > 0)) return fail(ctx, SQSM_ERR_INVALID_ARG, "model dt must be > 0");
  if (!theta) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta is null");
  if (linearization < SQSM_CUBATURE || linearization > SQSM_GAUSS_HERMITE)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "unknown linearization");
  if (batch < 1 || batch > (1 << 30)) return fail(ctx, SQSM_ERR_INVALID_ARG, "bad batch");
  if (!valid_offsets(offsets, batch))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "offsets must start at 0 and increase strictly");
  if (!y || !ms || !Ns || !F || !c || !SQ || !H || !d || !SR)
    return fail(ctx, SQSM_ERR_INVALID_ARG, "null pointer");
  if (!theta_finite(model, theta)) return fail(ctx, SQSM_ERR_INVALID_ARG, "theta not finite");
  if (!aligned(elem_bytes(dtype), {y, ms, Ns, F, c, SQ, H, d, SR}))
    return fail(ctx, SQSM_ERR_INVALID_ARG, "pointer not a multiple of its element size");
  DeviceGuard g(ctx->device);
  Plan* p = get_plan(ctx, offsets, batch);
  if (!p) return fail(ctx, SQSM_ERR_NO_MEMORY, "plan allocation failed");
  Workspace* w = get_ws(p, dtype, 5);
  if (!w || !ensure_ipls(w, p, dtype)) return fail(ctx, SQSM_ERR_NO_MEMORY, "workspace");
  IplsArgs a{};
  a.linearization = linearization;
  a.leaf = p->L0;
  copy_theta(a.theta, model, theta);
  a.dt = model->dt;
  for (int i = 0; i < 4; ++i) a.sensors[i] = model->sensors[i];
  a.y = y;
  a.ms = const_cast<void*>(ms);
  a.Ns = const_cast<void*>(Ns);
  a.F = F; a.c = c; a.SQ = SQ; a.H = H; a.d = d; a.SR = SR;
  a.params = w->params;
  cudaStream_t s = (cudaStream_t)stream;
  cudaGetLastError();
  const DevSeqs sq = seqs_of(p);
  if (dtype == SQSM_F32) {
    ipls_params_f32(a, s);
    ct_linearize_f32(a, p->filt, sq, s);
  } else {
    ipls_params_f64(a, s);
    ct_linearize_f64(a, p->filt, sq, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sqsm_ct_linearize launch");
  return SQSM_OK;
}

}  // extern "C"

namespace sqsm {
bool lgssm_shape_supported(int nx, int ny) {
#define SQSM_CASE(X, Y) \
  if (nx == X && ny == Y) return true;
  SQSM_LGSSM_SHAPES(SQSM_CASE)
#undef SQSM_CASE
  return false;
}
}  // namespace sqsm
