// Host-side enqueueing of the two scans over a plan (shared by the linear
// smoother and the IPLS loop).  Only launches kernels; no host compute on the
// data path.
#pragma once

#include <vector>

#include "wscan.cuh"
#include "refine_filter.cuh"

namespace sqsm {

// Levels of one scan (filter or smoother) for one batch layout.
// lv[l] (l = 0..Lc-1) folds the items of level l into items[l+1];
// n_items[l] is the number of items at level l (n_items[Lc] = B).
struct LevelSet {
  std::vector<DevLevel> lv;
  std::vector<int64_t> n_items;
  int64_t* leaf_chunk_off = nullptr;   // device, B+1
  // per item level l >= 1: first item of each sequence (device, B+1) and the
  // largest number of items any sequence has there (host)
  std::vector<int64_t*> seq_item_off;
  std::vector<int64_t> max_seq_items;
  int B = 0;
  // per chunk level l >= 1: 1 = one-warp Kogge-Stone chunks of 32 items,
  // 0 = sequential folds (one thread per chunk)
  std::vector<char> cs;
  bool chunk_scan(int l) const { return l < (int)cs.size() && cs[l]; }

  // Lowest item level whose per-sequence item count fits one Kogge-Stone block.
  int ks_level(int ks_max) const {
    const int Lc = (int)lv.size();
    for (int l = 1; l < Lc; ++l)
      if (max_seq_items[l] <= ks_max) return l;
    return Lc;
  }
};

// Device buffers of one scan for one (dtype, nx): items[l], carry[l],
// flag[l] for item levels l = 1..Lc (index 0 unused).
struct ScanBuffers {
  std::vector<void*> items, carry;
  std::vector<int*> flag;
};

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Kernel families, for per-kernel timing.
enum KernelKind {
  K_PARAMS = 0, K_INIT, K_SLR, K_FILTER_LEAF_UP, K_FILTER_UP, K_FILTER_DOWN, K_FILTER_LEAF_DOWN,
  K_SMOOTHER_LEAF_UP, K_SMOOTHER_UP, K_SMOOTHER_DOWN, K_SMOOTHER_LEAF_DOWN, K_LOGLIK,
  K_NUM_KINDS
};

// Optional per-launch CUDA events (recorded as external event nodes when
// the launches are captured into a graph).  Null = no instrumentation.
struct Prof {
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> rec;
  ~Prof() { clear(); }
  void clear() {
    for (auto& r : rec) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    rec.clear();
  }
  // Inside a stream capture the events become event-record nodes of the
  // graph (the external flag); outside one they are recorded as usual.
  static void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    cudaEventRecordWithFlags(
        e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
  void begin(int kind, cudaStream_t s) {
    Rec r{kind, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    record(r.a, s);
    rec.push_back(r);
  }
  void end(cudaStream_t s) { record(rec.back().b, s); }
};

struct ProfScope {
  Prof* p;
  cudaStream_t s;
  ProfScope(Prof* p_, int kind, cudaStream_t s_) : p(p_), s(s_) {
    if (p) p->begin(kind, s);
  }
  ~ProfScope() {
    if (p) p->end(s);
  }
};

// Chunk-scanned filter levels of at most this many chunks use three threads
// per combine (latency-bound); larger ones one (throughput-bound).
constexpr int64_t kCs3MaxChunks = 512;

inline bool cs3_level(const LevelSet& L, int l, bool r3) {
  return r3 && L.chunk_scan(l) && L.lv[l].n_chunks <= kCs3MaxChunks;
}

// Mean-only filter passes (FP32 refinement, refine_filter.cuh): for at most
// this many sequences the three-role levels and the top are latency-bound,
// and their combines are replayed from the table the full pass stores; for
// states smaller than kFMeansMinNx the full combine is cheaper than reading
// its factors back (measured on the population model, n_x = 1).
constexpr int kFMeansMaxSeqs = 64;
constexpr int kFMeansMinNx = 3;

// Where each level's part of that table starts (elements; -1: the level
// stores nothing) and its size, for elements of es bytes and state size nx:
// per three-role chunk level 5 Kogge-Stone rounds, at the top as many as its
// largest sequence needs; on = false (FP64, n_x < kFMeansMinNx, one leaf
// chunk per sequence, more sequences than kFMeansMaxSeqs): no table, full
// refinement passes.
// Kogge-Stone rounds over m items: d = 1, 2, 4, ... < m.
inline int ks_rounds(int64_t m) {
  int r = 0;
  while ((int64_t(1) << r) < m) ++r;
  return r;
}

struct FMeansLayout {
  std::vector<int64_t> rec, gm, fin;
  int64_t size = 0;
  bool on = false;
};

inline FMeansLayout fmeans_layout(const LevelSet& L, size_t es, int nx) {
  FMeansLayout f;
  const int Lc = (int)L.lv.size();
  if (es != 4 || nx < kFMeansMinNx || Lc <= 1 || L.B > kFMeansMaxSeqs) return f;
  const int rec = frec_size(nx), gm = fgm_size(nx);
  const int Lk = L.ks_level(ks3_max_items(rec * (int)es));
  f.rec.assign(Lc + 1, -1);
  f.gm = f.rec;
  f.fin = f.rec;
  auto add = [&](int l, int nr, bool fin) {
    const int64_t n = L.n_items[l];
    f.rec[l] = f.size;
    f.size += nr * n * rec;
    f.gm[l] = f.size;
    f.size += nr * n * gm;
    if (fin) {
      f.fin[l] = f.size;
      f.size += n * rec;
    }
  };
  for (int l = 1; l < Lk; ++l)
    if (cs3_level(L, l, true)) add(l, ks_rounds(kChunkScan), true);
  add(Lk, ks_rounds(L.max_seq_items[Lk]), false);
  f.on = true;
  return f;
}

// Allow a kernel the dynamic shared memory of its next launch where that
// exceeds the 48 KB default (a function attribute, not a stream operation,
// so it may be set while the stream is being captured).
template <typename K>
void dyn_smem(K* kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ftab (FP32, a table laid out by fmeans_layout): a full pass stores the
// factors of its three-role levels' and top's combines there, a means_only
// pass (the residual model of the pass that stored them) replays those
// levels on b and eta alone.
template <typename T, int NX, int NY, typename GV, typename FO>
void enqueue_filter(const LevelSet& L, const ScanBuffers& W, DevSeqs sq, GV gv,
                    const T* y, const T* m0, const T* N0, FO fo, double* partial,
                    int* status, cudaStream_t s, Prof* P = nullptr, T* ftab = nullptr,
                    bool means_only = false) {
  const int Lc = (int)L.lv.size();
  // FP32 takes three threads per combine at the top of the tree; FP64 records
  // and factors do not fit three such threads' registers.
  constexpr bool R3 = sizeof(T) == 4;
  constexpr int KS = R3 ? Ks3Max<T, FRec<NX>::size>::value : KsMax<T, FRec<NX>::size>::value;
  const int Lk = L.ks_level(KS);
  const FMeansLayout fm = ftab ? fmeans_layout(L, sizeof(T), NX) : FMeansLayout{};
  const bool mo = means_only && fm.on;
  auto tab = [&](int l) {
    FMeansTab<T> tb{nullptr, nullptr, nullptr, 0};
    if (fm.on && fm.rec[l] >= 0) {
      tb.rec = ftab + fm.rec[l];
      tb.gm = ftab + fm.gm[l];
      tb.fin = fm.fin[l] >= 0 ? ftab + fm.fin[l] : nullptr;
      tb.n = L.n_items[l];
    }
    return tb;
  };
  if (Lc > 1) {  // with one leaf chunk per sequence every carry is the prior
    {
      ProfScope ps(P, K_FILTER_LEAF_UP, s);
      filter_leaf_up<T, NX, NY, GV><<<grid_for(L.lv[0].n_chunks), kBlock, 0, s>>>(
          L.lv[0], sq, gv, y, m0, N0, (T*)W.items[1]);
    }
    for (int l = 1; l < Lk; ++l) {
      ProfScope ps(P, K_FILTER_UP, s);
      if constexpr (R3) {
        if (cs3_level(L, l, R3)) {
          const unsigned g = (unsigned)L.lv[l].n_chunks;
          if (mo) {
            const int nr = ks_rounds(kChunkScan);
            const size_t sm = fmeans_smem_bytes<T, NX>(kChunkScan, nr, true);
            dyn_smem(filter_up_cs_be<T, NX>, sm);
            filter_up_cs_be<T, NX><<<g, kFMeansThreads, sm, s>>>(L.lv[l], tab(l), (T*)W.items[l],
                                                                  (T*)W.items[l + 1], nr);
          }
          else if (tab(l).rec)
            filter_up_cs3<T, NX, true><<<g, 3 * kChunkScan, 0, s>>>(
                L.lv[l], (T*)W.items[l], (T*)W.items[l + 1], tab(l));
          else
            filter_up_cs3<T, NX, false><<<g, 3 * kChunkScan, 0, s>>>(
                L.lv[l], (T*)W.items[l], (T*)W.items[l + 1], tab(l));
          continue;
        }
      }
      if (L.chunk_scan(l))
        filter_up_cs<T, NX><<<(unsigned)L.lv[l].n_chunks, kChunkScan, 0, s>>>(
            L.lv[l], (T*)W.items[l], (T*)W.items[l + 1]);
      else if (L.lv[l].n_chunks <= kWarpLevelMaxChunks)
        filter_up_w<T, NX><<<wgrid_for(L.lv[l].n_chunks), kWarp * kWarpsPerBlock, 0, s>>>(
            L.lv[l], (const T*)W.items[l], (T*)W.items[l + 1]);
      else
        filter_up<T, NX><<<grid_for(L.lv[l].n_chunks), kBlock, 0, s>>>(
            L.lv[l], (const T*)W.items[l], (T*)W.items[l + 1]);
    }
    ProfScope ps(P, K_FILTER_UP, s);
    if constexpr (R3) {
      if (mo) {
        const int cap = (int)L.max_seq_items[Lk], nr = ks_rounds(cap);
        const size_t sm = fmeans_smem_bytes<T, NX>(cap, nr, false);
        dyn_smem(filter_top_ks_be<T, NX>, sm);
        filter_top_ks_be<T, NX><<<L.B, kFMeansThreads, sm, s>>>(
            L.seq_item_off[Lk], tab(Lk), (const T*)W.items[Lk], (T*)W.carry[Lk], W.flag[Lk], cap,
            nr);
      } else if (tab(Lk).rec)
        filter_top_ks3<T, NX, true><<<L.B, 3 * KS, 0, s>>>(
            L.seq_item_off[Lk], (const T*)W.items[Lk], (T*)W.carry[Lk], W.flag[Lk], tab(Lk));
      else
        filter_top_ks3<T, NX, false><<<L.B, 3 * KS, 0, s>>>(
            L.seq_item_off[Lk], (const T*)W.items[Lk], (T*)W.carry[Lk], W.flag[Lk], tab(Lk));
    } else
      filter_top_ks<T, NX><<<L.B, KS, 0, s>>>(L.seq_item_off[Lk], (const T*)W.items[Lk],
                                              (T*)W.carry[Lk], W.flag[Lk]);
  } else {
    cudaMemsetAsync(W.flag[Lc], 0, sizeof(int) * L.n_items[Lc], s);
  }
  for (int l = (Lc > 1 ? Lk : Lc) - 1; l >= 1; --l) {
    ProfScope ps(P, K_FILTER_DOWN, s);
    if (L.chunk_scan(l))
      filter_down_cs<T, NX><<<cs_down_grid(L.lv[l].n_chunks), kBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
          (T*)W.carry[l], W.flag[l]);
    else if (L.lv[l].n_chunks <= kWarpLevelMaxChunks)
      filter_down_w<T, NX><<<wgrid_for(L.lv[l].n_chunks), kWarp * kWarpsPerBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
          (T*)W.carry[l], W.flag[l]);
    else
      filter_down<T, NX><<<grid_for(L.lv[l].n_chunks), kBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
          (T*)W.carry[l], W.flag[l]);
  }
  ProfScope ps(P, K_FILTER_LEAF_DOWN, s);
  filter_leaf_down<T, NX, NY, GV, FO><<<grid_for(L.lv[0].n_chunks), kBlock, 0, s>>>(
      L.lv[0], sq, gv, y, m0, N0, (const T*)W.carry[1], W.flag[1], fo, partial, status);
}

template <typename T, int NX, int NY, typename GV, typename FO, typename SO>
void enqueue_smoother(const LevelSet& L, const ScanBuffers& W, DevSeqs sq, GV gv, FO fo, SO so,
                      int* status, cudaStream_t s, Prof* P = nullptr, bool add_nominal = false,
                      unsigned* dmax = nullptr, T* etab = nullptr) {
  const int Lc = (int)L.lv.size();
  constexpr int KS = KsMax<T, SRec<NX>::size>::value;
  const int Lk = L.ks_level(KS);
  if (Lc > 1) {
    {
      ProfScope ps(P, K_SMOOTHER_LEAF_UP, s);
      smoother_leaf_up<T, NX, NY, GV, FO><<<grid_for(L.lv[0].n_chunks), kBlock, 0, s>>>(
          L.lv[0], sq, gv, fo, (T*)W.items[1], etab);
    }
    for (int l = 1; l < Lk; ++l) {
      ProfScope ps(P, K_SMOOTHER_UP, s);
      if (L.chunk_scan(l))
        smoother_up_cs<T, NX><<<(unsigned)L.lv[l].n_chunks, kChunkScan, 0, s>>>(
            L.lv[l], (T*)W.items[l], (T*)W.items[l + 1]);
      else if (L.lv[l].n_chunks <= kWarpLevelMaxChunks)
        smoother_up_w<T, NX><<<wgrid_for(L.lv[l].n_chunks), kWarp * kWarpsPerBlock, 0, s>>>(
            L.lv[l], (const T*)W.items[l], (T*)W.items[l + 1]);
      else
        smoother_up<T, NX><<<grid_for(L.lv[l].n_chunks), kBlock, 0, s>>>(
            L.lv[l], (const T*)W.items[l], (T*)W.items[l + 1]);
    }
    ProfScope ps(P, K_SMOOTHER_UP, s);
    smoother_top_ks<T, NX><<<L.B, KS, 0, s>>>(L.seq_item_off[Lk],
                                                          (const T*)W.items[Lk], (T*)W.carry[Lk],
                                                          W.flag[Lk]);
  } else {
    cudaMemsetAsync(W.flag[Lc], 0, sizeof(int) * L.n_items[Lc], s);
  }
  for (int l = (Lc > 1 ? Lk : Lc) - 1; l >= 1; --l) {
    ProfScope ps(P, K_SMOOTHER_DOWN, s);
    if (L.chunk_scan(l))
      smoother_down_cs<T, NX><<<cs_down_grid(L.lv[l].n_chunks), kBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
          (T*)W.carry[l], W.flag[l]);
    else if (L.lv[l].n_chunks <= kWarpLevelMaxChunks)
      smoother_down_w<T, NX><<<wgrid_for(L.lv[l].n_chunks), kWarp * kWarpsPerBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
          (T*)W.carry[l], W.flag[l]);
    else
      smoother_down<T, NX><<<grid_for(L.lv[l].n_chunks), kBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
          (T*)W.carry[l], W.flag[l]);
  }
  ProfScope ps(P, K_SMOOTHER_LEAF_DOWN, s);
  smoother_leaf_down<T, NX, NY, GV, FO, SO><<<grid_for(L.lv[0].n_chunks), kBlock, 0, s>>>(
      L.lv[0], sq, gv, fo, (const T*)W.carry[1], W.flag[1], so, status, add_nominal, dmax);
}

// Record sizes (elements) of the scan buffers.
template <int NX> constexpr int filter_item_size() { return FRec<NX>::size; }
template <int NX> constexpr int smoother_item_size() { return SRec<NX>::size; }
template <int NX> constexpr int carry_size() { return NX + NX * NX; }

}  // namespace sqsm

#include "refine_scan.cuh"
