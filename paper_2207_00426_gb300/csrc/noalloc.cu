// sqsm_lgssm_smooth_noalloc: the linear smoother of sqsm_lgssm_smooth for
// callers that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is unavailable or not
// allowed -- for example inside a memory pool or allocator callback, in a
// process whose device memory is fully reserved up front by a framework, or
// in a real-time loop where an allocation (and the implicit device
// synchronisation of cudaFree) would break its timing guarantees.  Such a
// caller cannot create an sqsm_ctx (the context allocates its workspace), so
// this entry point takes no context and keeps every scratch buffer of the
// scan -- level tables, per-level scan items, carries, flags and the partial
// log-likelihood sums -- in one fixed-size array that is part of the loaded
// library image (kNoAllocScratchBytes per device, held until the process
// exits).
//
// Scan shape: leaf chunks of 4 steps and radix-4 folds at every upper level
// below the Kogge-Stone top block -- the shape of a context created with
// leaf_chunk = 4, radix = 4, whose results it reproduces bit for bit.  The
// default shape of a context (leaf 3 or 4, 32-item warp chunk scans on small
// levels) brackets the combines differently, so against a default context
// the results agree to rounding only.
//
// The scratch is shared by every call on a device and keeps the previous
// call's contents; everything a call reads is written (or cleared) by that
// same call first.  Calls whose GPU work overlaps -- on different streams or
// from different host threads -- race on the scratch and must be serialised
// by the caller.
#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <initializer_list>
#include <mutex>

#include "../../include/sqsm.h"
#include "dispatch.h"

using namespace sqsm;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxLevels = 40;   // per scan; n <= 2^31 needs at most 17 at radix 4

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

// Device address of g_scratch per device, looked up once with that device
// current (in host code g_scratch names a host-side stand-in, not a device
// address).  The address belongs to the CUDA context the library's device
// code was loaded into; if the caller resets the device (cudaDeviceReset)
// a new primary context loads the code again, possibly at another address.
// So each entry remembers the unique id of its context, and a call made
// under a different context repeats the look-up.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
};
ScratchSlot g_slots[kMaxDevices];
std::mutex g_setup_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the calling thread's current CUDA context (made current by the
// runtime call before); 0 and false if it cannot be read.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) !=
            cudaSuccess ||
        q0 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess)
      return false;
    get_current = (CtxGetCurrentFn)f0;
    get_id = (CtxGetIdFn)f1;
  }
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return SQSM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  // cudaSetDevice on the current device initialises its primary context
  // and makes it current, so that its id can be read
  if (cudaSetDevice(dev) != cudaSuccess) return SQSM_ERR_CUDA;
  unsigned long long id = 0;
  if (!current_context_id(&id)) return SQSM_ERR_CUDA;
  ScratchSlot& slot = g_slots[dev];
  if (!slot.ptr || slot.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SQSM_ERR_CUDA;
    slot.ptr = p;
    slot.ctx_id = id;
  }
  *out = slot.ptr;
  return SQSM_OK;
}

// Fills the chunk tables of all levels of one sequence (chunk c of a level
// covers items [c * size, min((c + 1) * size, items))).
struct TableDesc {
  int nlev;
  int64_t items[2 * kMaxLevels];
  int32_t size[2 * kMaxLevels];
  int64_t* first[2 * kMaxLevels];
  int32_t* count[2 * kMaxLevels];
  int32_t* seq[2 * kMaxLevels];
  int64_t* offsets;         // {0, n}
  int64_t* leaf_chunk_off;  // {0, filter leaf chunks}
  int64_t n, leaf_chunks;
  int nso;                  // per-level sequence item offsets {0, items}
  int64_t* so[2 * kMaxLevels];
  int64_t so_val[2 * kMaxLevels];
};

__global__ void fill_tables(TableDesc t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    t.offsets[0] = 0;
    t.offsets[1] = t.n;
    t.leaf_chunk_off[0] = 0;
    t.leaf_chunk_off[1] = t.leaf_chunks;
    for (int l = 0; l < t.nso; ++l) {
      t.so[l][0] = 0;
      t.so[l][1] = t.so_val[l];
    }
  }
  for (int l = 0; l < t.nlev; ++l) {
    const int64_t nch = (t.items[l] + t.size[l] - 1) / t.size[l];
    if (i < nch) {
      t.first[l][i] = i * t.size[l];
      const int64_t rest = t.items[l] - i * t.size[l];
      t.count[l][i] = (int32_t)(rest < t.size[l] ? rest : t.size[l]);
      t.seq[l][i] = 0;
    }
  }
}

struct Carver {
  unsigned char* base;
  size_t used = 0;
  void* take(size_t bytes) {
    used = (used + 255) & ~size_t(255);
    void* p = base ? base + used : nullptr;
    used += bytes;
    return p;
  }
};

// Lays out one scan (levels of `items0` items, leaf chunk L0, radix R) in the
// scratch; with base == nullptr only measures.
bool carve_scan(Carver& cv, int64_t items0, int L0, int R, size_t es, size_t rec, size_t crec,
                LevelSet& L, ScanBuffers& W, TableDesc& td) {
  L.lv.clear();
  L.seq_item_off.clear();
  L.max_seq_items.clear();
  L.B = 1;
  L.n_items.assign(1, items0);
  int64_t items = items0;
  int size = L0;
  for (;;) {
    if (td.nlev >= 2 * kMaxLevels) return false;
    const int64_t nch = (items + size - 1) / size;
    DevLevel d;
    d.n_chunks = nch;
    d.first = (int64_t*)cv.take(sizeof(int64_t) * nch);
    d.count = (int32_t*)cv.take(sizeof(int32_t) * nch);
    d.seq = (int32_t*)cv.take(sizeof(int32_t) * nch);
    td.items[td.nlev] = items;
    td.size[td.nlev] = size;
    td.first[td.nlev] = const_cast<int64_t*>(d.first);
    td.count[td.nlev] = const_cast<int32_t*>(d.count);
    td.seq[td.nlev] = const_cast<int32_t*>(d.seq);
    ++td.nlev;
    L.lv.push_back(d);
    L.n_items.push_back(nch);
    // one sequence: its items at the next level are [0, nch)
    int64_t* so = (int64_t*)cv.take(2 * sizeof(int64_t));
    td.so[td.nso] = so;
    td.so_val[td.nso] = nch;
    ++td.nso;
    if (L.seq_item_off.empty()) {
      L.seq_item_off.push_back(nullptr);
      L.max_seq_items.push_back(0);
    }
    L.seq_item_off.push_back(so);
    L.max_seq_items.push_back(nch);
    items = nch;
    size = R;
    if (nch == 1) break;
  }
  const size_t Lc = L.lv.size();
  W.items.assign(Lc + 1, nullptr);
  W.carry.assign(Lc + 1, nullptr);
  W.flag.assign(Lc + 1, nullptr);
  for (size_t l = 1; l <= Lc; ++l) {
    W.items[l] = cv.take(es * rec * L.n_items[l]);
    W.carry[l] = cv.take(es * crec * L.n_items[l]);
    W.flag[l] = (int*)cv.take(sizeof(int) * L.n_items[l]);
  }
  return true;
}

}  // namespace

extern "C" int sqsm_lgssm_smooth_noalloc(int dtype, int nx, int ny, int64_t n, const void* F,
                                         int64_t sF, const void* c, int64_t sc, const void* SQ,
                                         int64_t sSQ, const void* H, int64_t sH, const void* d,
                                         int64_t sd, const void* SR, int64_t sSR, const void* m0,
                                         const void* N0, const void* y, void* mf, void* Nf,
                                         void* ms, void* Ns, double* loglik, void* stream) {
  if (dtype != SQSM_F32 && dtype != SQSM_F64) return SQSM_ERR_INVALID_ARG;
  if (n < 1 || nx < 1 || ny < 1 || nx > 8 || ny > 8) return SQSM_ERR_INVALID_ARG;
  if (!lgssm_shape_supported(nx, ny)) return SQSM_ERR_UNSUPPORTED;
  if (!F || !c || !SQ || !H || !d || !SR || !m0 || !N0 || !y || !mf || !Nf || !ms || !Ns)
    return SQSM_ERR_INVALID_ARG;
  if (sF < 0 || sc < 0 || sSQ < 0 || sH < 0 || sd < 0 || sSR < 0) return SQSM_ERR_INVALID_ARG;
  const uintptr_t es_mask = (dtype == SQSM_F64 ? 8 : 4) - 1;
  for (const void* q : {F, c, SQ, H, d, SR, m0, N0, y, (const void*)mf, (const void*)Nf,
                        (const void*)ms, (const void*)Ns})
    if (reinterpret_cast<uintptr_t>(q) & es_mask) return SQSM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(loglik) & 7) return SQSM_ERR_INVALID_ARG;
  // an error the caller has pending stays theirs: run nothing, clear nothing
  if (cudaPeekAtLastError() != cudaSuccess) return SQSM_ERR_CUDA;
  // leaf chunks of 4 steps, radix-4 folds: the scan shape of a context with
  // leaf_chunk = 4, radix = 4
  const int L0 = 4, R = 4;
  const size_t es = dtype == SQSM_F64 ? 8 : 4;
  const size_t frec = frec_size(nx), srec = srec_size(nx),
               crec = std::max(nx + nx * nx, xrow_size(nx));   // carries: XRow records

  // measure first: reject problems that do not fit before touching the GPU
  for (int pass = 0; pass < 2; ++pass) {
    void* base = nullptr;
    if (pass == 1) {
      int dev = -1;
      if (cudaGetDevice(&dev) != cudaSuccess) return SQSM_ERR_CUDA;
      const int rc = scratch_address(dev, &base);
      if (rc != SQSM_OK) return rc;
    }
    Carver cv{(unsigned char*)base};
    TableDesc td{};
    LevelSet Lf, Ls;
    ScanBuffers Wf, Ws;
    td.offsets = (int64_t*)cv.take(2 * sizeof(int64_t));
    td.leaf_chunk_off = (int64_t*)cv.take(2 * sizeof(int64_t));
    if (!carve_scan(cv, n, L0, R, es, frec, crec, Lf, Wf, td) ||
        !carve_scan(cv, n + 1, L0, R, es, srec, crec, Ls, Ws, td))
      return SQSM_ERR_TOO_LARGE;
    double* partial = (double*)cv.take(sizeof(double) * Lf.lv[0].n_chunks);
    if (cv.used > kNoAllocScratchBytes) return SQSM_ERR_TOO_LARGE;
    if (pass == 0) continue;

    cudaStream_t s = (cudaStream_t)stream;
    td.n = n;
    td.leaf_chunks = Lf.lv[0].n_chunks;
    Lf.leaf_chunk_off = td.leaf_chunk_off;
    const int64_t widest = Ls.lv[0].n_chunks;
    fill_tables<<<(unsigned)((widest + 255) / 256), 256, 0, s>>>(td);
    DevSeqs sq;
    sq.B = 1;
    sq.offsets = td.offsets;
    sq.leaf_chunk_off = td.leaf_chunk_off;
    LgssmArgs a{nx, ny, F, c, SQ, H, d, SR, sF, sc, sSQ, sH, sd, sSR, m0, N0, y,
                mf, Nf, ms, Ns, nullptr};
    const int rc = dtype == SQSM_F32
                       ? lgssm_enqueue_f32(a, Lf, Wf, Ls, Ws, sq, partial, nullptr, s)
                       : lgssm_enqueue_f64(a, Lf, Wf, Ls, Ws, sq, partial, nullptr, s);
    if (rc) return rc;
    if (loglik) enqueue_loglik_reduce(sq, partial, loglik, nullptr, s);
    if (cudaGetLastError() != cudaSuccess) return SQSM_ERR_CUDA;
  }
  return SQSM_OK;
}
