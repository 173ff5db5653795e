// Upper scan levels with one warp per chunk (see warp_ops.cuh); used for the
// levels that hold few chunks, where one thread per chunk leaves most of the
// GPU idle and each combine's latency sets the time.
#pragma once

#include "scan.cuh"
#include "warp_ops.cuh"

namespace sqsm {

constexpr int kWarpsPerBlock = 4;
constexpr int64_t kWarpLevelMaxChunks = 2048;

template <typename T, int NX> struct WFilterBuf {
  T a[FRec<NX>::size], b[FRec<NX>::size], c[FRec<NX>::size];
  T cb[NX], cU[NX * NX], nb[NX], nU[NX * NX];
  WFilterWs<T, NX> ws;
};

// Lane-parallel forms of RowsPacked::load / store for the warp kernels: a
// scan carry (vector v, lower factor L) in the XRow layout at g.
template <typename T, int NX>
SQSM_DEV void wload_carry(const T* __restrict__ g, T* v, T* L, int lane) {
  for (int i = lane; i < NX * NX; i += kWarp) {
    const int r = i / NX, q = i % NX;
    L[i] = q <= r ? g[NX + r * (r + 1) / 2 + q] : T(0);
  }
  for (int i = lane; i < NX; i += kWarp) v[i] = g[i];
}

template <typename T, int NX>
SQSM_DEV void wstore_carry(T* __restrict__ g, const T* v, const T* L, int lane) {
  for (int i = lane; i < NX * NX; i += kWarp) {
    const int r = i / NX, q = i % NX;
    if (q <= r) g[NX + r * (r + 1) / 2 + q] = L[i];
  }
  for (int i = lane; i < NX; i += kWarp) g[i] = v[i];
}

template <typename T, int NX>
__global__ void __launch_bounds__(kWarp * kWarpsPerBlock)
filter_up_w(DevLevel lv, const T* __restrict__ in, T* __restrict__ out) {
  constexpr int REC = FRec<NX>::size;
  __shared__ WFilterBuf<T, NX> sh[kWarpsPerBlock];
  const int wid = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const int64_t c = blockIdx.x * (int64_t)kWarpsPerBlock + wid;
  if (c >= lv.n_chunks) return;   // uniform per warp
  WFilterBuf<T, NX>& B = sh[wid];
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T* agg = B.a;
  T* el = B.b;
  T* tmp = B.c;
  for (int i = lane; i < REC; i += kWarp) agg[i] = in[i0 * REC + i];
  __syncwarp();
  for (int j = 1; j < cnt; ++j) {
    for (int i = lane; i < REC; i += kWarp) el[i] = in[(i0 + j) * REC + i];
    __syncwarp();
    wfilter_combine<T, NX>(agg, el, tmp, B.ws, lane);
    T* t = agg;
    agg = tmp;
    tmp = t;
  }
  for (int i = lane; i < REC; i += kWarp) out[c * REC + i] = agg[i];
}

template <typename T, int NX>
__global__ void __launch_bounds__(kWarp * kWarpsPerBlock)
filter_down_w(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
              const int* __restrict__ flag_in, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = FRec<NX>::size, XS = XRow<NX>::size;
  __shared__ WFilterBuf<T, NX> sh[kWarpsPerBlock];
  const int wid = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const int64_t c = blockIdx.x * (int64_t)kWarpsPerBlock + wid;
  if (c >= lv.n_chunks) return;
  WFilterBuf<T, NX>& B = sh[wid];
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = flag_in[c];
  wload_carry<T, NX>(carry_in + c * XS, B.cb, B.cU, lane);
  __syncwarp();
  for (int j = 0; j < cnt; ++j) {
    const int64_t it = i0 + j;
    wstore_carry<T, NX>(carry_out + it * XS, B.cb, B.cU, lane);
    if (lane == 0) flag_out[it] = flag;
    __syncwarp();
    if (j + 1 < cnt) {
      if (flag) {
        for (int i = lane; i < REC; i += kWarp) B.a[i] = items[it * REC + i];
        __syncwarp();
        wfilter_apply<T, NX>(B.cb, B.cU, B.a, B.nb, B.nU, B.ws, lane);
        for (int i = lane; i < NX * NX; i += kWarp) B.cU[i] = B.nU[i];
        if (lane < NX) B.cb[lane] = B.nb[lane];
      } else {
        for (int i = lane; i < NX; i += kWarp) B.cb[i] = items[it * REC + FRec<NX>::b + i];
        for (int i = lane; i < NX * NX; i += kWarp) B.cU[i] = items[it * REC + FRec<NX>::U + i];
        flag = 1;
      }
      __syncwarp();
    }
  }
}

template <typename T, int NX> struct WSmootherBuf {
  T a[SRec<NX>::size], b[SRec<NX>::size], c[SRec<NX>::size];
  T cg[NX], cD[NX * NX];
  WSmootherWs<T, NX> ws;
};

template <typename T, int NX>
__global__ void __launch_bounds__(kWarp * kWarpsPerBlock)
smoother_up_w(DevLevel lv, const T* __restrict__ in, T* __restrict__ out) {
  constexpr int REC = SRec<NX>::size;
  __shared__ WSmootherBuf<T, NX> sh[kWarpsPerBlock];
  const int wid = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const int64_t c = blockIdx.x * (int64_t)kWarpsPerBlock + wid;
  if (c >= lv.n_chunks) return;
  WSmootherBuf<T, NX>& B = sh[wid];
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T* agg = B.a;
  T* el = B.b;
  T* tmp = B.c;
  for (int i = lane; i < REC; i += kWarp) agg[i] = in[(i0 + cnt - 1) * REC + i];
  __syncwarp();
  for (int j = cnt - 2; j >= 0; --j) {
    for (int i = lane; i < REC; i += kWarp) el[i] = in[(i0 + j) * REC + i];
    __syncwarp();
    wsmoother_combine<T, NX>(el, agg, tmp, B.ws, lane);
    T* t = agg;
    agg = tmp;
    tmp = t;
  }
  for (int i = lane; i < REC; i += kWarp) out[c * REC + i] = agg[i];
}

template <typename T, int NX>
__global__ void __launch_bounds__(kWarp * kWarpsPerBlock)
smoother_down_w(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
                const int* __restrict__ flag_in, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = SRec<NX>::size, XS = XRow<NX>::size;
  __shared__ WSmootherBuf<T, NX> sh[kWarpsPerBlock];
  const int wid = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const int64_t c = blockIdx.x * (int64_t)kWarpsPerBlock + wid;
  if (c >= lv.n_chunks) return;
  WSmootherBuf<T, NX>& B = sh[wid];
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = flag_in[c];
  wload_carry<T, NX>(carry_in + c * XS, B.cg, B.cD, lane);
  __syncwarp();
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t it = i0 + j;
    wstore_carry<T, NX>(carry_out + it * XS, B.cg, B.cD, lane);
    if (lane == 0) flag_out[it] = flag;
    __syncwarp();
    if (j > 0) {
      if (flag) {
        for (int i = lane; i < REC; i += kWarp) B.a[i] = items[it * REC + i];
        __syncwarp();
        wsmoother_apply<T, NX>(B.a, B.cg, B.cD, B.ws, lane);
      } else {
        for (int i = lane; i < NX; i += kWarp) B.cg[i] = items[it * REC + SRec<NX>::g + i];
        for (int i = lane; i < NX * NX; i += kWarp) B.cD[i] = items[it * REC + SRec<NX>::D + i];
        flag = 1;
      }
      __syncwarp();
    }
  }
}

inline unsigned wgrid_for(int64_t chunks) {
  return (unsigned)((chunks + kWarpsPerBlock - 1) / kWarpsPerBlock);
}

}  // namespace sqsm

namespace sqsm {

// Top of the tree in one launch: when every sequence has at most KS items at
// a level, one block per sequence runs a Kogge-Stone inclusive scan of them in
// shared memory (ceil(log2 KS) dependent combines) and writes each item's
// exclusive prefix (filter) / suffix (smoother) as its carry, replacing all
// higher up- and down-levels.
// Block width: 128 (FP32) / 64 (FP64) items, fewer if the records would not
// fit in 48 KB of static shared memory.
template <typename T, int REC> struct KsMax {
  static constexpr int cap = sizeof(T) == 4 ? 128 : 64;
  static constexpr int fit = (int)((48 * 1024) / (REC * sizeof(T)) / 32 * 32);
  static constexpr int value = cap < fit ? cap : fit;
};

template <typename T, int NX>
__global__ void __launch_bounds__((KsMax<T, FRec<NX>::size>::value))
filter_top_ks(const int64_t* __restrict__ seq_item_off, const T* __restrict__ items,
              T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = FRec<NX>::size, KS = KsMax<T, REC>::value;
  __shared__ __align__(16) T S[KS * REC];
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  T mine[REC], tmp[REC];
  if (t < c) vload<T, REC>(items + (i0 + t) * REC, mine);
  for (int d = 1; d < c; d <<= 1) {
    if (t < c) vstore<T, REC>(S + t * REC, mine);
    __syncthreads();
    if (t < c && t >= d) {
      filter_combine<T, NX>(S + (t - d) * REC, mine, tmp);
      copy<T, REC>(tmp, mine);
    }
    __syncthreads();
  }
  if (t < c) vstore<T, REC>(S + t * REC, mine);
  __syncthreads();
  if (t < c) {
    if (t > 0) {
      const T* p = S + (t - 1) * REC;
      RowsPacked<T, NX>{carry_out}.store(i0 + t, p + FRec<NX>::b, p + FRec<NX>::U);
    }
    flag_out[i0 + t] = t > 0 ? 1 : 0;
  }
}

template <typename T, int NX>
__global__ void __launch_bounds__((KsMax<T, SRec<NX>::size>::value))
smoother_top_ks(const int64_t* __restrict__ seq_item_off, const T* __restrict__ items,
                T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = SRec<NX>::size, KS = KsMax<T, REC>::value;
  __shared__ __align__(16) T S[KS * REC];
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  T mine[REC], tmp[REC];
  if (t < c) vload<T, REC>(items + (i0 + t) * REC, mine);
  for (int d = 1; d < c; d <<= 1) {
    if (t < c) vstore<T, REC>(S + t * REC, mine);
    __syncthreads();
    if (t + d < c) {
      smoother_combine<T, NX>(mine, S + (t + d) * REC, tmp);
      copy<T, REC>(tmp, mine);
    }
    __syncthreads();
  }
  if (t < c) vstore<T, REC>(S + t * REC, mine);
  __syncthreads();
  if (t < c) {
    if (t + 1 < c) {
      const T* p = S + (t + 1) * REC;
      RowsPacked<T, NX>{carry_out}.store(i0 + t, p + SRec<NX>::g, p + SRec<NX>::D);
    }
    flag_out[i0 + t] = t + 1 < c ? 1 : 0;
  }
}

}  // namespace sqsm

namespace sqsm {

// Upper levels in "chunk scan" form (radix kChunkScan = one warp): the up
// kernel scans each chunk with Kogge-Stone inside one warp, overwriting the
// items with their in-chunk inclusive prefixes (filter) / suffixes (smoother)
// and writing the chunk total; the down kernel gives every item its carry in
// one step, the chunk's carry applied to the neighbour's in-chunk prefix.
constexpr int kChunkScan = 32;

template <typename T, int NX>
__global__ void __launch_bounds__(kChunkScan)
filter_up_cs(DevLevel lv, T* __restrict__ items, T* __restrict__ out) {
  constexpr int REC = FRec<NX>::size;
  __shared__ __align__(16) T S[kChunkScan * REC];
  const int64_t c = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T mine[REC], tmp[REC];
  if (t < cnt) vload<T, REC>(items + (i0 + t) * REC, mine);
  for (int d = 1; d < cnt; d <<= 1) {
    if (t < cnt) vstore<T, REC>(S + t * REC, mine);
    __syncwarp();
    if (t < cnt && t >= d) {
      filter_combine<T, NX>(S + (t - d) * REC, mine, tmp);
      copy<T, REC>(tmp, mine);
    }
    __syncwarp();
  }
  if (t < cnt) vstore<T, REC>(items + (i0 + t) * REC, mine);
  if (t == cnt - 1) vstore<T, REC>(out + c * REC, mine);
}

// The carries of one chunk (cnt consecutive items, lane j holding item j's
// vector b[NX] and lower factor U[NX*NX]) written to their contiguous block
// of XRow records at g: packed into the warp's shared rows, then copied in
// 16-byte words, lane-strided, so that every store instruction covers
// consecutive words.
template <typename T, int NX>
SQSM_DEV void warp_store_carries(T* __restrict__ g, T* sh, const T* b, const T* U, int j, int cnt,
                                 bool active) {
  constexpr int XS = XRow<NX>::size, WPR = XS * (int)sizeof(T) / 16;
  static_assert(XS * sizeof(T) % 16 == 0, "whole 16-byte words per record");
  const int lane = threadIdx.x % kWarp;
  if (active) {
    T* o = sh + j * XS;
#pragma unroll
    for (int k = 0; k < NX; ++k) o[k] = b[k];
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = 0; q <= r; ++q) o[NX + r * (r + 1) / 2 + q] = U[r * NX + q];
#pragma unroll
    for (int k = NX + NX * (NX + 1) / 2; k < XS; ++k) o[k] = T(0);
  }
  __syncwarp();
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(sh);
    float4* g4 = reinterpret_cast<float4*>(g);
    for (int k = lane; k < cnt * WPR; k += kWarp) g4[k] = s4[k];
  } else {
    const double2* s4 = reinterpret_cast<const double2*>(sh);
    double2* g4 = reinterpret_cast<double2*>(g);
    for (int k = lane; k < cnt * WPR; k += kWarp) g4[k] = s4[k];
  }
}

// The W-value rows of one chunk's cnt consecutive items (lane j holding item
// j's row v) written to their contiguous block g: staged in the warp's
// shared rows sh, then stored lane-strided, each store instruction covering
// consecutive words.
template <typename T, int W>
SQSM_DEV void warp_store_rows(T* __restrict__ g, T* sh, const T* v, int j, int cnt, bool active) {
  const int lane = threadIdx.x % kWarp;
  if (active) {
#pragma unroll
    for (int k = 0; k < W; ++k) sh[j * W + k] = v[k];
  }
  __syncwarp();
  for (int k = lane; k < cnt * W; k += kWarp) g[k] = sh[k];
}

// One thread per item of the level; each warp is one chunk.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
filter_down_cs(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
               const int* __restrict__ flag_in, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = FRec<NX>::size, XS = XRow<NX>::size;
  static_assert(kChunkScan == kWarp && kBlock % kWarp == 0, "one chunk per warp");
  __shared__ __align__(16) T SO[kBlock / kWarp][kWarp * XS];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = tid / kChunkScan;
  if (c >= lv.n_chunks) return;   // uniform per warp
  const int j = (int)(tid - c * kChunkScan);
  const int cnt = lv.count[c];
  const bool active = j < cnt;
  const int64_t i0 = lv.first[c];
  const int64_t i = i0 + j;
  const int flag = flag_in[c];
  const RowsPacked<T, NX> cin{(T*)carry_in};
  T cb[NX], cU[NX * NX];
  if (!active) {
  } else if (j == 0) {
    cin.load(c, cb, cU);
  } else if (flag) {
    T pb[NX], pU[NX * NX], el[REC];
    cin.load(c, pb, pU);
    vload<T, REC>(items + (i - 1) * REC, el);
    filter_apply<T, NX>(pb, pU, el, cb, cU);
  } else {
    load<T, NX>(items + (i - 1) * REC + FRec<NX>::b, cb);
    load<T, NX * NX>(items + (i - 1) * REC + FRec<NX>::U, cU);
  }
  warp_store_carries<T, NX>(carry_out + i0 * XS, SO[threadIdx.x / kWarp], cb, cU, j, cnt,
                            active);
  if (active) flag_out[i] = j == 0 ? flag : 1;
}

template <typename T, int NX>
__global__ void __launch_bounds__(kChunkScan)
smoother_up_cs(DevLevel lv, T* __restrict__ items, T* __restrict__ out) {
  constexpr int REC = SRec<NX>::size;
  __shared__ __align__(16) T S[kChunkScan * REC];
  const int64_t c = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T mine[REC], tmp[REC];
  if (t < cnt) vload<T, REC>(items + (i0 + t) * REC, mine);
  for (int d = 1; d < cnt; d <<= 1) {
    if (t < cnt) vstore<T, REC>(S + t * REC, mine);
    __syncwarp();
    if (t + d < cnt) {
      smoother_combine<T, NX>(mine, S + (t + d) * REC, tmp);
      copy<T, REC>(tmp, mine);
    }
    __syncwarp();
  }
  if (t < cnt) vstore<T, REC>(items + (i0 + t) * REC, mine);
  if (t == 0 && cnt > 0) vstore<T, REC>(out + c * REC, mine);
}

template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
smoother_down_cs(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
                 const int* __restrict__ flag_in, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = SRec<NX>::size, XS = XRow<NX>::size;
  static_assert(kChunkScan == kWarp && kBlock % kWarp == 0, "one chunk per warp");
  __shared__ __align__(16) T SO[kBlock / kWarp][kWarp * XS];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = tid / kChunkScan;
  if (c >= lv.n_chunks) return;   // uniform per warp
  const int j = (int)(tid - c * kChunkScan);
  const int cnt = lv.count[c];
  const bool active = j < cnt;
  const int64_t i0 = lv.first[c];
  const int64_t i = i0 + j;
  const int flag = flag_in[c];
  const RowsPacked<T, NX> cin{(T*)carry_in};
  T cg[NX], cD[NX * NX];
  if (!active) {
  } else if (j == cnt - 1) {
    cin.load(c, cg, cD);
  } else if (flag) {
    T el[REC];
    cin.load(c, cg, cD);
    vload<T, REC>(items + (i + 1) * REC, el);
    smoother_apply<T, NX>(el, cg, cD);
  } else {
    load<T, NX>(items + (i + 1) * REC + SRec<NX>::g, cg);
    load<T, NX * NX>(items + (i + 1) * REC + SRec<NX>::D, cD);
  }
  warp_store_carries<T, NX>(carry_out + i0 * XS, SO[threadIdx.x / kWarp], cg, cD, j, cnt,
                            active);
  if (active) flag_out[i] = j == cnt - 1 ? flag : 1;
}

inline unsigned cs_down_grid(int64_t chunks) {
  return (unsigned)((chunks * kChunkScan + kBlock - 1) / kBlock);
}

// Where a full filter pass stores, for one level, what the mean-only
// refinement passes replay (refine_scan.cuh); rec null: nothing is stored.
// For Kogge-Stone round r and item i of the level (n items): the record at
// the round's start at rec[(r * n + i) * FRec] and the combine's G and
// A_j (I - U_i G^T) at gm[(r * n + i) * FGm]; for chunk levels also the
// records the scan leaves at fin[i * FRec] (fin null at the top).
template <typename T> struct FMeansTab {
  T* rec;
  T* gm;
  T* fin;
  int64_t n;
};

// Filter scans with three threads per combine.  In the latency-bound top
// levels (few chunks, one warp per SM or less) a combine's chain of dependent
// instructions sets the time per Kogge-Stone round.  Thread (role r, item t)
// computes only part r of S[t - d] (x) S[t] (r = 0: A, b, eta; 1: U; 2: Z;
// each forms the factors it needs itself), which shortens that chain; role
// r runs in warps of its own, so no warp diverges.
//
// With STORE, the rounds also store what the mean-only refinement passes
// replay (FMeansTab, here offset to the first item): the records at the
// start of round r at trec[(r * n + t) * REC] and each combine's G and
// A_j (I - U_i G^T) at tgm[(r * n + t) * FGm].
template <typename T, int NX, int CAP, bool STORE = false>
SQSM_DEV void filter_ks3(T* S, int c, T* trec = nullptr, T* tgm = nullptr, int64_t n = 0) {
  using R = FRec<NX>;
  constexpr int REC = R::size, W = REC * sizeof(T) / 16, GMS = FGm<NX>::size;
  static_assert(CAP % 32 == 0, "roles in whole warps");
  const int role = threadIdx.x / CAP, t = threadIdx.x - role * CAP;
  int r = 0;
  for (int d = 1; d < c; d <<= 1, ++r) {
    if constexpr (STORE) {   // S is read-only until the barrier below
      const float4* S4 = reinterpret_cast<const float4*>(S);
      float4* D4 = reinterpret_cast<float4*>(trec + r * n * REC);
      for (int w = threadIdx.x; w < c * W; w += blockDim.x) D4[w] = S4[w];
    }
    T part[REC];
    const bool act = t < c && t >= d;
    if (act) {
      const T* ei = S + (t - d) * REC;
      const T* ej = S + t * REC;
      if (role == 0) {
        if constexpr (STORE) filter_combine<T, NX, 1>(ei, ej, part, tgm + (r * n + t) * GMS);
        else filter_combine<T, NX, 1>(ei, ej, part);
      } else if (role == 1) filter_combine<T, NX, 2>(ei, ej, part);
      else filter_combine<T, NX, 4>(ei, ej, part);
    }
    __syncthreads();
    if (act) {
      T* o = S + t * REC;
      if (role == 0) {
#pragma unroll
        for (int i = R::A; i < R::U; ++i) o[i] = part[i];      // A, b
#pragma unroll
        for (int i = R::eta; i < R::Z; ++i) o[i] = part[i];    // eta
      } else if (role == 1) {
#pragma unroll
        for (int i = R::U; i < R::eta; ++i) o[i] = part[i];
      } else {
#pragma unroll
        for (int i = R::Z; i < R::Z + NX * NX; ++i) o[i] = part[i];
      }
    }
    __syncthreads();
  }
}

// Chunk-scan up level (see filter_up_cs) with three threads per combine: one
// block of 3 x 32 threads per chunk.  STORE: also fill tb (a full pass
// followed by mean-only ones).
template <typename T, int NX, bool STORE>
__global__ void __launch_bounds__(3 * kChunkScan)
filter_up_cs3(DevLevel lv, T* __restrict__ items, T* __restrict__ out, FMeansTab<T> tb) {
  constexpr int REC = FRec<NX>::size, W = REC * sizeof(T) / 16;   // 16-byte words
  __shared__ __align__(16) T S[kChunkScan * REC];
  const int64_t c = blockIdx.x;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  float4* S4 = reinterpret_cast<float4*>(S);
  float4* I4 = reinterpret_cast<float4*>(items + i0 * REC);
  for (int w = threadIdx.x; w < cnt * W; w += blockDim.x) S4[w] = I4[w];
  __syncthreads();
  if constexpr (STORE)
    filter_ks3<T, NX, kChunkScan, true>(S, cnt, tb.rec + i0 * REC, tb.gm + i0 * FGm<NX>::size,
                                        tb.n);
  else
    filter_ks3<T, NX, kChunkScan>(S, cnt);
  for (int w = threadIdx.x; w < cnt * W; w += blockDim.x) I4[w] = S4[w];
  if constexpr (STORE) {
    float4* F4 = reinterpret_cast<float4*>(tb.fin + i0 * REC);
    for (int w = threadIdx.x; w < cnt * W; w += blockDim.x) F4[w] = S4[w];
  }
  float4* O4 = reinterpret_cast<float4*>(out + c * REC);
  for (int w = threadIdx.x; w < W; w += blockDim.x) O4[w] = S4[(cnt - 1) * W + w];
}

// Top of the tree (see filter_top_ks) with three threads per combine, for
// sequences of at most Ks3Max items at that level (64, fewer where the
// records would not fit 48 KB of static shared memory).
constexpr int ks3_max_items(int rec_bytes) {
  return (48 * 1024) / rec_bytes / 32 * 32 < 64 ? (48 * 1024) / rec_bytes / 32 * 32 : 64;
}
template <typename T, int REC> struct Ks3Max {
  static constexpr int value = ks3_max_items(REC * (int)sizeof(T));
};

template <typename T, int NX, bool STORE>
__global__ void __launch_bounds__(3 * Ks3Max<T, FRec<NX>::size>::value)
filter_top_ks3(const int64_t* __restrict__ seq_item_off, const T* __restrict__ items,
               T* __restrict__ carry_out, int* __restrict__ flag_out, FMeansTab<T> tb) {
  constexpr int REC = FRec<NX>::size, W = REC * sizeof(T) / 16;
  constexpr int KS = Ks3Max<T, REC>::value;
  __shared__ __align__(16) T S[KS * REC];
  const int b = blockIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  float4* S4 = reinterpret_cast<float4*>(S);
  const float4* I4 = reinterpret_cast<const float4*>(items + i0 * REC);
  for (int w = threadIdx.x; w < c * W; w += blockDim.x) S4[w] = I4[w];
  __syncthreads();
  if constexpr (STORE)
    filter_ks3<T, NX, KS, true>(S, c, tb.rec + i0 * REC, tb.gm + i0 * FGm<NX>::size, tb.n);
  else
    filter_ks3<T, NX, KS>(S, c);
  const int t = threadIdx.x;
  if (t < c) {
    if (t > 0) {
      const T* p = S + (t - 1) * REC;
      RowsPacked<T, NX>{carry_out}.store(i0 + t, p + FRec<NX>::b, p + FRec<NX>::U);
    }
    flag_out[i0 + t] = t > 0 ? 1 : 0;
  }
}

}  // namespace sqsm
