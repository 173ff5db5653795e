// Mean-only upper levels of the filter scan, for the FP32 refinement passes
// of the iterated smoother.
//
// A refinement pass filters the residual model, whose factors equal those of
// the full pass before it (F, S_Q, H, S_R of every step and the prior
// factor; only the offsets and the prior mean differ).  So in every Table 3
// combine of the scan the factors A, U, Z and the gain G are those of the
// full pass, and only b and eta change, linearly, through A_i, U_i, Z_j, G
// and A_j (I - U_i G^T).  Where the upper levels are latency-bound (the
// three-role chunk levels and the top of few sequences) the full pass stores
// those per combine (FMeansTab, filter_ks3); these kernels replay the same
// Kogge-Stone rounds on (b, eta) alone through filter_combine_means, the
// operations the full operator performs, so b and eta equal those of a full
// pass bit for bit while no Tria runs.  Each level's records are then
// written whole (the full pass's final A, U, Z with the new b, eta), and the
// top's carries get their means (their factors stay as the full pass wrote
// them), so the down-sweeps and the leaf down-sweep run unchanged.
#pragma once

#include "wscan.cuh"

namespace sqsm {

// Threads of the mean-only launches: more than the at most 64 items of a
// top block, so that the staging copies below issue from four warps.
constexpr int kFMeansThreads = 128;

// A level's table for one block in shared memory: per round r < nr the
// records at the round's start ([r][cap] x FRec, cap items per round slab)
// and the combines' gain blocks ([r][cap] x FGm), then (chunk levels) the
// final records ([cap] x FRec).  Bytes of that layout:
template <typename T, int NX>
constexpr size_t fmeans_smem_bytes(int cap, int nr, bool fin) {
  return sizeof(T) * ((size_t)nr * cap * (FRec<NX>::size + FGm<NX>::size) +
                      (fin ? (size_t)cap * FRec<NX>::size : 0));
}

// n16 16-byte words from global src to shared dst, copied asynchronously by
// the block's threads (cp.async; one hardware wait in stage_wait, no spin).
SQSM_DEV void stage_async(void* dst, const void* src, int64_t n16) {
  const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
  const char* g = static_cast<const char*>(src);
  for (int64_t w = threadIdx.x; w < n16; w += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 16u * (unsigned)w),
                 "l"(g + 16 * w)
                 : "memory");
}

SQSM_DEV void stage_wait() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

// Stage the table of c items starting at item i0 of a level (tb, n items
// per round) into the layout of fmeans_smem_bytes.
template <typename T, int NX>
SQSM_DEV void stage_rounds(const FMeansTab<T>& tb, int64_t i0, int c, int cap, T* SR, T* SG,
                           T* SF) {
  constexpr int REC = FRec<NX>::size, GMS = FGm<NX>::size;
  constexpr int W = REC * sizeof(T) / 16, WG = GMS * sizeof(T) / 16;
  for (int r = 0; (1 << r) < c; ++r) {
    stage_async(SR + (int64_t)r * cap * REC, tb.rec + (r * tb.n + i0) * REC, (int64_t)c * W);
    stage_async(SG + (int64_t)r * cap * GMS, tb.gm + (r * tb.n + i0) * GMS, (int64_t)c * WG);
  }
  if (SF) stage_async(SF, tb.fin + i0 * REC, (int64_t)c * W);
}

// Kogge-Stone rounds over c items held as (b | eta) rows of SB, one thread
// per item: in round r item t combines with item t - d using the factors
// the full pass stored for that round, staged in SR / SG (cap items per
// round slab).
template <typename T, int NX>
SQSM_DEV void filter_ks_be(T* SB, int c, const T* SR, const T* SG, int cap) {
  using R = FRec<NX>;
  using GM = FGm<NX>;
  constexpr int REC = R::size, BE = 2 * NX;
  const int t = threadIdx.x;
  int r = 0;
  for (int d = 1; d < c; d <<= 1, ++r) {
    const bool act = t < c && t >= d;
    T nb[NX], ne[NX];
    if (act) {
      const T* ri = SR + (r * cap + t - d) * REC;
      const T* rj = SR + (r * cap + t) * REC;
      const T* gm = SG + (r * cap + t) * GM::size;
      const T* si = SB + (t - d) * BE;
      const T* sj = SB + t * BE;
      filter_combine_means<T, NX>(ri + R::A, ri + R::U, rj + R::Z, gm + GM::G, gm + GM::M, si,
                                  si + NX, sj, sj + NX, nb, ne);
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        SB[t * BE + i] = nb[i];
        SB[t * BE + NX + i] = ne[i];
      }
    }
    __syncthreads();
  }
}

// b and eta of item t of a record array into SB's row t.
template <typename T, int NX>
SQSM_DEV void load_be(const T* __restrict__ rec, T* sb) {
  using R = FRec<NX>;
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    sb[i] = rec[R::b + i];
    sb[NX + i] = rec[R::eta + i];
  }
}

// Chunk-scan up level (see filter_up_cs3), mean-only: one block per chunk,
// dynamic shared memory fmeans_smem_bytes(kChunkScan, nr, true).
template <typename T, int NX>
__global__ void __launch_bounds__(kFMeansThreads)
filter_up_cs_be(DevLevel lv, FMeansTab<T> tb, T* __restrict__ items, T* __restrict__ out, int nr) {
  using R = FRec<NX>;
  constexpr int REC = R::size, BE = 2 * NX, CAP = kChunkScan;
  extern __shared__ float4 fm_smem[];
  T* SR = reinterpret_cast<T*>(fm_smem);
  T* SG = SR + (int64_t)nr * CAP * REC;
  T* SF = SG + (int64_t)nr * CAP * FGm<NX>::size;
  __shared__ T SB[CAP * BE];
  const int64_t c = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  stage_rounds<T, NX>(tb, i0, cnt, CAP, SR, SG, SF);
  if (t < cnt) load_be<T, NX>(items + (i0 + t) * REC, SB + t * BE);
  stage_wait();
  filter_ks_be<T, NX>(SB, cnt, SR, SG, CAP);
  if (t < cnt) {
    T v[REC];
#pragma unroll
    for (int i = 0; i < REC; ++i) v[i] = SF[t * REC + i];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      v[R::b + i] = SB[t * BE + i];
      v[R::eta + i] = SB[t * BE + NX + i];
    }
    vstore<T, REC>(items + (i0 + t) * REC, v);
    if (t == cnt - 1) vstore<T, REC>(out + c * REC, v);
  }
}

// Top of the tree (see filter_top_ks3), mean-only: one block per sequence,
// one thread per item, dynamic shared memory fmeans_smem_bytes(cap, nr,
// false) for at most cap items per sequence; only the means of the carries
// are written.
template <typename T, int NX>
__global__ void __launch_bounds__(kFMeansThreads)
filter_top_ks_be(const int64_t* __restrict__ seq_item_off, FMeansTab<T> tb,
                 const T* __restrict__ items, T* __restrict__ carry_out, int* __restrict__ flag_out,
                 int cap, int nr) {
  using R = FRec<NX>;
  constexpr int REC = R::size, BE = 2 * NX, XS = XRow<NX>::size;
  constexpr int KS = Ks3Max<T, REC>::value;
  static_assert(KS <= kFMeansThreads, "one thread per item");
  extern __shared__ float4 fm_smem[];
  T* SR = reinterpret_cast<T*>(fm_smem);
  T* SG = SR + (int64_t)nr * cap * REC;
  __shared__ T SB[KS * BE];
  const int b = blockIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  const int t = threadIdx.x;
  stage_rounds<T, NX>(tb, i0, c, cap, SR, SG, nullptr);
  if (t < c) load_be<T, NX>(items + (i0 + t) * REC, SB + t * BE);
  stage_wait();
  filter_ks_be<T, NX>(SB, c, SR, SG, cap);
  if (t < c) {
    if (t > 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) carry_out[(i0 + t) * XS + i] = SB[(t - 1) * BE + i];
    }
    flag_out[i0 + t] = t > 0 ? 1 : 0;
  }
}

}  // namespace sqsm
