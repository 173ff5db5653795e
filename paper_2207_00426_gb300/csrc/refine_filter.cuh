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

// Hint the cache lines of n elements at p into L1, the block's threads
// taking one line each in turn (the whole table of a block's rounds fits
// L1, so only the first round waits on memory).
template <typename T>
SQSM_DEV void prefetch_l1(const T* p, int64_t n) {
  constexpr int64_t LINE = 128 / sizeof(T);
  if (n <= 0) return;
  for (int64_t k = threadIdx.x * LINE; k < n + LINE - 1; k += blockDim.x * LINE) {
    const T* a = p + (k < n ? k : n - 1);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
  }
}

// The table of the rounds of c items starting at item i0 of a level (and,
// for chunk levels, their final records) into L1.
template <typename T, int NX>
SQSM_DEV void prefetch_rounds(const FMeansTab<T>& tb, int64_t i0, int c) {
  constexpr int REC = FRec<NX>::size, GMS = FGm<NX>::size;
  for (int r = 0; (1 << r) < c; ++r) {
    prefetch_l1(tb.rec + (r * tb.n + i0) * REC, (int64_t)c * REC);
    prefetch_l1(tb.gm + (r * tb.n + i0) * GMS, (int64_t)c * GMS);
  }
  if (tb.fin) prefetch_l1(tb.fin + i0 * REC, (int64_t)c * REC);
}

// Kogge-Stone rounds over c items held as (b | eta) rows of SB, one thread
// per item: in round r item t combines with item t - d using the factors
// stored for that round (trec, tgm offset to the first item, n items per
// round, as in filter_ks3).
template <typename T, int NX>
SQSM_DEV void filter_ks_be(T* SB, int c, const T* __restrict__ trec, const T* __restrict__ tgm,
                           int64_t n) {
  using R = FRec<NX>;
  using GM = FGm<NX>;
  constexpr int REC = R::size, BE = 2 * NX, ZW = REC - R::Z;
  static_assert(R::Z % 4 == 0 && ZW % 4 == 0, "Z starts a 16-byte word");
  const int t = threadIdx.x;
  int r = 0;
  for (int d = 1; d < c; d <<= 1, ++r) {
    const bool act = t < c && t >= d;
    T nb[NX], ne[NX];
    if (act) {
      T ri[REC], zj[ZW], gm[GM::size];
      vload<T, REC>(trec + (r * n + t - d) * REC, ri);
      vload<T, ZW>(trec + (r * n + t) * REC + R::Z, zj);
      vload<T, GM::size>(tgm + (r * n + t) * GM::size, gm);
      const T* si = SB + (t - d) * BE;
      const T* sj = SB + t * BE;
      filter_combine_means<T, NX>(ri + R::A, ri + R::U, zj, gm + GM::G, gm + GM::M, si, si + NX,
                                  sj, sj + NX, nb, ne);
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

// Chunk-scan up level (see filter_up_cs3), mean-only: one warp per chunk.
template <typename T, int NX>
__global__ void __launch_bounds__(kChunkScan)
filter_up_cs_be(DevLevel lv, FMeansTab<T> tb, T* __restrict__ items, T* __restrict__ out) {
  using R = FRec<NX>;
  constexpr int REC = R::size, BE = 2 * NX;
  __shared__ T SB[kChunkScan * BE];
  const int64_t c = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  prefetch_rounds<T, NX>(tb, i0, cnt);
  if (t < cnt) load_be<T, NX>(items + (i0 + t) * REC, SB + t * BE);
  __syncthreads();
  filter_ks_be<T, NX>(SB, cnt, tb.rec + i0 * REC, tb.gm + i0 * FGm<NX>::size, tb.n);
  if (t < cnt) {
    T v[REC];
    vload<T, REC>(tb.fin + (i0 + t) * REC, v);
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
// one thread per item; only the means of the carries are written.
template <typename T, int NX>
__global__ void __launch_bounds__(Ks3Max<T, FRec<NX>::size>::value)
filter_top_ks_be(const int64_t* __restrict__ seq_item_off, FMeansTab<T> tb,
                 const T* __restrict__ items, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  using R = FRec<NX>;
  constexpr int REC = R::size, BE = 2 * NX, XS = XRow<NX>::size;
  constexpr int KS = Ks3Max<T, REC>::value;
  __shared__ T SB[KS * BE];
  const int b = blockIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  const int t = threadIdx.x;
  prefetch_rounds<T, NX>(tb, i0, c);
  if (t < c) load_be<T, NX>(items + (i0 + t) * REC, SB + t * BE);
  __syncthreads();
  filter_ks_be<T, NX>(SB, c, tb.rec + i0 * REC, tb.gm + i0 * FGm<NX>::size, tb.n);
  if (t < c) {
    if (t > 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) carry_out[(i0 + t) * XS + i] = SB[(t - 1) * BE + i];
    }
    flag_out[i0 + t] = t > 0 ? 1 : 0;
  }
}

}  // namespace sqsm
