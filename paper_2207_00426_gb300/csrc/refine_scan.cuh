// Mean-only smoother scan for the refinement passes of the iterated smoother.
//
// A refinement pass smooths the residual model, whose factors equal those of
// the pass before it (F, S_Q of every step and the filter factors N^f; only
// the offsets and the prior mean differ).  So every factor-dependent
// quantity of the smoother scan -- E and D of each element (Table 4), E_ij
// and D_ij of Table 5, the smoothed factors -- is the same, and only g and
// the smoothed means change.  These kernels recompute g alone, with the full
// kernels' operations in the same order (the shared helpers of elements.cuh;
// E_ij = E_i E_j again by the same product; each element's E_k read from the
// table the full pass's leaf up-sweep wrote), so the means equal those of a
// full pass bit for bit while no Tria runs.  The factors already held in the
// rows are left as the full pass wrote them; the D fields of the scan
// records and carries are not recomputed (the words these kernels store
// whole are zeroed or left stale there, and nothing reads them in this
// pass).
#pragma once

#include "wscan.cuh"

namespace sqsm {

// Leaf up-sweep: the chunk's elements (g from the stored E_k) folded right to
// left, E and g of the result written to the item.
template <typename T, int NX, int NY, typename GV, typename FO>
__global__ void __launch_bounds__(kBlock)
smoother_leaf_up_g(DevLevel lv, DevSeqs sq, GV gv, FO fo, const T* __restrict__ etab,
                   T* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  using R = SRec<NX>;
  constexpr int REC = R::size, ES = ETab<NX>::size, W = (R::g + NX + 3) / 4 * 4;
  const int b = lv.seq[c];
  const int64_t e0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t so = sq.offsets[b] + b;
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  T agg[W], el[W], tmp[W];   // E | g (| the first words of D, unused)
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t e = e0 + j;
    const int64_t k = e - so;
    T m[NX];
    fo.load_mean(e, m);
    T* dst = (j == cnt - 1) ? agg : el;
    if (k == nb) {   // E_n = 0, g_n = m^f_n
#pragma unroll
      for (int i = 0; i < NX * NX; ++i) dst[R::E + i] = T(0);
#pragma unroll
      for (int i = 0; i < NX; ++i) dst[R::g + i] = m[i];
    } else {
      Gamma<T, NX, NY> g;
      g.load_transition(gv, sq.offsets[b] + k);
      T Ek[ES];
      vload<T, ES>(etab + e * ES, Ek);
#pragma unroll
      for (int i = 0; i < NX * NX; ++i) dst[R::E + i] = Ek[i];
      smoother_element_g<T, NX>(Ek, g.F, g.c, m, dst + R::g);
    }
    if (j != cnt - 1) {
      smoother_combine_g<T, NX>(el + R::E, el + R::g, agg + R::E, agg + R::g, tmp + R::E,
                                tmp + R::g);
      copy<T, R::g + NX>(tmp, agg);
    }
  }
#pragma unroll
  for (int i = R::g + NX; i < W; ++i) agg[i] = T(0);
  vstore<T, W>(items + c * REC, agg);
}

// Chunk scan of an upper level (see smoother_up_cs), E and g only.
template <typename T, int NX>
__global__ void __launch_bounds__(kChunkScan)
smoother_up_cs_g(DevLevel lv, T* __restrict__ items, T* __restrict__ out) {
  using R = SRec<NX>;
  constexpr int REC = R::size, W = (R::g + NX + 3) / 4 * 4;
  __shared__ __align__(16) T S[kChunkScan * W];
  const int64_t c = blockIdx.x;
  const int t = threadIdx.x;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T mine[W], tmp[W];
  if (t < cnt) vload<T, W>(items + (i0 + t) * REC, mine);
  for (int d = 1; d < cnt; d <<= 1) {
    if (t < cnt) vstore<T, W>(S + t * W, mine);
    __syncwarp();
    if (t + d < cnt) {
      const T* o = S + (t + d) * W;
      smoother_combine_g<T, NX>(mine + R::E, mine + R::g, o + R::E, o + R::g, tmp + R::E,
                                tmp + R::g);
      copy<T, R::g + NX>(tmp, mine);
    }
    __syncwarp();
  }
  if (t < cnt) vstore<T, W>(items + (i0 + t) * REC, mine);
  if (t == 0 && cnt > 0) vstore<T, W>(out + c * REC, mine);
}

// Top of the tree (see smoother_top_ks), E and g only; writes each item's
// carry g (the first words of its packed carry record).
template <typename T, int NX>
__global__ void __launch_bounds__((KsMax<T, SRec<NX>::size>::value))
smoother_top_ks_g(const int64_t* __restrict__ seq_item_off, const T* __restrict__ items,
                  T* __restrict__ carry_out, int* __restrict__ flag_out) {
  using R = SRec<NX>;
  constexpr int REC = R::size, KS = KsMax<T, REC>::value, W = (R::g + NX + 3) / 4 * 4;
  constexpr int XS = XRow<NX>::size;
  __shared__ __align__(16) T S[KS * W];
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  T mine[W], tmp[W];
  if (t < c) vload<T, W>(items + (i0 + t) * REC, mine);
  for (int d = 1; d < c; d <<= 1) {
    if (t < c) vstore<T, W>(S + t * W, mine);
    __syncthreads();
    if (t + d < c) {
      const T* o = S + (t + d) * W;
      smoother_combine_g<T, NX>(mine + R::E, mine + R::g, o + R::E, o + R::g, tmp + R::E,
                                tmp + R::g);
      copy<T, R::g + NX>(tmp, mine);
    }
    __syncthreads();
  }
  if (t < c) vstore<T, W>(S + t * W, mine);
  __syncthreads();
  if (t < c) {
    if (t + 1 < c) {
      const T* p = S + (t + 1) * W;
      T* co = carry_out + (i0 + t) * XS;
#pragma unroll
      for (int i = 0; i < NX; ++i) co[i] = p[R::g + i];
    }
    flag_out[i0 + t] = t + 1 < c ? 1 : 0;
  }
}

// Chunk down-sweep (see smoother_down_cs), g only: each item's carry g.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
smoother_down_cs_g(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
                   const int* __restrict__ flag_in, T* __restrict__ carry_out,
                   int* __restrict__ flag_out) {
  using R = SRec<NX>;
  constexpr int REC = R::size, XS = XRow<NX>::size, W = (R::g + NX + 3) / 4 * 4;
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
  T cg[NX], zD[NX * NX];
#pragma unroll
  for (int q = 0; q < NX * NX; ++q) zD[q] = T(0);
  if (!active) {
  } else if (j == cnt - 1) {
    cin.load_mean(c, cg);
  } else if (flag) {
    T el[W];
    cin.load_mean(c, cg);
    vload<T, W>(items + (i + 1) * REC, el);
    smoother_apply_g<T, NX>(el + R::E, el + R::g, cg);
  } else {
    load<T, NX>(items + (i + 1) * REC + R::g, cg);
  }
  warp_store_carries<T, NX>(carry_out + i0 * XS, SO[threadIdx.x / kWarp], cg, zD, j, cnt,
                            active);
  if (active) flag_out[i] = j == cnt - 1 ? flag : 1;
}

// Leaf down-sweep (see smoother_leaf_down with add_nominal), means only: the
// RTS steps' g from the stored E_k, the new nominal mean (previous + the
// deviation) written into the mean words of each row, its factor words kept.
template <typename T, int NX, int NY, typename GV, typename FO>
__global__ void __launch_bounds__(kBlock)
smoother_leaf_down_g(DevLevel lv, DevSeqs sq, GV gv, FO fo, const T* __restrict__ etab,
                     const T* __restrict__ carry, const int* __restrict__ flag,
                     RowsPacked<T, NX> out_rows, int* status) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int ES = ETab<NX>::size, MV = XRow<NX>::mvec, XS = XRow<NX>::size;
  const int b = lv.seq[c];
  const int64_t e0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t r0 = sq.offsets[b] + b;
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  T gm[NX];
  if (flag[c]) RowsPacked<T, NX>{(T*)carry}.load_mean(c, gm);
  bool ok = true;
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t e = e0 + j;
    const int64_t k = e - r0;
    T m[NX];
    fo.load_mean(e, m);
    if (k == nb) {
      copy<T, NX>(m, gm);
    } else {
      Gamma<T, NX, NY> g;
      g.load_transition(gv, sq.offsets[b] + k);
      T Ek[ES], gk[NX];
      vload<T, ES>(etab + e * ES, Ek);
      smoother_element_g<T, NX>(Ek, g.F, g.c, m, gk);
      smoother_apply_g<T, NX>(Ek, gk, gm);
    }
    // the row's leading words hold the mean (then factor entries): read them
    // whole, replace the mean, write them back
    T w[MV];
    T* row = out_rows.rec + e * XS;
    vload<T, MV>(row, w);
#pragma unroll
    for (int i = 0; i < NX; ++i) w[i] = w[i] + gm[i];
    vstore<T, MV>(row, w);
#pragma unroll
    for (int i = 0; i < NX; ++i) ok = ok && finite(gm[i]);
  }
  if (!ok) flag_status(status, 8);
}

// Enqueues the mean-only smoother scan when the sequences span more than one
// leaf chunk (the full pass's leaf up-sweep then wrote every E_k) and every
// upper level of L is a chunk-scan level (the shape the default scan takes
// below 160000 items per level); returns false otherwise, and the caller runs
// the full scan.
template <typename T, int NX, int NY, typename GV, typename FO>
bool enqueue_smoother_means(const LevelSet& L, const ScanBuffers& W, DevSeqs sq, GV gv, FO fo,
                            RowsPacked<T, NX> so, const T* etab, int* status, cudaStream_t s,
                            Prof* P = nullptr) {
  const int Lc = (int)L.lv.size();
  constexpr int KS = KsMax<T, SRec<NX>::size>::value;
  const int Lk = L.ks_level(KS);
  if (Lc <= 1) return false;
  for (int l = 1; l < Lk; ++l)
    if (!L.chunk_scan(l)) return false;
  {
    {
      ProfScope ps(P, K_SMOOTHER_LEAF_UP, s);
      smoother_leaf_up_g<T, NX, NY, GV, FO><<<grid_for(L.lv[0].n_chunks), kBlock, 0, s>>>(
          L.lv[0], sq, gv, fo, etab, (T*)W.items[1]);
    }
    for (int l = 1; l < Lk; ++l) {
      ProfScope ps(P, K_SMOOTHER_UP, s);
      smoother_up_cs_g<T, NX><<<(unsigned)L.lv[l].n_chunks, kChunkScan, 0, s>>>(
          L.lv[l], (T*)W.items[l], (T*)W.items[l + 1]);
    }
    ProfScope ps(P, K_SMOOTHER_UP, s);
    smoother_top_ks_g<T, NX><<<L.B, KS, 0, s>>>(L.seq_item_off[Lk], (const T*)W.items[Lk],
                                                (T*)W.carry[Lk], W.flag[Lk]);
  }
  for (int l = Lk - 1; l >= 1; --l) {
    ProfScope ps(P, K_SMOOTHER_DOWN, s);
    smoother_down_cs_g<T, NX><<<cs_down_grid(L.lv[l].n_chunks), kBlock, 0, s>>>(
        L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1],
        (T*)W.carry[l], W.flag[l]);
  }
  ProfScope ps(P, K_SMOOTHER_LEAF_DOWN, s);
  smoother_leaf_down_g<T, NX, NY, GV, FO><<<grid_for(L.lv[0].n_chunks), kBlock, 0, s>>>(
      L.lv[0], sq, gv, fo, etab, (const T*)W.carry[1], W.flag[1], so, status);
  return true;
}

}  // namespace sqsm
