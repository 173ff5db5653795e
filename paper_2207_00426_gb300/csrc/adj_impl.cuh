// Enqueue of one NLL + gradient evaluation (forward IPLS, the linearisation
// pass at the final trajectory, and the fixed-point adjoint iterations).
#pragma once

#include <algorithm>

#include "adjoint_kernels.cuh"
#include "dispatch.h"

namespace sqsm {

constexpr int kAdjPerStepMaxLeaf = 8;

// Upper levels 1 .. Lk-1 of an adjoint scan (items[1] already written by
// the leaf up-sweep), then the Kogge-Stone top over the items of level Lk.
template <typename T, bool FWD>
void adj_scan_up(const LevelSet& L, const ScanBuffers& W, int Lk, cudaStream_t s) {
  constexpr int KS = KsMax<T, MapRec<5>::size>::value;
  for (int l = 1; l < Lk; ++l)
    if (L.chunk_scan(l))
      adj_up_cs<T, FWD><<<(unsigned)L.lv[l].n_chunks, kChunkScan, 0, s>>>(
          L.lv[l], (T*)W.items[l], (T*)W.items[l + 1]);
    else
      adj_up<T, FWD><<<grid_for(L.lv[l].n_chunks), kBlock, 0, s>>>(L.lv[l], (const T*)W.items[l],
                                                                   (T*)W.items[l + 1]);
  adj_top_ks<T, FWD><<<L.B, KS, 0, s>>>(L.seq_item_off[Lk], (const T*)W.items[Lk],
                                         (T*)W.carry[Lk], W.flag[Lk]);
}

// Down-sweep of an adjoint scan from the carries of level `top` to level 1.
template <typename T, bool FWD>
void adj_scan_down(const LevelSet& L, const ScanBuffers& W, int top, cudaStream_t s) {
  for (int l = top - 1; l >= 1; --l)
    if (L.chunk_scan(l))
      adj_down_cs<T, FWD><<<cs_down_grid(L.lv[l].n_chunks), kBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1], (T*)W.carry[l],
          W.flag[l]);
    else
      adj_down<T, FWD><<<grid_for(L.lv[l].n_chunks), kBlock, 0, s>>>(
          L.lv[l], (const T*)W.items[l], (const T*)W.carry[l + 1], W.flag[l + 1], (T*)W.carry[l],
          W.flag[l]);
}

template <typename T>
void adj_enqueue(const IplsArgs& a, const AdjArgs& g, const LevelSet& Lf, const ScanBuffers& Wf,
                 const LevelSet& Ls, const ScanBuffers& Ws, const ScanBuffers& Wa, DevSeqs sq,
                 double* partial, int* status, cudaStream_t s) {
  constexpr int NX = 5, NY = 2, X = XRec<NX>::size, MREC = MapRec<NX>::size;
  const int64_t rows = Ls.n_items[0];
  // 1. Alg. 3 for M iterations: the nominal trajectory lands in a.ms / a.Ns.
  IplsArgs fw = a;
  fw.loglik = nullptr;
  if (a.M > 0) {
    if (sizeof(T) == 4) ipls_enqueue_f32(fw, Lf, Wf, Ls, Ws, sq, partial, status, s);
    else ipls_enqueue_f64(fw, Lf, Wf, Ls, Ws, sq, partial, status, s);
  } else {
    cudaMemcpyAsync(a.ms, a.init_ms, sizeof(T) * NX * rows, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(a.Ns, a.init_Ns, sizeof(T) * NX * NX * rows, cudaMemcpyDeviceToDevice, s);
  }
  // 2. linearise at it (printed absolute form), filter and smoother once more,
  //    and the pseudo log-likelihood of that linearisation.
  cudaMemcpyAsync(g.nom_m, a.ms, sizeof(T) * NX * rows, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(g.nom_N, a.Ns, sizeof(T) * NX * NX * rows, cudaMemcpyDeviceToDevice, s);
  const RowsSplit<T, NX> nom{(T*)g.nom_m, (T*)g.nom_N}, fo{(T*)a.mf, (T*)a.Nf},
      so{(T*)g.ms2, (T*)g.Ns2};
  launch_ct_slr<T, true>(grid_for(Lf.lv[0].n_chunks * a.leaf), s, a.linearization, Lf.lv[0],
                         a.leaf, sq, (const CTParams<T>*)a.params, 0, nom, (const T*)a.y, (T*)a.F,
                         (T*)nullptr,
                         (T*)nullptr, (T*)nullptr, (T*)nullptr, (T*)nullptr);
  const GammaPacked<T> gv{(T*)a.F};
  enqueue_filter<T, NX, NY>(Lf, Wf, sq, gv, (const T*)a.y, (const T*)a.m0, (const T*)a.N0, fo,
                            partial, status, s);
  enqueue_smoother<T, NX, NY>(Ls, Ws, sq, gv, fo, so, status, s);
  enqueue_loglik_reduce(sq, partial, g.ll, status, s);
  adj_nll_kernel<<<1, 1, 0, s>>>(sq.B, g.ll, -1.0, g.nll);
  // how far n* is from a fixed point of Alg. 3: the relative change of the
  // smoothing means in that one more iteration (words 2, 3)
  unsigned* words = (unsigned*)g.change_words;
  const unsigned change_blocks =
      (unsigned)std::min<int64_t>((X * rows + 255) / 256, 4 * 152);
  cudaMemsetAsync(words, 0, 4 * sizeof(unsigned), s);
  adj_change_partial<T><<<change_blocks, 256, 0, s>>>(NX * rows, (const T*)g.ms2,
                                                     (const T*)g.nom_m, words + 2);
  // 3. per-step tables of that linearisation (fixed over the iterations)
  AdjBufs ab{a.mf, a.Nf, g.ms2, g.Ns2, g.nom_m, g.nom_N, a.y, a.F,
             g.dir, g.dfilt, g.gbar, g.ktab, g.rtab, g.stab};
  adj_tables_kernel<T><<<grid_for(Lf.lv[0].n_chunks * a.leaf), kBlock, 0, s>>>(
      Lf.lv[0], a.leaf, (const CTParams<T>*)a.params, ab, a.linearization == 0);
  // 4. fixed-point iterations of the adjoint (NLL = -l, so lbar = -1)
  const T lbar = T(-1);
  T* lam_a = (T*)g.lam_a;
  T* lam_b = (T*)g.lam_b;
  cudaMemsetAsync(lam_a, 0, sizeof(T) * X * rows, s);
  cudaMemsetAsync(g.dir, 0, sizeof(T) * X * rows, s);   // step 1 of lam = 0
  const int Lc = (int)Lf.lv.size();
  const int Lk = Lf.ks_level(KsMax<T, MREC>::value);
  const unsigned slr_blocks = grid_for(Ls.lv[0].n_chunks * a.leaf);
  // leaf down-sweeps: one thread per step for short leaf chunks (each replays
  // at most kAdjPerStepMaxLeaf - 1 maps), one per chunk for long ones
  const bool per_step = a.leaf <= kAdjPerStepMaxLeaf;
  const unsigned down_grid = grid_for(Lf.lv[0].n_chunks * (per_step ? a.leaf : 1));
  for (int it = 0; it < g.iters; ++it) {
    // smoother adjoint: forward-in-time scan of maps
    if (Lc > 1) {
      adj_smoother_leaf_up<T><<<grid_for(Lf.lv[0].n_chunks), kBlock, 0, s>>>(Lf.lv[0], sq, ab,
                                                                             (T*)Wa.items[1]);
      adj_scan_up<T, true>(Lf, Wa, Lk, s);
    } else {
      cudaMemsetAsync(Wa.flag[Lc], 0, sizeof(int) * Lf.n_items[Lc], s);
    }
    adj_scan_down<T, true>(Lf, Wa, Lc > 1 ? Lk : Lc, s);
    adj_smoother_leaf_down<T><<<down_grid, kBlock, 0, s>>>(
        Lf.lv[0], a.leaf, per_step, sq, ab, (const T*)Wa.carry[1], Wa.flag[1]);
    // filter adjoint: backward-in-time scan of maps
    if (Lc > 1) {
      adj_filter_leaf_up<T><<<grid_for(Lf.lv[0].n_chunks), kBlock, 0, s>>>(Lf.lv[0], sq, ab, lbar,
                                                                           (T*)Wa.items[1]);
      adj_scan_up<T, false>(Lf, Wa, Lk, s);
    } else {
      cudaMemsetAsync(Wa.flag[Lc], 0, sizeof(int) * Lf.n_items[Lc], s);
    }
    adj_scan_down<T, false>(Lf, Wa, Lc > 1 ? Lk : Lc, s);
    adj_filter_leaf_down<T><<<down_grid, kBlock, 0, s>>>(
        Lf.lv[0], a.leaf, per_step, sq, ab, lbar, (const T*)Wa.carry[1], Wa.flag[1]);
    // SLR adjoint -> next cotangent of the nominal trajectory (and its direct
    // cotangents for the next iteration), theta partials
    {
      const CTParams<T>* Pp = (const CTParams<T>*)a.params;
      switch (a.linearization) {
        case 1:
          adj_slr_kernel<T, 1><<<slr_blocks, kBlock, 0, s>>>(Ls.lv[0], a.leaf, sq, Pp, ab, lam_b,
                                                              g.th_partial);
          break;
        case 2:
          adj_slr_kernel<T, 2><<<slr_blocks, kBlock, 0, s>>>(Ls.lv[0], a.leaf, sq, Pp, ab, lam_b,
                                                              g.th_partial);
          break;
        case 3:
          adj_slr_kernel<T, 3><<<slr_blocks, kBlock, 0, s>>>(Ls.lv[0], a.leaf, sq, Pp, ab, lam_b,
                                                              g.th_partial);
          break;
        default:
          adj_slr_kernel<T, 0><<<slr_blocks, kBlock, 0, s>>>(Ls.lv[0], a.leaf, sq, Pp, ab, lam_b,
                                                              g.th_partial);
      }
    }
    if (it + 1 == g.iters)   // the last iteration's change of lambda (words 0, 1)
      adj_change_partial<T><<<change_blocks, 256, 0, s>>>(X * rows, lam_b, lam_a, words);
    T* t = lam_a;
    lam_a = lam_b;
    lam_b = t;
  }
  if (g.iters > 0) adj_theta_reduce<<<1, 256, 0, s>>>(slr_blocks, g.th_partial, 1.0, g.n_theta, g.grad);
  else cudaMemsetAsync(g.grad, 0, g.n_theta * sizeof(double), s);
  adj_settle_check<<<1, 1, 0, s>>>(words, g.iters > 0 ? 1 : 0, g.tol, g.change, g.ichange, status);
}

}  // namespace sqsm
