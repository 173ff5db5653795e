// Iterated posterior linearisation smoother (Alg. 3) for the CT model.
//
// The iterations keep the nominal trajectory and the filter output as packed
// state rows (RowsPacked) and the linearised model as packed records (PRec);
// the caller's arrays are read once (warm start) and written once (result).
#pragma once

#include "ct_model.cuh"
#include "pop_model.cuh"
#include "dispatch.h"

namespace sqsm {

template <typename T>
void pop_params(const IplsArgs& a, cudaStream_t s) {
  pop_params_kernel<T><<<1, 1, 0, s>>>(a.theta[0], a.theta[1], a.theta[2], (PopParams<T>*)a.params);
}

template <typename T>
void ipls_params(const IplsArgs& a, cudaStream_t s) {
  ct_params_kernel<T><<<1, 1, 0, s>>>(a.theta[0], a.theta[1], a.theta[2], a.theta[3], a.dt,
                                      a.sensors[0],
                                      a.sensors[1], a.sensors[2], a.sensors[3],
                                      (CTParams<T>*)a.params);
}

// sqsm_ct_linearize: the printed (absolute) form, caller's layout in and out.
template <typename T>
void ct_linearize(const IplsArgs& a, const LevelSet& Lf, DevSeqs sq, cudaStream_t s) {
  const RowsSplit<T, 5> nom{(T*)a.ms, (T*)a.Ns};
  launch_ct_slr<T, false>(grid_for(Lf.lv[0].n_chunks * a.leaf), s, a.linearization, Lf.lv[0],
                          a.leaf, sq, (const CTParams<T>*)a.params, 0, nom, (const T*)a.y,
                          (T*)a.F, (T*)a.c, (T*)a.SQ, (T*)a.H, (T*)a.d, (T*)a.SR);
}

// One phase of Alg. 3 (IPLS_PRE: initial nominal trajectory; IPLS_ITER: one
// iteration, with dmax set also the largest change of the nominal means;
// IPLS_POST: the result into the caller's arrays and the log-likelihood).
// NX, NY: the model's dimensions; slr(nom, s) launches the model's SLR of
// every step about the nominal rows.
template <typename T, int NX, int NY, typename SLR>
void ipls_phase_model(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s, int phase, unsigned* dmax, SLR slr) {
  const int64_t rows = Ls.n_items[0];
  const RowsPacked<T, NX> nom{(T*)a.nrows}, fr{(T*)a.frows};
  if (phase == IPLS_PRE) {
    ProfScope ps(a.prof, K_INIT, s);
    if (a.init_ms) {
      const RowsSplit<T, NX> init{(T*)a.init_ms, (T*)a.init_Ns};
      rows_copy_kernel<T, NX><<<grid_for(rows), kBlock, 0, s>>>(rows, init, nom);
    } else {
      broadcast_prior_kernel<T, NX><<<grid_for(Ls.lv[0].n_chunks), kBlock, 0, s>>>(
          Ls.lv[0], (const T*)a.m0, (const T*)a.N0, nom);
    }
    return;
  }
  if (phase == IPLS_POST) {
    {
      ProfScope ps(a.prof, K_INIT, s);
      const RowsSplit<T, NX> user{(T*)a.ms, (T*)a.Ns};
      rows_copy_kernel<T, NX><<<grid_for(rows), kBlock, 0, s>>>(rows, nom, user);
    }
    if (a.loglik) enqueue_loglik_reduce(sq, partial, a.loglik, status, s, a.prof);
    return;
  }
  // the linearised model of every step, packed (a.F holds the PRec records)
  const GammaPacked<T> gv{(T*)a.F};
  // Each iteration smooths the linearised model in deviation coordinates
  // dx_k = x_k - m_k about its own nominal trajectory m (the previous
  // smoothing means): the SLR writes c~, d~ of that form, the prior becomes
  // m0 - m_0, and the smoother adds m back when it writes the new nominal.
  // (With a.centered = 0 the printed absolute form is smoothed instead.)
  {
    ProfScope ps(a.prof, K_SLR, s);
    slr(nom, s);
  }
  if (a.centered) {
    ProfScope ps(a.prof, K_INIT, s);
    center_prior_kernel<T, NX><<<(sq.B + 127) / 128, 128, 0, s>>>(sq, (const T*)a.m0, nom,
                                                                   (T*)a.dm0);
  }
  // refinement passes need the nominal rows from before each smoother pass
  const int passes = a.centered ? a.refine : 0;
  const RowsPacked<T, NX> prev{(T*)a.prevrows};
  auto keep_prev = [&]() {
    ProfScope ps(a.prof, K_INIT, s);
    cudaMemcpyAsync(prev.rec, nom.rec, sizeof(T) * XRow<NX>::size * rows,
                    cudaMemcpyDeviceToDevice, s);
  };
  if (passes > 0) keep_prev();
  // with refinement passes to follow, the first filter pass stores the
  // factors of its latency-bound levels' combines (refine_filter.cuh)
  T* ftab = passes > 0 ? (T*)a.ftab : nullptr;
  enqueue_filter<T, NX, NY>(Lf, Wf, sq, gv, (const T*)a.y,
                            (const T*)(a.centered ? a.dm0 : a.m0), (const T*)a.N0, fr, partial,
                            status, s, a.prof, ftab);
  // with refinement passes to follow, the first pass keeps each row's E_k
  T* etab = passes > 0 ? (T*)a.etab : nullptr;
  enqueue_smoother<T, NX, NY>(Ls, Ws, sq, gv, fr, nom, status, s, a.prof, a.centered != 0, dmax,
                              etab);
  // Mixed-precision iterative refinement: the smoother's FP32 error is that
  // of a linear solve, so one more pass on the residual model about its own
  // result (offsets formed beyond FP32 precision) removes most of it; the
  // factors do not change, so the pass's smoother recomputes only the means
  // (refine_scan.cuh; the full scan where the level shape has no mean-only
  // form), and so do its filter scan's latency-bound upper levels
  // (refine_filter.cuh).  The change measure and the log-likelihood stay
  // those of the first pass.
  for (int r = 0; r < passes; ++r) {
    {
      ProfScope ps(a.prof, K_INIT, s);
      refine_residual_kernel<T, NX, NY><<<grid_for(Lf.lv[0].n_chunks * a.leaf), kBlock, 0, s>>>(
          Lf.lv[0], a.leaf, prev, nom, (T*)a.F);
      center_prior_kernel<T, NX><<<(sq.B + 127) / 128, 128, 0, s>>>(sq, (const T*)a.m0, nom,
                                                                     (T*)a.dm0);
    }
    if (r + 1 < passes) keep_prev();
    enqueue_filter<T, NX, NY>(Lf, Wf, sq, gv, (const T*)a.y, (const T*)a.dm0, (const T*)a.N0, fr,
                              a.partial2, status, s, a.prof, ftab, true);
    if (!etab || !enqueue_smoother_means<T, NX, NY>(Ls, Ws, sq, gv, fr, nom, etab, status, s,
                                                    a.prof))
      enqueue_smoother<T, NX, NY>(Ls, Ws, sq, gv, fr, nom, status, s, a.prof, true, nullptr);
  }
}

// The CT bearings model's phase.
template <typename T>
void ipls_phase(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf, const LevelSet& Ls,
                const ScanBuffers& Ws, DevSeqs sq, double* partial, int* status, cudaStream_t s,
                int phase, unsigned* dmax) {
  auto slr = [&](RowsPacked<T, 5> nom, cudaStream_t st) {
    launch_ct_slr<T, true>(grid_for(Lf.lv[0].n_chunks * a.leaf), st, a.linearization, Lf.lv[0],
                           a.leaf, sq, (const CTParams<T>*)a.params, a.centered, nom,
                           (const T*)a.y, (T*)a.F, (T*)nullptr, (T*)nullptr, (T*)nullptr,
                           (T*)nullptr, (T*)nullptr, a.textbook);
  };
  ipls_phase_model<T, 5, 2>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, phase, dmax, slr);
}

// The Ricker population model's phase.
template <typename T>
void pop_phase(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf, const LevelSet& Ls,
               const ScanBuffers& Ws, DevSeqs sq, double* partial, int* status, cudaStream_t s,
               int phase, unsigned* dmax) {
  auto slr = [&](RowsPacked<T, 1> nom, cudaStream_t st) {
    launch_pop_slr<T>(grid_for(Lf.lv[0].n_chunks * a.leaf), st, a.linearization, Lf.lv[0],
                      a.leaf, sq, (const PopParams<T>*)a.params, a.centered, nom, (const T*)a.y,
                      (T*)a.F);
  };
  ipls_phase_model<T, 1, 1>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, phase, dmax, slr);
}

// M iterations of Alg. 3.
template <typename T>
void ipls_enqueue(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                  const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                  int* status, cudaStream_t s) {
  ipls_phase<T>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, IPLS_PRE, nullptr);
  for (int it = 0; it < a.M; ++it)
    ipls_phase<T>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, IPLS_ITER, nullptr);
  ipls_phase<T>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, IPLS_POST, nullptr);
}

}  // namespace sqsm
