// Iterated posterior linearisation smoother (Alg. 3) for the CT model, float.
#include "ct_model.cuh"
#include "dispatch.h"

namespace sqsm {

void ipls_params_f32(const IplsArgs& a, cudaStream_t s) {
  ct_params_kernel<float><<<1, 1, 0, s>>>(a.theta[0], a.theta[1], a.theta[2], a.dt,
                                       a.sensors[0], a.sensors[1], a.sensors[2], a.sensors[3],
                                       (CTParams<float>*)a.params);
}

void ct_linearize_f32(const IplsArgs& a, const LevelSet& Lf, DevSeqs sq, cudaStream_t s) {
  using T = float;
  ct_slr_kernel<T, false><<<grid_for(Lf.lv[0].n_chunks * a.leaf), kBlock, 0, s>>>(
      Lf.lv[0], a.leaf, sq, (const CTParams<T>*)a.params, a.linearization, 0, (const T*)a.ms,
      (const T*)a.Ns, (const T*)a.y, (T*)a.F, (T*)a.c, (T*)a.SQ, (T*)a.H, (T*)a.d, (T*)a.SR);
}

void ipls_enqueue_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s) {
  using T = float;
  constexpr int NX = 5, NY = 2;
  T* ms = (T*)a.ms;
  T* Ns = (T*)a.Ns;
  const int64_t rows = Ls.n_items[0];
  if (a.init_ms) {
    cudaMemcpyAsync(ms, a.init_ms, sizeof(T) * NX * rows, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(Ns, a.init_Ns, sizeof(T) * NX * NX * rows, cudaMemcpyDeviceToDevice, s);
  } else {
    ProfScope ps(a.prof, K_INIT, s);
    broadcast_prior_kernel<T, NX><<<grid_for(Ls.lv[0].n_chunks), kBlock, 0, s>>>(
        Ls.lv[0], (const T*)a.m0, (const T*)a.N0, ms, Ns);
  }
  // the linearised model of every step, packed (a.F holds the PRec records)
  const GammaPacked<T> gv{(T*)a.F};
  // Each iteration smooths the linearised model in deviation coordinates
  // dx_k = x_k - m_k about its own nominal trajectory m (the previous
  // smoothing means, held in ms): the SLR writes c~, d~ of that form, the
  // prior becomes m0 - m_0, and the smoother adds m back when it writes ms.
  for (int it = 0; it < a.M; ++it) {
    {
      ProfScope ps(a.prof, K_SLR, s);
      ct_slr_kernel<T, true><<<grid_for(Lf.lv[0].n_chunks * a.leaf), kBlock, 0, s>>>(
          Lf.lv[0], a.leaf, sq, (const CTParams<T>*)a.params, a.linearization, 1, ms, Ns,
          (const T*)a.y, (T*)a.F, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    {
      ProfScope ps(a.prof, K_INIT, s);
      center_prior_kernel<T, NX><<<(sq.B + 127) / 128, 128, 0, s>>>(sq, (const T*)a.m0, ms,
                                                                     (T*)a.dm0);
    }
    enqueue_filter<T, NX, NY>(Lf, Wf, sq, gv, (const T*)a.y, (const T*)a.dm0, (const T*)a.N0,
                              (T*)a.mf, (T*)a.Nf, partial, status, s, a.prof);
    enqueue_smoother<T, NX, NY>(Ls, Ws, sq, gv, (const T*)a.mf, (const T*)a.Nf, ms, Ns, status,
                                s, a.prof, ms);
  }
  if (a.loglik) enqueue_loglik_reduce(sq, partial, a.loglik, status, s, a.prof);
}

}  // namespace sqsm
