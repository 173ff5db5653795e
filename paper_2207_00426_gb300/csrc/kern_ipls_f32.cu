// Iterated posterior linearisation smoother (Alg. 3) for the CT model, float.
#include "ipls_impl.cuh"

namespace sqsm {

void ipls_params_f32(const IplsArgs& a, cudaStream_t s) { ipls_params<float>(a, s); }

void ct_linearize_f32(const IplsArgs& a, const LevelSet& Lf, DevSeqs sq, cudaStream_t s) {
  ct_linearize<float>(a, Lf, sq, s);
}

void ipls_phase_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                    const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                    int* status, cudaStream_t s, int phase, unsigned* dmax) {
  ipls_phase<float>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, phase, dmax);
}

void pop_params_f32(const IplsArgs& a, cudaStream_t s) { pop_params<float>(a, s); }

void pop_phase_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                   const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                   int* status, cudaStream_t s, int phase, unsigned* dmax) {
  pop_phase<float>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, phase, dmax);
}

void ipls_enqueue_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s) {
  ipls_enqueue<float>(a, Lf, Wf, Ls, Ws, sq, partial, status, s);
}

}  // namespace sqsm
