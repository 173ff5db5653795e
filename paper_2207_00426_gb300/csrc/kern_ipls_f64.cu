// Iterated posterior linearisation smoother (Alg. 3) for the CT model, double.
#include "ipls_impl.cuh"

namespace sqsm {

void ipls_params_f64(const IplsArgs& a, cudaStream_t s) { ipls_params<double>(a, s); }

void ct_linearize_f64(const IplsArgs& a, const LevelSet& Lf, DevSeqs sq, cudaStream_t s) {
  ct_linearize<double>(a, Lf, sq, s);
}

void ipls_phase_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                    const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                    int* status, cudaStream_t s, int phase, unsigned* dmax) {
  ipls_phase<double>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, phase, dmax);
}

void pop_params_f64(const IplsArgs& a, cudaStream_t s) { pop_params<double>(a, s); }

void pop_phase_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                   const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                   int* status, cudaStream_t s, int phase, unsigned* dmax) {
  pop_phase<double>(a, Lf, Wf, Ls, Ws, sq, partial, status, s, phase, dmax);
}

void ipls_enqueue_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s) {
  ipls_enqueue<double>(a, Lf, Wf, Ls, Ws, sq, partial, status, s);
}

}  // namespace sqsm
