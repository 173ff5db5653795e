// Standard (covariance) form of Alg. 3 for the CT model, float.
#include "std_form.cuh"

namespace sqsm {

void std_ipls_enqueue_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                          const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                          int* status, cudaStream_t s) {
  std_ipls_enqueue<float>(a, Lf, Wf, Ls, Ws, sq, partial, status, s);
}

}  // namespace sqsm
