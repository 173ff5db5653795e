// NLL + gradient through the IPLS fixed point (Sec. 5.2), double.
#include "adj_impl.cuh"

namespace sqsm {

void adj_enqueue_f64(const IplsArgs& a, const AdjArgs& g, const LevelSet& Lf,
                    const ScanBuffers& Wf, const LevelSet& Ls, const ScanBuffers& Ws,
                    const ScanBuffers& Wa, DevSeqs sq, double* partial, int* status,
                    cudaStream_t s) {
  adj_enqueue<double>(a, g, Lf, Wf, Ls, Ws, Wa, sq, partial, status, s);
}

}  // namespace sqsm
