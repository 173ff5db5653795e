// Kernels shared by all paths.
#include "dispatch.h"

namespace sqsm {

// One block per sequence: strided FP64 partial sums, then a fixed-order
// shared-memory tree, so the result does not depend on scheduling.
__global__ void loglik_reduce(DevSeqs sq, const double* __restrict__ partial,
                              double* __restrict__ loglik, int* status) {
  __shared__ double buf[256];
  const int b = blockIdx.x;
  const int64_t lo = sq.leaf_chunk_off[b], hi = sq.leaf_chunk_off[b + 1];
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += partial[i];
  buf[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loglik[b] = buf[0];
    if (!isfinite(buf[0]) && status) atomicOr(status, 8);
  }
}

void enqueue_loglik_reduce(DevSeqs sq, const double* partial, double* loglik, int* status,
                           cudaStream_t s, Prof* P) {
  ProfScope ps(P, K_LOGLIK, s);
  loglik_reduce<<<sq.B, 256, 0, s>>>(sq, partial, loglik, status);
}

namespace {

__global__ void ipls_tol_check(unsigned* dmax, int* iters, int max_iters, float tol,
                               cudaGraphConditionalHandle handle, int use_handle, int* go) {
  const float d = __uint_as_float(*dmax);
  const int it = *iters + 1;
  *iters = it;
  *dmax = 0u;
  const unsigned more = (!(d < tol) && it < max_iters) ? 1u : 0u;
  if (use_handle) cudaGraphSetConditional(handle, more);
  if (go) *go = (int)more;
}

}  // namespace

void enqueue_tol_check(unsigned* dmax, int* iters, int max_iters, float tol,
                       cudaGraphConditionalHandle handle, int use_handle, int* go, cudaStream_t s) {
  ipls_tol_check<<<1, 1, 0, s>>>(dmax, iters, max_iters, tol, handle, use_handle, go);
}

}  // namespace sqsm
