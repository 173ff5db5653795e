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

// N0 = chol(P0) per sequence in FP64 (one thread per sequence; the lower
// triangle of P0 is read, the factor is written with zeros above the
// diagonal).  A pivot that is not positive (P0 not positive definite) or not
// finite makes the whole factor NaN and sets SQSM_ERR_NOT_PD (4).
template <typename T>
__global__ void prior_cholesky(int64_t batch, int nx, const T* __restrict__ P0,
                               T* __restrict__ N0, int* status) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const T* P = P0 + b * nx * nx;
  T* N = N0 + b * nx * nx;
  double L[kMaxPriorNx * kMaxPriorNx];
  bool pd = true;
  for (int j = 0; j < nx; ++j) {
    double d = (double)P[j * nx + j];
    for (int k = 0; k < j; ++k) d -= L[j * kMaxPriorNx + k] * L[j * kMaxPriorNx + k];
    if (!(d > 0.0) || !isfinite(d)) pd = false;
    const double ljj = sqrt(d > 0.0 ? d : 1.0);
    L[j * kMaxPriorNx + j] = ljj;
    for (int i = j + 1; i < nx; ++i) {
      double v = (double)P[i * nx + j];
      for (int k = 0; k < j; ++k) v -= L[i * kMaxPriorNx + k] * L[j * kMaxPriorNx + k];
      L[i * kMaxPriorNx + j] = v / ljj;
    }
  }
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < nx; ++j)
      N[i * nx + j] = !pd ? T(NAN) : j <= i ? (T)L[i * kMaxPriorNx + j] : T(0);
  if (!pd && status) atomicOr(status, 4);
}

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

// One group of a grouped NLL + gradient evaluation: g = {nll, grad[n_theta],
// adj_change, ipls_change} of the group; the first group is copied, later
// ones are added (nll, grad) or maxed (changes; NaN, an unsettled change,
// stays NaN).
__global__ void nll_grad_group_add(int first, int n_theta, const double* __restrict__ g,
                                   double* nll, double* grad, double* adj_change,
                                   double* ipls_change) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  auto mx = [](double a, double b) { return (a != a || b != b) ? NAN : (a > b ? a : b); };
  if (first) {
    nll[0] = g[0];
    for (int i = 0; i < n_theta; ++i) grad[i] = g[1 + i];
    if (adj_change) adj_change[0] = g[5];
    if (ipls_change) ipls_change[0] = g[6];
  } else {
    nll[0] += g[0];
    for (int i = 0; i < n_theta; ++i) grad[i] += g[1 + i];
    if (adj_change) adj_change[0] = mx(adj_change[0], g[5]);
    if (ipls_change) ipls_change[0] = mx(ipls_change[0], g[6]);
  }
}

}  // namespace

void enqueue_nll_grad_group_add(int first, int n_theta, const double* g, double* nll, double* grad,
                                double* adj_change, double* ipls_change, cudaStream_t s) {
  nll_grad_group_add<<<1, 1, 0, s>>>(first, n_theta, g, nll, grad, adj_change, ipls_change);
}

void enqueue_prior_cholesky(int dtype_f64, int64_t batch, int nx, const void* P0, void* N0,
                            int* status, cudaStream_t s) {
  const unsigned blocks = (unsigned)((batch + 127) / 128);
  if (dtype_f64)
    prior_cholesky<double><<<blocks, 128, 0, s>>>(batch, nx, (const double*)P0, (double*)N0,
                                                  status);
  else
    prior_cholesky<float><<<blocks, 128, 0, s>>>(batch, nx, (const float*)P0, (float*)N0, status);
}

void enqueue_tol_check(unsigned* dmax, int* iters, int max_iters, float tol,
                       cudaGraphConditionalHandle handle, int use_handle, int* go, cudaStream_t s) {
  ipls_tol_check<<<1, 1, 0, s>>>(dmax, iters, max_iters, tol, handle, use_handle, go);
}

}  // namespace sqsm
