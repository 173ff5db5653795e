// FP32 FMA-pipe probe: a kernel whose only work is independent chains of
// fused multiply-adds, so that its event-timed rate is the FP32 roof the
// scan and SLR kernels are measured against (they are ALU-bound on <= 10 x 10
// matrices held in registers).  Not part of the method.
#include <cuda_runtime.h>

#include "../../include/sqsm.h"

namespace {

constexpr int kChains = 8;    // independent accumulators per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop trip

__global__ void fp32_fma_probe(int iters, float b, float c, float* __restrict__ out) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (threadIdx.x + j) * 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int sqsm_fp32_fma_probe(int iters, int blocks, int threads, void* out, double* flops,
                                   void* stream) {
  if (iters < 1 || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || !out ||
      !flops)
    return SQSM_ERR_INVALID_ARG;
  *flops = 2.0 * kChains * kUnroll * double(iters) * double(blocks) * double(threads);
  fp32_fma_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, 0.9999999f, 1e-7f,
                                                               (float*)out);
  return cudaGetLastError() == cudaSuccess ? SQSM_OK : SQSM_ERR_CUDA;
}
