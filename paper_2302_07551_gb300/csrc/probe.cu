// FP64 multiply-add rate of the GPU (diagnostic for the roofline denominator;
// no counterpart in the paper).  Every thread runs kChains independent chains
// x <- fma(x, a, b) for `iters` steps, so the FP64 pipe always has
// independent work; the block's sum is stored so that nothing is dead code.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mc.h"

namespace {

constexpr int kChains = 8;
constexpr int kMaxProbeBlocks = 8192;

__device__ double g_probe_out[kMaxProbeBlocks];
__device__ double g_probe_coef[kChains + 1];

// REG: the multipliers and the addend are loaded from memory into registers
// (one multiplier per chain); otherwise they are kernel parameters.
template <bool REG>
__global__ void k_dfma_rate(int64_t iters, double a, double b) {
  double x[kChains], y[kChains];
  double z = b;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = 1e-3 * (threadIdx.x + c);
    y[c] = REG ? g_probe_coef[c] : a;
  }
  if (REG) z = g_probe_coef[kChains];
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], y[c], z);
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) t += x[c];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    g_probe_out[blockIdx.x] = s;
  }
}

}  // namespace

extern "C" int mc_fp64_rate(void* cuda_stream, int blocks, int threads, int64_t iters,
                            int reg, double* tflops) {
  if (!tflops || blocks < 1 || blocks > kMaxProbeBlocks || threads < 32 || threads > 1024 ||
      threads % 32 != 0 || iters < 1 || iters > (int64_t)1 << 32)
    return MC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MC_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MC_ERR_CUDA;
  if (rc == MC_OK && reg) {
    double coef[kChains + 1];
    for (int c = 0; c < kChains; ++c) coef[c] = 1.0 - 1e-12 * (c + 1);
    coef[kChains] = 1e-13;
    if (cudaMemcpyToSymbolAsync(g_probe_coef, coef, sizeof(coef), 0, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      rc = MC_ERR_CUDA;
  }
  if (rc == MC_OK && cudaEventRecord(e0, s) != cudaSuccess) rc = MC_ERR_CUDA;
  if (rc == MC_OK) {
    if (reg)
      k_dfma_rate<true><<<blocks, threads, 0, s>>>(iters, 1.0 - 1e-12, 1e-13);
    else
      k_dfma_rate<false><<<blocks, threads, 0, s>>>(iters, 1.0 - 1e-12, 1e-13);
    if (cudaGetLastError() != cudaSuccess) rc = MC_ERR_CUDA;
  }
  if (rc == MC_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = MC_ERR_CUDA;
  float ms = 0.0f;
  if (rc == MC_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f))
    rc = MC_ERR_CUDA;
  if (rc == MC_OK)
    *tflops = 2.0 * kChains * (double)iters * threads * (double)blocks / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
