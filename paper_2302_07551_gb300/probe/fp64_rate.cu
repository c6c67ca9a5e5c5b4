// FP64 multiply-add rate of the GPU: the measured denominator of the FP64
// roofline of the sweep kernels (no counterpart in the paper; not part of
// libmc -- this is a separate library, libmcprobe.so, used only by the
// benchmark's --measure-fp64-peak mode).
//
// Every thread runs C independent chains x_c <- fma(x_c, y_c, z) for `iters`
// steps, U steps per loop trip, so the FP64 pipe always has independent work
// and the loop bookkeeping is amortised; the block's sum is stored so that no
// chain is dead code.  The multipliers and the addend are in registers
// (loaded from memory) or are kernel parameters.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kMaxProbeBlocks = 16384;
constexpr int kMaxChains = 32;

__device__ double g_probe_out[kMaxProbeBlocks];
__device__ double g_probe_coef[kMaxChains + 1];

template <int C, int U, bool REG>
__global__ void k_dfma_rate(int64_t trips, double a, double b) {
  double x[C], y[C];
  double z = b;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    x[c] = 1e-3 * (threadIdx.x + c);
    y[c] = REG ? g_probe_coef[c] : a;
  }
  if (REG) z = g_probe_coef[kMaxChains];
  for (int64_t i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < C; ++c) x[c] = fma(x[c], y[c], z);
  }
  double t = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) t += x[c];
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

// Largest block the kernel's register use allows.
template <int C, int U>
int max_threads(bool reg) {
  cudaFuncAttributes fa{};
  const cudaError_t e = reg ? cudaFuncGetAttributes(&fa, k_dfma_rate<C, U, true>)
                            : cudaFuncGetAttributes(&fa, k_dfma_rate<C, U, false>);
  return e == cudaSuccess ? fa.maxThreadsPerBlock : 0;
}

template <int C, int U>
cudaError_t launch(bool reg, int blocks, int threads, int64_t trips, cudaStream_t s) {
  if (reg)
    k_dfma_rate<C, U, true><<<blocks, threads, 0, s>>>(trips, 1.0 - 1e-12, 1e-13);
  else
    k_dfma_rate<C, U, false><<<blocks, threads, 0, s>>>(trips, 1.0 - 1e-12, 1e-13);
  return cudaGetLastError();
}

}  // namespace

// Run `blocks` blocks of `threads` threads (a multiple of 32, at most 1024;
// 1 <= blocks <= 16384), each thread `chains` (8, 16 or 32) independent fma
// chains of `iters` steps (a multiple of 4, 4 <= iters <= 2^32), multipliers
// and addend in registers loaded from memory (reg != 0) or kernel parameters
// (reg == 0).  *tflops receives 2 * chains * iters * threads * blocks / (event
// time) in TFLOP/s.  Syncs cuda_stream.  Returns 0, 1 (bad argument, or a
// block larger than the kernel's register use allows) or 3 (a CUDA call
// failed).
extern "C" int mcprobe_fp64_rate(void* cuda_stream, int blocks, int threads, int64_t iters,
                                 int chains, int reg, double* tflops) {
  if (!tflops || blocks < 1 || blocks > kMaxProbeBlocks || threads < 32 || threads > 1024 ||
      threads % 32 != 0 || iters < 4 || iters > (int64_t)1 << 32 || iters % 4 != 0 ||
      (chains != 8 && chains != 16 && chains != 32))
    return 1;
  const int tmax = chains == 8    ? max_threads<8, 4>(reg != 0)
                   : chains == 16 ? max_threads<16, 4>(reg != 0)
                                  : max_threads<32, 4>(reg != 0);
  if (threads > tmax) return 1;   // more registers than the block can hold
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = 3;
  if (rc == 0 && reg) {
    double coef[kMaxChains + 1];
    for (int c = 0; c < kMaxChains; ++c) coef[c] = 1.0 - 1e-12 * (c + 1);
    coef[kMaxChains] = 1e-13;
    if (cudaMemcpyToSymbolAsync(g_probe_coef, coef, sizeof(coef), 0, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      rc = 3;
  }
  if (rc == 0 && cudaEventRecord(e0, s) != cudaSuccess) rc = 3;
  if (rc == 0) {
    const int64_t trips = iters / 4;
    cudaError_t e = cudaSuccess;
    switch (chains) {
      case 8: e = launch<8, 4>(reg != 0, blocks, threads, trips, s); break;
      case 16: e = launch<16, 4>(reg != 0, blocks, threads, trips, s); break;
      default: e = launch<32, 4>(reg != 0, blocks, threads, trips, s); break;
    }
    if (e != cudaSuccess) rc = 3;
  }
  if (rc == 0 && cudaEventRecord(e1, s) != cudaSuccess) rc = 3;
  float ms = 0.0f;
  if (rc == 0 && (cudaEventSynchronize(e1) != cudaSuccess ||
                  cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f))
    rc = 3;
  if (rc == 0)
    *tflops = 2.0 * chains * (double)iters * threads * (double)blocks / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
