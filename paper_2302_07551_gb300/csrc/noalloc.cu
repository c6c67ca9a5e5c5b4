// mc_residual_noalloc: the direct residual ||Q^T pi||_1 without any caller
// workspace and without any device allocation by the library.
//
// Some callers cannot allocate device memory at the point where they want a
// residual: code running while a CUDA graph is being captured (cudaMalloc is
// not a stream operation and may not be called then), real-time or serving
// loops whose device memory is owned by another allocator or budget, and
// plug-ins that are handed only device pointers to someone else's data.  This
// entry point serves them: the caller passes the generator blocks, pi and a
// device output; the only scratch is the file-scope array below, which every
// GPU that loads the library keeps until the process exits.
//
// Scratch contents: one |.|-sum per level (so at most kNoAllocMaxLevels
// levels) and one ticket counter for the last-block-done reduction.  The
// ticket is cleared only by a memset enqueued at the start of every call
// (which also recovers from an earlier launch that did not finish); the
// per-level slots are all overwritten before they are read.  Calls share the array, so
// two calls whose kernels overlap on the GPU (different streams, or different
// host threads) race and must be serialised by the caller.
//
// The first call on a device resolves the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call outside any stream capture.
#include <math.h>
#include <mutex>

#include "mc_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxLevels = 1 << 16;   // 512 KB of per-level sums
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  double level_sum[kNoAllocMaxLevels];
  unsigned int ticket;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

NoAllocScratch* g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mu;

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum_na(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// acc[r] += B(row, j) v_j for a column-major m x m block B (a row-major Q
// block read as its transpose), v_j owned by lane j % 32 in v[j / 32].
template <int R>
__device__ __forceinline__ void gemv_na(double (&acc)[R], const double* __restrict__ B,
                                        const double (&v)[R], int m, int lane) {
#pragma unroll
  for (int kk = 0; kk < R; ++kk) {
    const int jb = kk * 32;
    if (jb >= m) break;
    const int jn = min(32, m - jb);
    for (int q = 0; q < jn; ++q) {
      const int j = jb + q;
      const double vj = __shfl_sync(kFull, v[kk], q);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = lane + 32 * r;
        if (row < m) acc[r] = fma(__ldg(B + (size_t)j * m + row), vj, acc[r]);
      }
    }
  }
}

template <int R>
__device__ __forceinline__ void vec_na(double (&v)[R], const double* __restrict__ p, int m,
                                       int lane) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = lane + 32 * r;
    v[r] = row < m ? p[row] : 0.0;
  }
}

// One warp per level: level_sum[l] = || (Q^T pi)_l ||_1 with
// (Q^T pi)_l = up[l-1]^T pi_{l-1} + loc[l]^T pi_l + dn[l+1]^T pi_{l+1};
// the last block adds level_sum[0..L) into *out in a fixed order (per-thread
// strided partial sums, then a warp and block shuffle tree), which is
// deterministic for the 256-thread block.
template <int R>
__global__ void __launch_bounds__(256) k_residual_noalloc(const double* __restrict__ dn,
                                                          const double* __restrict__ loc,
                                                          const double* __restrict__ up,
                                                          const double* __restrict__ pi,
                                                          int64_t L, int m, double* out,
                                                          NoAllocScratch* sc) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const size_t mm = (size_t)m * m;
  for (int64_t l = gw; l < L; l += nw) {
    double acc[R], v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    if (l > 0) {
      vec_na<R>(v, pi + (l - 1) * m, m, lane);
      gemv_na<R>(acc, up + (size_t)(l - 1) * mm, v, m, lane);
    }
    vec_na<R>(v, pi + l * m, m, lane);
    gemv_na<R>(acc, loc + (size_t)l * mm, v, m, lane);
    if (l < L - 1) {
      vec_na<R>(v, pi + (l + 1) * m, m, lane);
      gemv_na<R>(acc, dn + (size_t)(l + 1) * mm, v, m, lane);
    }
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) s += fabs(acc[r]);
    s = warp_sum_na(s);
    if (lane == 0) sc->level_sum[l] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned tk = atomicAdd(&sc->ticket, 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int64_t l = threadIdx.x; l < L; l += blockDim.x) t += __ldcg(sc->level_sum + l);
  t = warp_sum_na(t);
  if (lane == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    u = warp_sum_na(u);
    if (threadIdx.x == 0) *out = u;
  }
}

// Device address of the scratch array on the current device (resolved once).
int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MC_ERR_CUDA;
    g_scratch_ptr[dev] = (NoAllocScratch*)p;
  }
  *out = g_scratch_ptr[dev];
  return MC_OK;
}

}  // namespace

extern "C" int mc_residual_noalloc(const double* dn, const double* loc, const double* up,
                                   int64_t L, int32_t m, const double* pi, double* resid_dev,
                                   void* cuda_stream) {
  if (!dn || !loc || !up || !pi || !resid_dev) return MC_ERR_ARG;
  if (((uintptr_t)dn | (uintptr_t)loc | (uintptr_t)up | (uintptr_t)pi | (uintptr_t)resid_dev) & 7u)
    return MC_ERR_ARG;
  if (L < 2 || L > kNoAllocMaxLevels || m < 1 || m > mc::kMaxM) return MC_ERR_ARG;
  NoAllocScratch* sc = nullptr;
  const int rc = scratch_for_current_device(&sc);
  if (rc != MC_OK) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) return MC_ERR_CUDA;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MC_ERR_CUDA;
  int64_t warps = 16LL * sms;
  if (warps > L) warps = L;
  const int nb = (int)((warps + 7) / 8);
  switch ((m + 31) / 32) {
    case 1: k_residual_noalloc<1><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    case 2: k_residual_noalloc<2><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    case 3: k_residual_noalloc<3><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    case 4: k_residual_noalloc<4><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    case 5: k_residual_noalloc<5><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    case 6: k_residual_noalloc<6><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    case 7: k_residual_noalloc<7><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
    default: k_residual_noalloc<8><<<nb, 256, 0, s>>>(dn, loc, up, pi, L, m, resid_dev, sc); break;
  }
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_ERR_CUDA;
}
