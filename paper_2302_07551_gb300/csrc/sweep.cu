// Hot path of the block staircase iteration (Algorithm 2, Eq. (2)).
//
// One sweep = two half-sweeps + one normalisation:
//   half-sweep 1: diagonal-only block rows of the stair matrix
//                 z_l = (-Q_ll)^{-1} (Q_{l,l-1} x_{l-1} + Q_{l,l+1} x_{l+1})
//                 (steps 1 and 2 of Algorithm 2);
//   half-sweep 2: coupled rows, same formula with z in place of x (step 3);
//   normalise:    x_new = z / e^T z,  step = ||x_new - x_old||_1.
// All Q blocks here are blocks of Q^T, stored column-major (see
// mc_internal.cuh).
//
// Mapping (FP64 pipe bound on GB300: one DFMA per 8 streamed bytes and only
// ~2 DFMA/clk/SM): one WARP owns one level.  Lane k owns rows k, k+32, ...
// (R = ceil(m/32) rows), so every block column j is one coalesced 256-byte
// load per 32 rows and every multiply-add lands in the lane's own
// accumulator: no cross-lane reductions, no idle FP64 slots for m % 32 == 0.
// The vector entry v_j is broadcast with a shuffle from the lane that owns
// it; the intermediate g = Q_{l,l-1} v + Q_{l,l+1} v of the inverse mode has
// exactly the same ownership, so the second product needs no shared memory
// and no barrier.  Warps stream levels with a static stride, and each warp
// writes one partial of e^T z (fixed order -> bitwise deterministic sums).
#include <math.h>

#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// acc[r] += sum_j M(row_r, j) * v_j  over the m columns of a column-major
// m x m block M, with v_j held by lane (j % 32) in v[j / 32].
template <int R>
__device__ __forceinline__ void gemv_acc(double (&acc)[R], const double* __restrict__ M,
                                         const double (&v)[R], int m, int lane) {
  // columns per load batch: a power of two dividing 32, about 16 loads in flight
  constexpr int U = R <= 1 ? 16 : R <= 2 ? 8 : R <= 4 ? 4 : 2;
#pragma unroll
  for (int kk = 0; kk < R; ++kk) {
    const int jb = kk * 32;
    if (jb >= m) break;
    const int jn = min(32, m - jb);
    for (int j0 = 0; j0 < jn; j0 += U) {
      double t[U][R];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int j = jb + j0 + q;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int row = lane + 32 * r;
          t[q][r] = (j0 + q < jn && row < m) ? ld_stream(M + (size_t)j * m + row) : 0.0;
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const double vj = __shfl_sync(kFull, v[kk], (j0 + q) & 31);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fma(t[q][r], vj, acc[r]);
      }
    }
  }
}

template <int R>
__device__ __forceinline__ void load_vec(double (&v)[R], const double* __restrict__ p, int m,
                                         int lane) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = lane + 32 * r;
    v[r] = row < m ? p[row] : 0.0;
  }
}

template <int R, bool COUPLED>
__global__ void __launch_bounds__(256) k_phase(PhaseArgs a) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int m = a.m;
  double wsum = 0.0;
  for (int64_t u = gw; u < a.P; u += nw) {
    const int64_t l = 2 * u + a.parity;
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    if (l > 0) {
      double v[R];
      load_vec<R>(v, a.src + (l - 1) * m, m, lane);
      gemv_acc<R>(acc, a.A + (size_t)l * a.ms, v, m, lane);
    }
    if (l < a.L - 1) {
      double v[R];
      load_vec<R>(v, a.src + (l + 1) * m, m, lane);
      gemv_acc<R>(acc, a.B + (size_t)l * a.ms, v, m, lane);
    }
    if (!COUPLED) {
      double g[R];
#pragma unroll
      for (int r = 0; r < R; ++r) { g[r] = acc[r]; acc[r] = 0.0; }
      gemv_acc<R>(acc, a.C + (size_t)l * a.ms, g, m, lane);
    }
    double ls = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = lane + 32 * r;
      if (row < m) {
        a.dst[l * m + row] = acc[r];
        ls += acc[r];
      }
    }
    wsum += warp_sum(ls);
  }
  if (lane == 0) a.wpart[gw] = wsum;
}

// Deterministic block-wide sum (fixed shuffle tree, fixed warp order).
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = lane < nw ? sh[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

__global__ void __launch_bounds__(kNormThreads) k_normalise(NormArgs a) {
  __shared__ double sh[32];
  __shared__ bool last;
  double t = 0.0;
  for (int i = threadIdx.x; i < a.n_wpart; i += blockDim.x) t += a.wpart[i];
  const double s = block_sum(t, sh);
  const bool ok = (s > 0.0) && isfinite(s);
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) latch(a.hdr, MC_ERR_BREAKDOWN);
  const double inv = 1.0 / s;
  double d = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride) {
    const double p = a.z[i] * inv;
    d += fabs(p - a.x_old[i]);
    a.x_new[i] = p;
  }
  d = block_sum(d, sh);
  if (threadIdx.x == 0) {
    a.dpart[blockIdx.x] = d;
    __threadfence();
    const unsigned tk = atomicAdd(&a.hdr->ticket[0], 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double e = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) e += __ldcg(a.dpart + i);
    e = block_sum(e, sh);
    if (threadIdx.x == 0) {
      a.hdr->stats[0] = s;
      a.hdr->stats[1] = e;
      a.hdr->stats[2] = nan("");
      if (a.stats_out) {
        a.stats_out[0] = s;
        a.stats_out[1] = e;
        a.stats_out[2] = nan("");
      }
      a.hdr->ticket[0] = 0u;
    }
  }
}

// Direct residual ||Q^T x||_1 from the stored FP64 blocks (Eq. (1)).
template <int R>
__global__ void __launch_bounds__(256) k_residual(ResidArgs a) {
  __shared__ double sh[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int m = a.m;
  double wsum = 0.0;
  for (int64_t l = gw; l < a.L; l += nw) {
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    double v[R];
    if (l > 0) {
      load_vec<R>(v, a.x + (l - 1) * m, m, lane);
      gemv_acc<R>(acc, a.TLO + (size_t)l * a.ms, v, m, lane);
    }
    load_vec<R>(v, a.x + l * m, m, lane);
    gemv_acc<R>(acc, a.TDD + (size_t)l * a.ms, v, m, lane);
    if (l < a.L - 1) {
      load_vec<R>(v, a.x + (l + 1) * m, m, lane);
      gemv_acc<R>(acc, a.TUP + (size_t)l * a.ms, v, m, lane);
    }
    double ls = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) ls += fabs(acc[r]);
    wsum += warp_sum(ls);
  }
  if (lane == 0) {
    a.rpart[gw] = wsum;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned tk = atomicAdd(&a.hdr->ticket[1], 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double e = 0.0;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) e += __ldcg(a.rpart + i);
    e = block_sum(e, sh);
    if (threadIdx.x == 0) {
      a.hdr->stats[2] = e;
      if (a.out) a.out[0] = e;
      a.hdr->ticket[1] = 0u;
    }
  }
}

__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// x = x0 / sum(x0) with a check that x0 >= 0 and sum > 0 (single block,
// fixed-order sum).
__global__ void __launch_bounds__(1024) k_check_scale(const double* x0, double* x, int64_t n,
                                                      Header* hdr) {
  __shared__ double sh[32];
  double t = 0.0;
  int neg = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = x0[i];
    t += v;
    neg |= !(v >= 0.0);
  }
  neg = __syncthreads_or(neg);
  const double s = block_sum(t, sh);
  if (neg || !(s > 0.0) || !isfinite(s)) {
    if (threadIdx.x == 0) latch(hdr, MC_ERR_ARG);
    return;
  }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = x0[i] / s;
}

template <bool C>
cudaError_t phase_dispatch(const PhaseArgs& a, int nb, cudaStream_t s) {
  const int R = (a.m + 31) / 32;
  switch (R) {
    case 1: k_phase<1, C><<<nb, 256, 0, s>>>(a); break;
    case 2: k_phase<2, C><<<nb, 256, 0, s>>>(a); break;
    case 3: k_phase<3, C><<<nb, 256, 0, s>>>(a); break;
    case 4: k_phase<4, C><<<nb, 256, 0, s>>>(a); break;
    case 5: k_phase<5, C><<<nb, 256, 0, s>>>(a); break;
    case 6: k_phase<6, C><<<nb, 256, 0, s>>>(a); break;
    case 7: k_phase<7, C><<<nb, 256, 0, s>>>(a); break;
    case 8: k_phase<8, C><<<nb, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_phase(const PhaseArgs& a, int coupled, int n_blocks, cudaStream_t s) {
  return coupled ? phase_dispatch<true>(a, n_blocks, s) : phase_dispatch<false>(a, n_blocks, s);
}

cudaError_t launch_normalise(const NormArgs& a, int n_blocks, cudaStream_t s) {
  k_normalise<<<n_blocks, kNormThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_residual(const ResidArgs& a, int nb, cudaStream_t s) {
  const int R = (a.m + 31) / 32;
  switch (R) {
    case 1: k_residual<1><<<nb, 256, 0, s>>>(a); break;
    case 2: k_residual<2><<<nb, 256, 0, s>>>(a); break;
    case 3: k_residual<3><<<nb, 256, 0, s>>>(a); break;
    case 4: k_residual<4><<<nb, 256, 0, s>>>(a); break;
    case 5: k_residual<5><<<nb, 256, 0, s>>>(a); break;
    case 6: k_residual<6><<<nb, 256, 0, s>>>(a); break;
    case 7: k_residual<7><<<nb, 256, 0, s>>>(a); break;
    case 8: k_residual<8><<<nb, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fill(double* x, int64_t n, double v, cudaStream_t s) {
  const int nb = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  k_fill<<<nb > 0 ? nb : 1, 256, 0, s>>>(x, n, v);
  return cudaGetLastError();
}

cudaError_t launch_check_scale(const double* x0, double* x, int64_t n, Header* hdr, double*,
                               cudaStream_t s) {
  k_check_scale<<<1, 1024, 0, s>>>(x0, x, n, hdr);
  return cudaGetLastError();
}

}  // namespace mc
