// Device helpers shared by the single-chain and the batched FP64 kernels.
//
// Warp-per-level products: lane k owns rows k, k+32, ... (R = ceil(m/32)
// rows) of a column-major m x m block; input vectors sit in a per-warp
// shared-memory slice (zero beyond m) and are read as broadcast pairs.
#pragma once
#include <math.h>

#include "mc_internal.cuh"

namespace mc {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp index for the persistent loop  for (u = w; u < P; u += nw).  With
// several rounds it is block-major: a block's warps take consecutive units, so
// the grid streams one window of neighbouring levels.  When all P units fit in
// one partial round it is block-minor instead, so that the busy warps spread
// evenly over the blocks (hence over the SMs) rather than filling the first
// blocks.  Both orders are permutations of [0, nw).
__device__ __forceinline__ int sched_warp(int64_t P, int nw) {
  if (P >= nw) return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  return (int)((threadIdx.x >> 5) * gridDim.x + blockIdx.x);
}

template <int R>
struct Tune {
  static constexpr int U = R <= 1 ? 16 : R <= 2 ? 8 : R <= 4 ? 4 : 2;  // columns per batch
  static constexpr int NA = 1;                                         // accumulators per row
  static constexpr int MINB = R <= 4 ? 3 : 2;                          // blocks per SM
};

// acc[r][c] += M(row_r, j) * v[j] for the m columns j of a column-major block
// M; column j feeds accumulator j % NA.  v: per-warp shared slice, zero
// beyond m (so the pair load at an odd m reads a zero).  UM multiplies the
// columns per batch (more loads in flight for kernels with few warps).
template <int R, int UM = 1>
__device__ __forceinline__ void gemv_acc(double (&acc)[R][Tune<R>::NA],
                                         const double* __restrict__ M, const double* v, int m,
                                         int lane) {
  constexpr int U = Tune<R>::U * UM, NA = Tune<R>::NA;
  for (int j0 = 0; j0 < m; j0 += U) {
    double t[U][R];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int j = j0 + q;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = lane + 32 * r;
        t[q][r] = (j < m && row < m) ? ld_stream(M + (size_t)j * m + row) : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < U; q += 2) {
      const double2 vv = *reinterpret_cast<const double2*>(v + j0 + q);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        acc[r][q % NA] = fma(t[q][r], vv.x, acc[r][q % NA]);
        acc[r][(q + 1) % NA] = fma(t[q + 1][r], vv.y, acc[r][(q + 1) % NA]);
      }
    }
  }
}

// As gemv_acc, restricted to columns [j0, j1) and row groups r in [R0, R1)
// (rows lane + 32 r): the structurally nonzero part of a block.
template <int R, int R0, int R1>
__device__ __forceinline__ void gemv_acc_part(double (&acc)[R][Tune<R>::NA],
                                              const double* __restrict__ M, const double* v,
                                              int j0b, int j1, int m, int lane) {
  // batch size follows the rows actually read (about 16 loads in flight)
  constexpr int U = Tune<R1 - R0>::U, NA = Tune<R>::NA;
  for (int j0 = j0b; j0 < j1; j0 += U) {
    double t[U][R1 - R0];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int j = j0 + q;
#pragma unroll
      for (int r = R0; r < R1; ++r) {
        const int row = lane + 32 * r;
        t[q][r - R0] = (j < j1 && row < m) ? ld_stream(M + (size_t)j * m + row) : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < U; q += 2) {
      const double2 vv = *reinterpret_cast<const double2*>(v + j0 + q);
#pragma unroll
      for (int r = R0; r < R1; ++r) {
        acc[r][q % NA] = fma(t[q][r - R0], vv.x, acc[r][q % NA]);
        acc[r][(q + 1) % NA] = fma(t[q + 1][r - R0], vv.y, acc[r][(q + 1) % NA]);
      }
    }
  }
}

// Products with the off-diagonal Q^T blocks of a paired block-pentadiagonal
// chain (m = 32 R, R even): T_lo is zero in rows m/2.. of columns ..m/2,
// T_up in rows ..m/2 of columns m/2..; only the nonzero quadrants are read.
template <int R>
__device__ __forceinline__ void gemv_lo_paired(double (&acc)[R][Tune<R>::NA],
                                               const double* __restrict__ M, const double* v,
                                               int m, int lane) {
  gemv_acc_part<R, 0, R / 2>(acc, M, v, 0, m / 2, m, lane);
  gemv_acc_part<R, 0, R>(acc, M, v, m / 2, m, m, lane);
}
template <int R>
__device__ __forceinline__ void gemv_up_paired(double (&acc)[R][Tune<R>::NA],
                                               const double* __restrict__ M, const double* v,
                                               int m, int lane) {
  gemv_acc_part<R, 0, R>(acc, M, v, 0, m / 2, m, lane);
  gemv_acc_part<R, R / 2, R>(acc, M, v, m / 2, m, m, lane);
}

// v = p * scale (scale = 1 / e^T z of the previous sweep when the previous
// sweep was not normalised in memory; 1 otherwise: fl(z * (1/s)) is exactly
// the value the normalisation would have stored).
// CG: p was written by other SMs during this kernel, so it is read from L2
// (ld.global.cg), never from a possibly stale L1 line.
template <int R, bool CG = false>
__device__ __forceinline__ void stage_vec(double* v, const double* __restrict__ p, int m,
                                          int lane, double scale = 1.0) {
  if (scale != 1.0) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = lane + 32 * r;
      v[row] = row < m ? (CG ? __ldcg(p + row) : p[row]) * scale : 0.0;
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = lane + 32 * r;
      v[row] = row < m ? (CG ? __ldcg(p + row) : p[row]) : 0.0;
    }
  }
}

template <int R>
__device__ __forceinline__ void zero_acc(double (&acc)[R][Tune<R>::NA]) {
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < Tune<R>::NA; ++c) acc[r][c] = 0.0;
}

template <int R>
__device__ __forceinline__ double fold(const double (&a)[Tune<R>::NA]) {
  if constexpr (Tune<R>::NA == 1) {
    return a[0];
  } else if constexpr (Tune<R>::NA == 4) {
    return (a[0] + a[1]) + (a[2] + a[3]);
  } else {
    return a[0] + a[1];
  }
}

// Deterministic block-wide sum (fixed shuffle tree, fixed warp order).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = lane < nw ? sh[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

// One level of a half-sweep (Algorithm 2): z_l = (-T_dd)^{-1}(T_lo v_{l-1} +
// T_up v_{l+1}) (inverse mode: A = T_lo, B = T_up, C = (-T_dd)^{-1}) or
// z_l = W_lo v_{l-1} + W_up v_{l+1} (coupled: A = W_lo, B = W_up), written to
// dst; returns sum_i z_l[i] on every lane.  slice: 3 * 32 R doubles of the
// warp's shared memory.
// Off-staircase terms of a block-banded Q^T: acc += sum_j T_{l,l+d_j} v_{l+d_j}
// with v = xlo for d_j < 0 and xup for d_j > 0 (staged through slice).
template <int R, bool CG = false>
__device__ __forceinline__ void far_terms(double (&acc)[R][Tune<R>::NA], const FarDesc* far,
                                          const double* xlo, const double* xup, int64_t l,
                                          int64_t L, int m, int ms, double* slice, int lane) {
  const int n = far->n;
  for (int j = 0; j < n; ++j) {
    const int64_t k = l + far->off[j];
    if (k < 0 || k >= L) continue;
    __syncwarp();
    stage_vec<R, CG>(slice, (far->off[j] < 0 ? xlo : xup) + k * m, m, lane);
    __syncwarp();
    gemv_acc<R>(acc, far->plane[j] + (size_t)l * ms, slice, m, lane);
  }
  __syncwarp();
}

// Returns sum_i z_l[i]: on every lane (WARP_TOTAL) or the lane's own rows
// only (callers that only need a total over many levels reduce once at the end);
// want_sum = false skips the sum (0 is returned): the FP64 adds it costs are a
// share of an FP64-bound kernel, and a fused launch only needs the sums of its
// last two sweeps.
// CG: neighbour vectors written by other SMs during this kernel (L2 reads).
template <int R, bool COUPLED, bool PAIRED = false, bool WARP_TOTAL = true, bool CG = false,
          int UM = 1>
__device__ __forceinline__ double level_sweep2(const double* A, const double* B, const double* C,
                                               const double* src, const double* src_up,
                                               double* dst, int64_t l, int64_t L, int m, int ms,
                                               double* slice, int lane, double scale = 1.0,
                                               const FarDesc* far = nullptr,
                                               const double* xfar_lo = nullptr,
                                               const double* xfar_up = nullptr,
                                               bool want_sum = true) {
  constexpr int NA = Tune<R>::NA, W = 32 * R;
  double* v_lo = slice;
  double* v_up = slice + W;
  double* v_g = slice + 2 * W;
  const bool has_lo = l > 0, has_up = l < L - 1;
  if (has_lo) stage_vec<R, CG>(v_lo, src + (l - 1) * m, m, lane, scale);
  if (has_up) stage_vec<R, CG>(v_up, src_up + (l + 1) * m, m, lane, scale);
  __syncwarp();
  double acc[R][NA];
  zero_acc<R>(acc);
  if constexpr (PAIRED) {
    if (has_lo) gemv_lo_paired<R>(acc, A + (size_t)l * ms, v_lo, m, lane);
    if (has_up) gemv_up_paired<R>(acc, B + (size_t)l * ms, v_up, m, lane);
  } else {
    if (has_lo) gemv_acc<R, UM>(acc, A + (size_t)l * ms, v_lo, m, lane);
    if (has_up) gemv_acc<R, UM>(acc, B + (size_t)l * ms, v_up, m, lane);
  }
  if (far) far_terms<R, CG>(acc, far, xfar_lo, xfar_up, l, L, m, ms, v_lo, lane);
  if (!COUPLED) {
#pragma unroll
    for (int r = 0; r < R; ++r) v_g[lane + 32 * r] = fold<R>(acc[r]);
    __syncwarp();
    zero_acc<R>(acc);
    gemv_acc<R, UM>(acc, C + (size_t)l * ms, v_g, m, lane);
  }
  double ls = 0.0;
  if (want_sum) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = lane + 32 * r;
      const double zr = fold<R>(acc[r]);
      if (row < m) {
        dst[l * m + row] = zr;
        ls += zr;
      }
    }
    if (WARP_TOTAL) ls = warp_sum(ls);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = lane + 32 * r;
      if (row < m) dst[l * m + row] = fold<R>(acc[r]);
    }
  }
  __syncwarp();   // the slice is rewritten for the next level
  return ls;
}

// Residual of a sweep's result at a diagonal-only stair row l, from the
// splitting instead of a product with all three blocks: the sweep solved
// M z = N x, so Q^T z = M z - N z = N (x - z), which is zero on the coupled
// rows (N has no entries there) and equals T_lo d_{l-1} + T_up d_{l+1},
// d = z - x, on the diagonal-only rows.  z, x: the sweep's result and input
// (written by other SMs during the launch: read from L2).  d is small near
// convergence, so its product rounds far below the direct residual's
// cancellation.  Returns ||(Q^T z)_l||_1 on every lane.
template <int R, bool PAIRED>
__device__ __forceinline__ double level_resid_split(const double* TLO, const double* TUP,
                                                    const double* z, const double* x, int64_t l,
                                                    int64_t L, int m, int ms, double* slice,
                                                    int lane) {
  constexpr int NA = Tune<R>::NA, W = 32 * R;
  double* v_lo = slice;
  double* v_up = slice + W;
  const bool has_lo = l > 0, has_up = l < L - 1;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = lane + 32 * r;
    if (has_lo)
      v_lo[row] = row < m ? __ldcg(z + (l - 1) * m + row) - __ldcg(x + (l - 1) * m + row) : 0.0;
    if (has_up)
      v_up[row] = row < m ? __ldcg(z + (l + 1) * m + row) - __ldcg(x + (l + 1) * m + row) : 0.0;
  }
  __syncwarp();
  double acc[R][NA];
  zero_acc<R>(acc);
  if constexpr (PAIRED) {
    if (has_lo) gemv_lo_paired<R>(acc, TLO + (size_t)l * ms, v_lo, m, lane);
    if (has_up) gemv_up_paired<R>(acc, TUP + (size_t)l * ms, v_up, m, lane);
  } else {
    if (has_lo) gemv_acc<R>(acc, TLO + (size_t)l * ms, v_lo, m, lane);
    if (has_up) gemv_acc<R>(acc, TUP + (size_t)l * ms, v_up, m, lane);
  }
  double ls = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) ls += fabs(fold<R>(acc[r]));
  const double total = warp_sum(ls);
  __syncwarp();   // the slice is rewritten for the next level
  return total;
}

// One level of the direct residual r_l = (Q^T x)_l = T_lo x_{l-1} + T_dd x_l +
// T_up x_{l+1} (Eq. (1)); returns ||r_l||_1 on every lane.  With q != NULL
// also stores q_l = (-T_dd)^{-1} r_l in FP32.
template <int R, bool PAIRED = false>
__device__ __forceinline__ double level_resid(const double* TLO, const double* TDD,
                                              const double* TUP, const double* NINV,
                                              const double* x, float* q, int64_t l, int64_t L,
                                              int m, int ms, double* slice, int lane,
                                              const FarDesc* far = nullptr) {
  constexpr int NA = Tune<R>::NA, W = 32 * R;
  double* v_lo = slice;
  double* v_dd = slice + W;
  double* v_up = slice + 2 * W;
  if (l > 0) stage_vec<R>(v_lo, x + (l - 1) * m, m, lane);
  stage_vec<R>(v_dd, x + l * m, m, lane);
  if (l < L - 1) stage_vec<R>(v_up, x + (l + 1) * m, m, lane);
  __syncwarp();
  double acc[R][NA];
  zero_acc<R>(acc);
  if (l > 0) {
    if constexpr (PAIRED)
      gemv_lo_paired<R>(acc, TLO + (size_t)l * ms, v_lo, m, lane);
    else
      gemv_acc<R>(acc, TLO + (size_t)l * ms, v_lo, m, lane);
  }
  gemv_acc<R>(acc, TDD + (size_t)l * ms, v_dd, m, lane);
  if (l < L - 1) {
    if constexpr (PAIRED)
      gemv_up_paired<R>(acc, TUP + (size_t)l * ms, v_up, m, lane);
    else
      gemv_acc<R>(acc, TUP + (size_t)l * ms, v_up, m, lane);
  }
  if (far) far_terms<R>(acc, far, x, x, l, L, m, ms, v_lo, lane);
  double ls = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) ls += fabs(fold<R>(acc[r]));
  const double total = warp_sum(ls);
  if (q) {
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) v_lo[lane + 32 * r] = fold<R>(acc[r]);
    __syncwarp();
    zero_acc<R>(acc);
    gemv_acc<R>(acc, NINV + (size_t)l * ms, v_lo, m, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = lane + 32 * r;
      if (row < m) q[l * m + row] = (float)fold<R>(acc[r]);
    }
  }
  __syncwarp();
  return total;
}

}  // namespace dev
}  // namespace mc
