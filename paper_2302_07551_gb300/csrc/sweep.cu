// Hot path of the block staircase iteration (Algorithm 2, Eq. (2)).
//
// One sweep = two half-sweeps + one normalisation:
//   half-sweep 1: diagonal-only block rows of the stair matrix
//                 z_l = (-Q_ll)^{-1} (Q_{l,l-1} x_{l-1} + Q_{l,l+1} x_{l+1})
//                 (steps 1 and 2 of Algorithm 2);
//   half-sweep 2: coupled rows, same formula with z in place of x (step 3);
//                 its last block also reduces e^T z;
//   normalise:    x_new = z / e^T z,  step = ||x_new - x_old||_1.
// All Q blocks here are blocks of Q^T, stored column-major (see
// mc_internal.cuh).
//
// Mapping (FP64 pipe bound on GB300: one DFMA per 8 streamed bytes and only
// 2 DFMA/clk/SM): one WARP owns one level.  Lane k owns rows k, k+32, ...
// (R = ceil(m/32) rows), so every block column j is one coalesced 256-byte
// load per 32 rows and every multiply-add lands in the lane's own
// accumulators: no cross-lane reductions and no idle FP64 slots when
// m % 32 == 0.  The level's input vectors sit in a per-warp slice of shared
// memory and v_j, v_{j+1} reach all lanes with one broadcast 16-byte load;
// the intermediate g of the inverse mode goes through the same slice, so the
// second product needs no block barrier.  Each row keeps NA independent
// accumulators (columns interleaved) so that consecutive DFMAs do not wait
// on each other.  Warps stream levels with a static stride; each warp writes
// one partial of e^T z and the last block of half-sweep 2 sums them in a
// fixed order (bitwise deterministic).
#include <math.h>

#include "mc_internal.cuh"
#include "sweep_dev.cuh"

namespace mc {

namespace {

using namespace dev;

// One block Jacobi sweep (stride 1: every level from x) or one half-sweep
// (stride 2) per launch; used for the block Jacobi comparison splitting (the
// stair splittings run fused, fused.cu).
template <int R, bool COUPLED>
__global__ void __launch_bounds__(256, Tune<R>::MINB) k_phase(PhaseArgs a) {
  extern __shared__ double vsh[];
  __shared__ double red[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * R;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int gw = sched_warp(a.P, nw);
  double wsum = 0.0;
  for (int64_t u = gw; u < a.P; u += nw) {
    const int64_t l = a.stride * u + a.parity;
    wsum += level_sweep2<R, COUPLED, false, false>(a.A, a.B, a.C, a.src, a.src, a.dst, l, a.L,
                                                    a.m, a.ms, slice, lane, 1.0, a.far, a.xfar,
                                                    a.xfar);
  }
  wsum = warp_sum(wsum);   // the lanes' partials over all of this warp's levels
  if (lane == 0) {
    a.wpart[gw] = wsum;
    if (a.reduce_s) __threadfence();
  }
  if (!a.reduce_s) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned tk = atomicAdd(&a.hdr->ticket[2], 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // partials of both half-sweeps, [0, n_wpart) starting at half-sweep 1's
  const double* parts = a.wpart - (a.n_wpart - nw);
  double t = 0.0;
  for (int i = threadIdx.x; i < a.n_wpart; i += blockDim.x) t += __ldcg(parts + i);
  t = block_sum(t, red);
  if (threadIdx.x == 0) {
    a.hdr->stats[0] = t;
    a.hdr->ticket[2] = 0u;
  }
}

// Block Gauss-Seidel (Sect. 2 comparison splitting): M = block lower
// triangle, so level l needs the new z_{l-1}; one warp walks l = 0..L-1.
template <int R, bool COUPLED>
__global__ void __launch_bounds__(32) k_bgs(PhaseArgs a) {
  __shared__ double slice[3 * 32 * R];
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int64_t l = 0; l < a.L; ++l) {
    s += level_sweep2<R, COUPLED>(a.A, a.B, a.C, a.dst, a.src_up, a.dst, l, a.L, a.m, a.ms, slice,
                                  lane, 1.0, a.far, a.dst, a.src_up);
    __syncwarp();   // z_l (global, written by all lanes) is read by all lanes next
  }
  if (lane == 0) a.hdr->stats[0] = s;
}

__global__ void __launch_bounds__(kNormThreads) k_normalise(NormArgs a) {
  __shared__ double sh[32];
  __shared__ double rcp[2];
  __shared__ bool last;
  const double s = *a.s;
  const bool ok = (s > 0.0) && isfinite(s);
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) latch(a.hdr, MC_ERR_BREAKDOWN);
  const double so = a.s_old ? *a.s_old : 1.0;
  // the reciprocals once per block: FP64 division is costly at this FP64 rate
  if (threadIdx.x == 0) {
    rcp[0] = 1.0 / s;
    rcp[1] = 1.0 / so;   // exactly 1 for a normalised x_old
  }
  __syncthreads();
  const double inv = rcp[0];
  const double pinv = rcp[1];
  double d = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool vec = ((((uintptr_t)a.x_old) | ((uintptr_t)a.x_new) | ((uintptr_t)a.z)) & 15u) == 0;
  if (!a.x_old) {
    if (((((uintptr_t)a.x_new) | ((uintptr_t)a.z)) & 15u) == 0) {
      // 16-byte loads and stores (the destination may be page-locked host
      // memory, written over the CPU-GPU link)
      const int64_t n2 = a.N / 2;
      const double2* z2 = reinterpret_cast<const double2*>(a.z);
      double2* y2 = reinterpret_cast<double2*>(a.x_new);
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
        const double2 v = z2[i];
        y2[i] = make_double2(v.x * inv, v.y * inv);
      }
      if (blockIdx.x == 0 && threadIdx.x == 0 && (a.N & 1)) a.x_new[a.N - 1] = a.z[a.N - 1] * inv;
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride)
        a.x_new[i] = a.z[i] * inv;
    }
  } else if (vec) {
    // batches of kNormV pairs per thread: all loads of a batch are issued
    // before its stores (x_new may alias x_old entry by entry)
    constexpr int kNormV = 4;
    const int64_t n2 = a.N / 2;
    const double2* z2 = reinterpret_cast<const double2*>(a.z);
    const double2* x2 = reinterpret_cast<const double2*>(a.x_old);
    double2* y2 = reinterpret_cast<double2*>(a.x_new);
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x * kNormV; b < n2; b += stride * kNormV) {
      double2 zz[kNormV], xx[kNormV];
#pragma unroll
      for (int v = 0; v < kNormV; ++v) {
        const int64_t i = b + v * blockDim.x + threadIdx.x;
        if (i < n2) {
          zz[v] = z2[i];
          xx[v] = x2[i];
        }
      }
#pragma unroll
      for (int v = 0; v < kNormV; ++v) {
        const int64_t i = b + v * blockDim.x + threadIdx.x;
        if (i < n2) {
          double2 p;
          p.x = zz[v].x * inv;
          p.y = zz[v].y * inv;
          d += fabs(p.x - xx[v].x * pinv) + fabs(p.y - xx[v].y * pinv);
          y2[i] = p;
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (a.N & 1)) {
      const int64_t i = a.N - 1;
      const double p = a.z[i] * inv;
      d += fabs(p - a.x_old[i] * pinv);
      a.x_new[i] = p;
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride) {
      const double p = a.z[i] * inv;
      d += fabs(p - a.x_old[i] * pinv);
      a.x_new[i] = p;
    }
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
      // e^T z relative to the previous iterate (s itself when that was normalised)
      const double sr = s / so;
      // ||Q^T z||_1 / e^T z = ||Q^T x_new||_1
      const double res = a.r ? *a.r * inv : nan("");
      a.hdr->stats[0] = sr;
      a.hdr->stats[1] = e;
      a.hdr->stats[2] = res;
      if (a.stats_out) {
        a.stats_out[0] = sr;
        a.stats_out[1] = e;
        a.stats_out[2] = res;
      }
      a.hdr->ticket[0] = 0u;
    }
  }
}

// Direct residual ||Q^T x||_1 from the stored FP64 blocks (Eq. (1)).  With
// WITH_Q the level's residual r_l also yields q_l = (-T_dd)^{-1} r_l, stored
// in FP32 for the correction sweeps of iterative refinement.
template <int R, bool WITH_Q, bool PAIRED>
__global__ void __launch_bounds__(256, Tune<R>::MINB) k_residual(ResidArgs a) {
  extern __shared__ double vsh[];
  __shared__ double sh[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * R;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int gw = sched_warp(a.L, nw);
  double wsum = 0.0;
  for (int64_t l = gw; l < a.L; l += nw)
    wsum += level_resid<R, PAIRED>(a.TLO, a.TDD, a.TUP, a.NINV, a.x, WITH_Q ? a.q : nullptr, l,
                                   a.L, a.m, a.ms, slice, lane, a.far);
  if (lane == 0) {
    a.rpart[gw] = wsum;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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

template <int R>
constexpr size_t vec_smem() {
  return (size_t)kWarpsPerBlock * 3 * 32 * R * sizeof(double);
}

// Opt a kernel into more than 48 KB of dynamic shared memory (once).
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes, bool& done) {
  if (done || bytes <= 40 * 1024) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int R, bool C>
cudaError_t phase_r(const PhaseArgs& a, int nb, cudaStream_t s) {
  static bool done = false;
  const cudaError_t e = allow_smem(k_phase<R, C>, vec_smem<R>(), done);
  if (e != cudaSuccess) return e;
  k_phase<R, C><<<nb, 256, vec_smem<R>(), s>>>(a);
  return cudaGetLastError();
}

template <bool C>
cudaError_t phase_dispatch(const PhaseArgs& a, int nb, cudaStream_t s) {
  switch ((a.m + 31) / 32) {
    case 1: return phase_r<1, C>(a, nb, s);
    case 2: return phase_r<2, C>(a, nb, s);
    case 3: return phase_r<3, C>(a, nb, s);
    case 4: return phase_r<4, C>(a, nb, s);
    case 5: return phase_r<5, C>(a, nb, s);
    case 6: return phase_r<6, C>(a, nb, s);
    case 7: return phase_r<7, C>(a, nb, s);
    case 8: return phase_r<8, C>(a, nb, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int R, bool P = false>
cudaError_t resid_r(const ResidArgs& a, int nb, cudaStream_t s) {
  static bool done = false, done_q = false;
  if (a.q) {
    const cudaError_t e = allow_smem(k_residual<R, true, P>, vec_smem<R>(), done_q);
    if (e != cudaSuccess) return e;
    k_residual<R, true, P><<<nb, 256, vec_smem<R>(), s>>>(a);
    return cudaGetLastError();
  }
  const cudaError_t e = allow_smem(k_residual<R, false, P>, vec_smem<R>(), done);
  if (e != cudaSuccess) return e;
  k_residual<R, false, P><<<nb, 256, vec_smem<R>(), s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <int R, bool C>
cudaError_t bgs_r(const PhaseArgs& a, cudaStream_t s) {
  k_bgs<R, C><<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool C>
cudaError_t bgs_dispatch(const PhaseArgs& a, cudaStream_t s) {
  switch ((a.m + 31) / 32) {
    case 1: return bgs_r<1, C>(a, s);
    case 2: return bgs_r<2, C>(a, s);
    case 3: return bgs_r<3, C>(a, s);
    case 4: return bgs_r<4, C>(a, s);
    case 5: return bgs_r<5, C>(a, s);
    case 6: return bgs_r<6, C>(a, s);
    case 7: return bgs_r<7, C>(a, s);
    case 8: return bgs_r<8, C>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

int phase_blocks_per_sm(int m) { return (m + 31) / 32 <= 4 ? 3 : 2; }

cudaError_t launch_phase(const PhaseArgs& a, int coupled, int n_blocks, cudaStream_t s) {
  return coupled ? phase_dispatch<true>(a, n_blocks, s) : phase_dispatch<false>(a, n_blocks, s);
}

cudaError_t launch_bgs(const PhaseArgs& a, int coupled, cudaStream_t s) {
  return coupled ? bgs_dispatch<true>(a, s) : bgs_dispatch<false>(a, s);
}

cudaError_t launch_normalise(const NormArgs& a, int n_blocks, cudaStream_t s) {
  k_normalise<<<n_blocks, kNormThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_residual(const ResidArgs& a, int nb, cudaStream_t s) {
  if (a.paired) {
    switch (a.m / 32) {
      case 2: return resid_r<2, true>(a, nb, s);
      case 4: return resid_r<4, true>(a, nb, s);
      case 6: return resid_r<6, true>(a, nb, s);
      case 8: return resid_r<8, true>(a, nb, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch ((a.m + 31) / 32) {
    case 1: return resid_r<1>(a, nb, s);
    case 2: return resid_r<2>(a, nb, s);
    case 3: return resid_r<3>(a, nb, s);
    case 4: return resid_r<4>(a, nb, s);
    case 5: return resid_r<5>(a, nb, s);
    case 6: return resid_r<6>(a, nb, s);
    case 7: return resid_r<7>(a, nb, s);
    case 8: return resid_r<8>(a, nb, s);
    default: return cudaErrorInvalidValue;
  }
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
