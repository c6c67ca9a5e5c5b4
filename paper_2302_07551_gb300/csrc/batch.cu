// Batched kernels of the solve server (see batch.cuh): the per-level bodies
// of the single-chain kernels (level_sweep, level_resid, level_sweep_lp)
// applied to every level of every active request in one persistent launch.
#include <cuda_bf16.h>
#include <math.h>

#include "batch.cuh"
#include "lowprec_dev.cuh"
#include "sweep_dev.cuh"

namespace mc {

namespace {

using namespace dev;

// Largest r in [lo, hi) with off[r] <= i (off is non-decreasing).
__device__ __forceinline__ int find_req(const int64_t* off, int lo, int hi, int64_t i) {
  hi -= 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Item range and request range of a bucket.
__device__ __forceinline__ void bucket(const BTable* t, const int64_t* off, bool large, int& r0,
                                       int& r1, int64_t& i0, int64_t& i1) {
  r0 = large ? t->n_small : 0;
  r1 = large ? t->n : t->n_small;
  i0 = off[r0];
  i1 = off[r1];
}

template <bool COUPLED, bool LARGE>
__global__ void __launch_bounds__(256) k_b_phase(const BTable* __restrict__ t, int half) {
  extern __shared__ double vsh[];
  constexpr int RMAX = LARGE ? 8 : 4;
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * RMAX;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t* off = half == 0 ? t->off_h1 : t->off_h2;
  int r0, r1;
  int64_t i0, i1;
  bucket(t, off, LARGE, r0, r1, i0, i1);
  for (int64_t i = i0 + gw; i < i1; i += nw) {
    const int r = find_req(off, r0, r1, i);
    const BReq* q = &t->r[r];
    const int par = half == 0 ? q->p1 : 1 - q->p1;
    const int64_t l = 2 * (i - off[r]) + par;
    const double* src = half == 0 ? q->x : q->z;
    double ls;
    if (LARGE) {
      ls = level_sweep<8, COUPLED>(q->A, q->B, q->C, src, q->z, l, q->L, q->m, q->ms, slice, lane);
    } else {
      switch (q->R) {
        case 1: ls = level_sweep<1, COUPLED>(q->A, q->B, q->C, src, q->z, l, q->L, q->m, q->ms, slice, lane); break;
        case 2: ls = level_sweep<2, COUPLED>(q->A, q->B, q->C, src, q->z, l, q->L, q->m, q->ms, slice, lane); break;
        case 3: ls = level_sweep<3, COUPLED>(q->A, q->B, q->C, src, q->z, l, q->L, q->m, q->ms, slice, lane); break;
        default: ls = level_sweep<4, COUPLED>(q->A, q->B, q->C, src, q->z, l, q->L, q->m, q->ms, slice, lane); break;
      }
    }
    if (lane == 0) q->lsum[l] = ls;
  }
}

template <bool LARGE>
__global__ void __launch_bounds__(256) k_b_resid(const BTable* __restrict__ t, int with_q) {
  extern __shared__ double vsh[];
  constexpr int RMAX = LARGE ? 8 : 4;
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * RMAX;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int r0, r1;
  int64_t i0, i1;
  bucket(t, t->off_lv, LARGE, r0, r1, i0, i1);
  for (int64_t i = i0 + gw; i < i1; i += nw) {
    const int r = find_req(t->off_lv, r0, r1, i);
    const BReq* q = &t->r[r];
    const int64_t l = i - t->off_lv[r];
    float* qv = with_q ? q->q : nullptr;
    double ls;
    if (LARGE) {
      ls = level_resid<8>(q->TLO, q->TDD, q->TUP, q->NINV, q->x, qv, l, q->L, q->m, q->ms, slice, lane);
    } else {
      switch (q->R) {
        case 1: ls = level_resid<1>(q->TLO, q->TDD, q->TUP, q->NINV, q->x, qv, l, q->L, q->m, q->ms, slice, lane); break;
        case 2: ls = level_resid<2>(q->TLO, q->TDD, q->TUP, q->NINV, q->x, qv, l, q->L, q->m, q->ms, slice, lane); break;
        case 3: ls = level_resid<3>(q->TLO, q->TDD, q->TUP, q->NINV, q->x, qv, l, q->L, q->m, q->ms, slice, lane); break;
        default: ls = level_resid<4>(q->TLO, q->TDD, q->TUP, q->NINV, q->x, qv, l, q->L, q->m, q->ms, slice, lane); break;
      }
    }
    if (lane == 0) q->lsum[l] = ls;
  }
}

// which: 0 -> s = e^T z (with the breakdown check), 1 -> step, 2 -> residual.
// One block per request (grid-stride), fixed order: thread k adds levels
// k, k + blockDim, ..., then a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_b_reqsum(const BTable* __restrict__ t, BOut* out,
                                                  int which) {
  __shared__ double sh[32];
  for (int r = blockIdx.x; r < t->n; r += gridDim.x) {
    const BReq* q = &t->r[r];
    double v = 0.0;
    for (int64_t l = threadIdx.x; l < q->L; l += blockDim.x) v += q->lsum[l];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
      if (which == 0) {
        out[r].s = v;
        if (!(v > 0.0) || !isfinite(v)) out[r].status = MC_ERR_BREAKDOWN;
      } else if (which == 1) {
        out[r].step = v;
      } else {
        out[r].resid = v;
      }
    }
    __syncthreads();
  }
}

// x_l = src_l / s per level (src = z, or xb after a refinement update), with
// the level's step error |x_new - x_old|_1 into lsum.
__global__ void __launch_bounds__(256) k_b_norm(const BTable* __restrict__ t, const BOut* out,
                                                int from_xb) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tot = t->off_lv[t->n];
  for (int64_t i = gw; i < tot; i += nw) {
    const int r = find_req(t->off_lv, 0, t->n, i);
    const BReq* q = &t->r[r];
    const int64_t l = i - t->off_lv[r];
    const double inv = 1.0 / out[r].s;
    const double* src = from_xb ? q->xb : q->z;
    double e = 0.0;
    for (int k = lane; k < q->m; k += 32) {
      const int64_t j = l * q->m + k;
      const double p = src[j] * inv;
      e += fabs(p - q->x[j]);
      q->x[j] = p;
    }
    e = warp_sum(e);
    if (lane == 0) q->lsum[l] = e;
  }
}

// Refinement update per level: xb = x + d, level sum into lsum.
__global__ void __launch_bounds__(256) k_b_update(const BTable* __restrict__ t) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tot = t->off_lv[t->n];
  for (int64_t i = gw; i < tot; i += nw) {
    const int r = find_req(t->off_lv, 0, t->n, i);
    const BReq* q = &t->r[r];
    const int64_t l = i - t->off_lv[r];
    double e = 0.0;
    for (int k = lane; k < q->m; k += 32) {
      const int64_t j = l * q->m + k;
      const double v = q->x[j] + (double)q->d[j];
      q->xb[j] = v;
      e += v;
    }
    e = warp_sum(e);
    if (lane == 0) q->lsum[l] = e;
  }
}

__global__ void __launch_bounds__(256) k_b_zero_d(const BTable* __restrict__ t) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tot = t->off_lv[t->n];
  for (int64_t i = gw; i < tot; i += nw) {
    const int r = find_req(t->off_lv, 0, t->n, i);
    const BReq* q = &t->r[r];
    const int64_t l = i - t->off_lv[r];
    for (int k = lane; k < q->m; k += 32) q->d[l * q->m + k] = 0.0f;
  }
}

// Low-precision size classes: small bucket m <= 64 (G = GF = 1) and
// m <= 128 (G = GF = 2, FP32 or two-row BF16); large bucket m <= 256
// (FP32 G = 4, four-row BF16 G = 2; GF = 4).
template <typename TS, typename TL, bool COUPLED, bool LARGE>
__global__ void __launch_bounds__(256) k_b_phase_lp(const BTable* __restrict__ t, int half) {
  extern __shared__ float fsh[];
  constexpr int SL = LARGE ? 256 : 128;
  const int lane = threadIdx.x & 31;
  float* slice = fsh + (threadIdx.x >> 5) * 3 * SL;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t* off = half == 0 ? t->off_h1 : t->off_h2;
  int r0, r1;
  int64_t i0, i1;
  bucket(t, off, LARGE, r0, r1, i0, i1);
  for (int64_t i = i0 + gw; i < i1; i += nw) {
    const int r = find_req(off, r0, r1, i);
    const BReq* q = &t->r[r];
    const int par = half == 0 ? q->p1 : 1 - q->p1;
    const int64_t l = 2 * (i - off[r]) + par;
    if (LARGE) {
      constexpr int G = Pack<TL>::V == 2 ? 4 : 2;
      level_sweep_lp<TL, G, 4, COUPLED>((const TL*)q->lA, (const TL*)q->lB, q->lC, q->sc, q->d,
                                        q->q, l, q->L, q->m, q->lp_bs, q->lp_cbs, slice, lane);
    } else if (q->m <= 64) {
      level_sweep_lp<TS, 1, 1, COUPLED>((const TS*)q->lA, (const TS*)q->lB, q->lC, q->sc, q->d,
                                        q->q, l, q->L, q->m, q->lp_bs, q->lp_cbs, slice, lane);
    } else {
      level_sweep_lp<TS, 2, 2, COUPLED>((const TS*)q->lA, (const TS*)q->lB, q->lC, q->sc, q->d,
                                        q->q, l, q->L, q->m, q->lp_bs, q->lp_cbs, slice, lane);
    }
  }
}

template <typename K>
cudaError_t allow(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool C>
cudaError_t phase_pair(const BTable* t, int half, BGrid g, cudaStream_t s) {
  const size_t sm_small = (size_t)(g.threads / 32) * 3 * 32 * 4 * sizeof(double);
  const size_t sm_large = (size_t)(g.threads / 32) * 3 * 32 * 8 * sizeof(double);
  cudaError_t e = allow(k_b_phase<C, true>, sm_large);
  if (e != cudaSuccess) return e;
  k_b_phase<C, false><<<g.blocks, g.threads, sm_small, s>>>(t, half);
  k_b_phase<C, true><<<g.blocks, g.threads, sm_large, s>>>(t, half);
  return cudaGetLastError();
}

template <typename TS, typename TL, bool C>
cudaError_t lp_pair(const BTable* t, int half, BGrid g, cudaStream_t s) {
  const size_t sm_small = (size_t)(g.threads / 32) * 3 * 128 * sizeof(float);
  const size_t sm_large = (size_t)(g.threads / 32) * 3 * 256 * sizeof(float);
  cudaError_t e = allow(k_b_phase_lp<TS, TL, C, true>, sm_large);
  if (e != cudaSuccess) return e;
  k_b_phase_lp<TS, TL, C, false><<<g.blocks, g.threads, sm_small, s>>>(t, half);
  k_b_phase_lp<TS, TL, C, true><<<g.blocks, g.threads, sm_large, s>>>(t, half);
  return cudaGetLastError();
}

}  // namespace

cudaError_t b_sweep(const BTable* t, BOut* out, int coupled, BGrid g, cudaStream_t s) {
  for (int half = 0; half < 2; ++half) {
    const cudaError_t e = coupled ? phase_pair<true>(t, half, g, s) : phase_pair<false>(t, half, g, s);
    if (e != cudaSuccess) return e;
  }
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 0);
  k_b_norm<<<g.blocks, g.threads, 0, s>>>(t, out, 0);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 1);
  return cudaGetLastError();
}

cudaError_t b_resid(const BTable* t, BOut* out, int with_q, BGrid g, cudaStream_t s) {
  const size_t sm_small = (size_t)(g.threads / 32) * 3 * 32 * 4 * sizeof(double);
  const size_t sm_large = (size_t)(g.threads / 32) * 3 * 32 * 8 * sizeof(double);
  cudaError_t e = allow(k_b_resid<true>, sm_large);
  if (e != cudaSuccess) return e;
  k_b_resid<false><<<g.blocks, g.threads, sm_small, s>>>(t, with_q);
  k_b_resid<true><<<g.blocks, g.threads, sm_large, s>>>(t, with_q);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 2);
  return cudaGetLastError();
}

cudaError_t b_lp_step(const BTable* t, BOut* out, int bf16, int coupled, int inner, BGrid g,
                      cudaStream_t s) {
  k_b_zero_d<<<g.blocks, g.threads, 0, s>>>(t);
  for (int k = 0; k < inner; ++k)
    for (int half = 0; half < 2; ++half) {
      cudaError_t e;
      if (bf16)
        e = coupled ? lp_pair<Bf16x2, __nv_bfloat16, true>(t, half, g, s)
                    : lp_pair<Bf16x2, __nv_bfloat16, false>(t, half, g, s);
      else
        e = coupled ? lp_pair<float, float, true>(t, half, g, s)
                    : lp_pair<float, float, false>(t, half, g, s);
      if (e != cudaSuccess) return e;
    }
  k_b_update<<<g.blocks, g.threads, 0, s>>>(t);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 0);
  k_b_norm<<<g.blocks, g.threads, 0, s>>>(t, out, 1);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 1);
  return cudaGetLastError();
}

}  // namespace mc
