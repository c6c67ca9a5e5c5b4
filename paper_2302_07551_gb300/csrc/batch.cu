// Batched kernels of the solve server (see batch.cuh): the per-level bodies
// of the single-chain kernels (level_sweep2, level_resid, level_sweep_lp)
// applied to every level of every active request in one persistent launch.
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "batch.cuh"
#include "lowprec_dev.cuh"
#include "sweep_dev.cuh"
#include "wave_dev.cuh"

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

// Request range [r0, r1) of the size classes [c0, c1) (the table is ordered
// by class).
__device__ __forceinline__ void class_range(const BTable* t, int c0, int c1, int& r0, int& r1) {
  r0 = c0 == 0 ? 0 : t->cls_end[c0 - 1];
  r1 = t->cls_end[c1 - 1];
}

constexpr unsigned long long kWaitNs = 2000000000ull;   // bound of one neighbour wait

// Unit q of a fused chunk of K sweeps over one bucket: sweep k, half-sweep h,
// request r and its levels l, l + 2, ..., l + 2 (n - 1) (a group of at most
// the request's G levels of one half-sweep: half-sweep 1 groups [a0, a1) of
// off_h1, then half-sweep 2 groups [b0, b1) of off_h2).
struct BUnit {
  int64_t k, l;
  int r, n;
  bool h2;
};

__device__ __forceinline__ BUnit unit_of(const BTable* t, unsigned long long q, int64_t n1,
                                         int64_t U, int64_t a0, int64_t b0, int r0, int r1) {
  BUnit u;
  u.k = (int64_t)(q / (unsigned long long)U);
  const int64_t rr = (int64_t)q - u.k * U;
  u.h2 = rr >= n1;
  const int64_t* off = u.h2 ? t->off_h2 : t->off_h1;
  const int64_t i = u.h2 ? b0 + (rr - n1) : a0 + rr;
  u.r = find_req(off, r0, r1, i);
  const BReq* Q = &t->r[u.r];
  const int par = u.h2 ? 1 - Q->p1 : Q->p1;
  const int64_t P = (Q->L - par + 1) / 2;        // levels of this half-sweep
  const int64_t g = i - off[u.r];
  const int G = Q->G;
  u.l = 2 * G * g + par;
  const int64_t left = P - (int64_t)G * g;
  u.n = left < G ? (int)left : G;
  return u;
}

// K FP64 sweeps of every request of one bucket (size classes [c0, c1), rows
// per lane up to RMAX) in one launch.  Per request: sweep 0 reads x, sweeps
// 0..K-2 write xb in place, sweep K-1 writes z (so xb keeps the previous
// sweep for the step error).
template <bool COUPLED, int RMAX>
__global__ void __launch_bounds__(256) k_b_sweeps(const BTable* __restrict__ t, int K, int c0,
                                                  int c1, unsigned long long* claim, BOut* out) {
  extern __shared__ double vsh[];
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * RMAX;
  int r0, r1;
  class_range(t, c0, c1, r0, r1);
  const int64_t a0 = t->off_h1[r0], a1 = t->off_h1[r1];
  const int64_t b0 = t->off_h2[r0], b1 = t->off_h2[r1];
  const int64_t n1 = a1 - a0, U = n1 + (b1 - b0);
  if (U == 0) return;
  const unsigned long long total = (unsigned long long)K * (unsigned long long)U;
  const int base = t->epoch;
  unsigned long long q0 = claim_unit(claim, lane);
  unsigned long long q = __shfl_sync(kFull, q0, 0);
  while (q < total) {
    q0 = claim_unit(claim, lane);
    const BUnit u = unit_of(t, q, n1, U, a0, b0, r0, r1);
    const BReq* Q = &t->r[u.r];
    const bool last = u.k == K - 1;
    double* dst = last ? Q->z : Q->xb;
    const double* src = u.h2 ? dst : (u.k == 0 ? Q->x : Q->xb);
    if (u.h2 || u.k > 0)
      wait_levels(Q->ver, u.l - 1, 2, u.n + 1, Q->L, base + (int)(u.h2 ? u.k + 1 : u.k),
                  &out[u.r].status, lane, kWaitNs);
    const bool want = u.k >= K - 2;   // e^T z of the last two sweeps only
    for (int i = 0; i < u.n; ++i) {
      const int64_t l = u.l + 2 * i;
      double ls;
      if constexpr (RMAX == 8) {
        ls = level_sweep2<8, COUPLED, false, true, true>(Q->A, Q->B, Q->C, src, src, dst, l,
                                                         Q->L, Q->m, Q->ms, slice, lane, 1.0,
                                                         nullptr, nullptr, nullptr, want);
      } else {
        switch (Q->R) {
          case 1: ls = level_sweep2<1, COUPLED, false, true, true>(Q->A, Q->B, Q->C, src, src, dst, l, Q->L, Q->m, Q->ms, slice, lane, 1.0, nullptr, nullptr, nullptr, want); break;
          case 2: ls = level_sweep2<2, COUPLED, false, true, true>(Q->A, Q->B, Q->C, src, src, dst, l, Q->L, Q->m, Q->ms, slice, lane, 1.0, nullptr, nullptr, nullptr, want); break;
          case 3: ls = level_sweep2<RMAX == 4 ? 3 : 2, COUPLED, false, true, true>(Q->A, Q->B, Q->C, src, src, dst, l, Q->L, Q->m, Q->ms, slice, lane, 1.0, nullptr, nullptr, nullptr, want); break;
          default: ls = level_sweep2<RMAX, COUPLED, false, true, true>(Q->A, Q->B, Q->C, src, src, dst, l, Q->L, Q->m, Q->ms, slice, lane, 1.0, nullptr, nullptr, nullptr, want); break;
        }
      }
      if (want && lane == 0) Q->lsum2[(u.k & 1) * Q->L + l] = ls;
    }
    publish_levels(Q->ver, u.l, 2, u.n, base + (int)u.k + 1, lane);
    q = __shfl_sync(kFull, q0, 0);
  }
}

// Direct residual of every request of the size classes up to m <= 128
// (LARGE = false) or m > 128 (LARGE = true).
template <bool LARGE>
__global__ void __launch_bounds__(256) k_b_resid(const BTable* __restrict__ t, int with_q) {
  extern __shared__ double vsh[];
  constexpr int RMAX = LARGE ? 8 : 4;
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * RMAX;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int r0, r1;
  class_range(t, LARGE ? 3 : 0, LARGE ? 4 : 3, r0, r1);
  const int64_t i0 = t->off_lv[r0], i1 = t->off_lv[r1];
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

// which: 0 -> s = e^T z (with the breakdown check), 1 -> step, 2 -> residual,
// 3 -> e^T z of the last two sweeps of a fused chunk of K sweeps (from lsum2).
// One block per request (grid-stride), fixed order: thread k adds levels
// k, k + blockDim, ..., then a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_b_reqsum(const BTable* __restrict__ t, BOut* out,
                                                  int which, int K = 1) {
  __shared__ double sh[32];
  for (int r = blockIdx.x; r < t->n; r += gridDim.x) {
    const BReq* q = &t->r[r];
    if (which == 3) {
      const double* a = q->lsum2 + ((K - 1) & 1) * q->L;
      const double* b = q->lsum2 + ((K - 2) & 1) * q->L;
      double va = 0.0, vb = 0.0;
      for (int64_t l = threadIdx.x; l < q->L; l += blockDim.x) {
        va += a[l];
        if (K >= 2) vb += b[l];
      }
      va = block_sum(va, sh);
      vb = block_sum(vb, sh);
      if (threadIdx.x == 0) {
        const double sp = K >= 2 ? vb : 1.0;
        out[r].s_last = va;
        out[r].s_prev = sp;
        out[r].s = va / sp;
        if (!(va > 0.0) || !isfinite(va) || !(sp > 0.0) || !isfinite(sp))
          out[r].status = MC_ERR_BREAKDOWN;
      }
      __syncthreads();
      continue;
    }
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

// x_l = src_l / s per level with the level's step error into lsum:
//   mode 0: src = z, s = e^T z, step against x;
//   mode 1: src = xb (refinement update), as mode 0;
//   mode 2: fused chunk of K sweeps: src = z / s_last, step against
//           x_prev / s_prev with x_prev = xb (K >= 2) or x (K = 1).
__global__ void __launch_bounds__(256) k_b_norm(const BTable* __restrict__ t, const BOut* out,
                                                int mode, int K = 1) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t tot = t->off_lv[t->n];
  for (int64_t i = gw; i < tot; i += nw) {
    const int r = find_req(t->off_lv, 0, t->n, i);
    const BReq* q = &t->r[r];
    const int64_t l = i - t->off_lv[r];
    const double inv = 1.0 / (mode == 2 ? out[r].s_last : out[r].s);
    const double pinv = mode == 2 ? 1.0 / out[r].s_prev : 1.0;
    const double* src = mode == 1 ? q->xb : q->z;
    const double* prev = (mode == 2 && K >= 2) ? q->xb : q->x;
    double e = 0.0;
    for (int k = lane; k < q->m; k += 32) {
      const int64_t j = l * q->m + k;
      const double p = src[j] * inv;
      e += fabs(p - prev[j] * pinv);
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

// Low-precision correction sweeps of one bucket (size classes [c0, c1)), all
// K sweeps of a refinement step in one launch, d in place.  Paths by the
// request's block size: m <= 64 -> 16-byte lane loads, BW loads in flight,
// several lanes per column; 64 < m <= 128 -> G = GF = 2 (FP32 or two-row
// BF16); m > 128 -> FP32 G = 4, four-row BF16 G = 2, GF = 4.  CLS bounds the
// paths a kernel holds (0: m <= 64, 1: m <= 128, 2: m > 128), so that each
// kernel has the register count of its largest path.
template <typename TS, typename TL, bool COUPLED, int CLS, int BW>
__global__ void __launch_bounds__(256) k_b_sweeps_lp(const BTable* __restrict__ t, int K, int c0,
                                                     int c1, unsigned long long* claim,
                                                     BOut* out) {
  extern __shared__ float fsh[];
  constexpr int SL = CLS == 2 ? 256 : 128;
  const int lane = threadIdx.x & 31;
  float* slice = fsh + (threadIdx.x >> 5) * 3 * SL;
  int r0, r1;
  class_range(t, c0, c1, r0, r1);
  const int64_t a0 = t->off_h1[r0], a1 = t->off_h1[r1];
  const int64_t b0 = t->off_h2[r0], b1 = t->off_h2[r1];
  const int64_t n1 = a1 - a0, U = n1 + (b1 - b0);
  if (U == 0) return;
  const unsigned long long total = (unsigned long long)K * (unsigned long long)U;
  const int base = t->epoch;
  unsigned long long q0 = claim_unit(claim, lane);
  unsigned long long q = __shfl_sync(kFull, q0, 0);
  while (q < total) {
    q0 = claim_unit(claim, lane);
    const BUnit u = unit_of(t, q, n1, U, a0, b0, r0, r1);
    const BReq* Q = &t->r[u.r];
    if (u.h2 || u.k > 0)
      wait_levels(Q->ver, u.l - 1, 2, u.n + 1, Q->L, base + (int)(u.h2 ? u.k + 1 : u.k),
                  &out[u.r].status, lane, kWaitNs);
    for (int i = 0; i < u.n; ++i) {
      const int64_t l = u.l + 2 * i;
      // the path follows the request's m alone (never the bucket), so every
      // bucketing computes a level with the same arithmetic
      if constexpr (CLS == 2) {
        constexpr int GL = Pack<TL>::V == 2 ? 4 : 2;
        level_sweep_lp<TL, GL, 4, COUPLED, true>((const TL*)Q->lA, (const TL*)Q->lB, Q->lC,
                                                 Q->sc, Q->d, Q->q, l, Q->L, Q->m, Q->lp_bs,
                                                 Q->lp_cbs, slice, lane);
      } else if (CLS == 1 && Q->m > 64) {
        level_sweep_lp<TS, 2, 2, COUPLED, true>((const TS*)Q->lA, (const TS*)Q->lB, Q->lC,
                                                Q->sc, Q->d, Q->q, l, Q->L, Q->m, Q->lp_bs,
                                                Q->lp_cbs, slice, lane);
      } else if (sizeof(TS) == 4 || Q->m % 8 == 0) {
        // 16-byte lane loads (BF16 columns 16-byte aligned when m % 8 == 0)
        using S = typename std::conditional<sizeof(TS) == 4 && !std::is_same<TS, Bf16x2>::value,
                                            float, unsigned short>::type;
        if (Q->m <= 16)
          level_sweep_lp_small<S, 16, COUPLED, true, BW>((const S*)Q->lA, (const S*)Q->lB,
                                                         Q->lC, Q->sc, Q->d, Q->q, l, Q->L, Q->m,
                                                         Q->lp_bs, Q->lp_cbs, slice, lane);
        else if (Q->m <= 32)
          level_sweep_lp_small<S, 32, COUPLED, true, BW>((const S*)Q->lA, (const S*)Q->lB,
                                                         Q->lC, Q->sc, Q->d, Q->q, l, Q->L, Q->m,
                                                         Q->lp_bs, Q->lp_cbs, slice, lane);
        else
          level_sweep_lp_small<S, 64, COUPLED, true, BW>((const S*)Q->lA, (const S*)Q->lB,
                                                         Q->lC, Q->sc, Q->d, Q->q, l, Q->L, Q->m,
                                                         Q->lp_bs, Q->lp_cbs, slice, lane);
      } else {
        level_sweep_lp<TS, 1, 1, COUPLED, true>((const TS*)Q->lA, (const TS*)Q->lB, Q->lC,
                                                Q->sc, Q->d, Q->q, l, Q->L, Q->m, Q->lp_bs,
                                                Q->lp_cbs, slice, lane);
      }
    }
    publish_levels(Q->ver, u.l, 2, u.n, base + (int)u.k + 1, lane);
    q = __shfl_sync(kFull, q0, 0);
  }
}

template <typename K>
cudaError_t allow(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Every bucket of a tuning: FP64 kernels sized for R <= 2, 4 or 8 rows per
// lane by the bucket's largest class.
template <bool C>
cudaError_t sweeps_buckets(const BTable* t, unsigned long long* claim, BOut* out, int K,
                           BTune g, cudaStream_t s) {
  const BBuckets b = buckets_of(g.split64);
  for (int i = 0; i < b.n; ++i) {
    const int rmax = b.c1[i] <= 2 ? 2 : b.c1[i] <= 3 ? 4 : 8;
    const size_t sm = (size_t)(g.threads / 32) * 3 * 32 * rmax * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (rmax == 2) {
      k_b_sweeps<C, 2><<<g.blocks, g.threads, sm, s>>>(t, K, b.c0[i], b.c1[i], claim + i, out);
    } else if (rmax == 4) {
      k_b_sweeps<C, 4><<<g.blocks, g.threads, sm, s>>>(t, K, b.c0[i], b.c1[i], claim + i, out);
    } else {
      e = allow(k_b_sweeps<C, 8>, sm);
      if (e != cudaSuccess) return e;
      k_b_sweeps<C, 8><<<g.blocks, g.threads, sm, s>>>(t, K, b.c0[i], b.c1[i], claim + i, out);
    }
  }
  return cudaGetLastError();
}

template <typename TS, typename TL, bool C>
cudaError_t lp_buckets(const BTable* t, unsigned long long* claim, BOut* out, int K, BTune g,
                       cudaStream_t s) {
  const BBuckets b = buckets_of(g.split64);
  const size_t sm_small = (size_t)(g.threads / 32) * 3 * 128 * sizeof(float);
  const size_t sm_large = (size_t)(g.threads / 32) * 3 * 256 * sizeof(float);
  cudaError_t e = allow(k_b_sweeps_lp<TS, TL, C, 2, 8>, sm_large);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < b.n; ++i) {
    const int c0 = b.c0[i], c1 = b.c1[i];
    if (c1 <= 2) {          // m <= 64
      if (g.deep)
        k_b_sweeps_lp<TS, TL, C, 0, 16><<<g.blocks, g.threads, sm_small, s>>>(t, K, c0, c1,
                                                                            claim + i, out);
      else
        k_b_sweeps_lp<TS, TL, C, 0, 8><<<g.blocks, g.threads, sm_small, s>>>(t, K, c0, c1,
                                                                           claim + i, out);
    } else if (c1 <= 3) {   // m <= 128
      k_b_sweeps_lp<TS, TL, C, 1, 8><<<g.blocks, g.threads, sm_small, s>>>(t, K, c0, c1,
                                                                         claim + i, out);
    } else {
      k_b_sweeps_lp<TS, TL, C, 2, 8><<<g.blocks, g.threads, sm_large, s>>>(t, K, c0, c1,
                                                                         claim + i, out);
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t b_sweeps(const BTable* t, unsigned long long* t_claim, BOut* out, int coupled, int K,
                     BTune g, cudaStream_t s) {
  return coupled ? sweeps_buckets<true>(t, t_claim, out, K, g, s)
                 : sweeps_buckets<false>(t, t_claim, out, K, g, s);
}

cudaError_t b_sweeps_finish(const BTable* t, BOut* out, int K, BTune g, cudaStream_t s) {
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 3, K);
  k_b_norm<<<g.blocks, g.threads, 0, s>>>(t, out, 2, K);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 1);
  return cudaGetLastError();
}

cudaError_t b_resid(const BTable* t, BOut* out, int with_q, BTune g, cudaStream_t s) {
  const size_t sm_small = (size_t)(g.threads / 32) * 3 * 32 * 4 * sizeof(double);
  const size_t sm_large = (size_t)(g.threads / 32) * 3 * 32 * 8 * sizeof(double);
  cudaError_t e = allow(k_b_resid<true>, sm_large);
  if (e != cudaSuccess) return e;
  k_b_resid<false><<<g.blocks, g.threads, sm_small, s>>>(t, with_q);
  k_b_resid<true><<<g.blocks, g.threads, sm_large, s>>>(t, with_q);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 2);
  return cudaGetLastError();
}

cudaError_t b_lp_zero(const BTable* t, BTune g, cudaStream_t s) {
  k_b_zero_d<<<g.blocks, g.threads, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t b_lp_sweeps(const BTable* t, unsigned long long* t_claim, BOut* out, int bf16,
                        int coupled, int inner, BTune g, cudaStream_t s) {
  cudaError_t e;
  if (bf16)
    e = coupled ? lp_buckets<Bf16x2, __nv_bfloat16, true>(t, t_claim, out, inner, g, s)
                : lp_buckets<Bf16x2, __nv_bfloat16, false>(t, t_claim, out, inner, g, s);
  else
    e = coupled ? lp_buckets<float, float, true>(t, t_claim, out, inner, g, s)
                : lp_buckets<float, float, false>(t, t_claim, out, inner, g, s);
  return e;
}

cudaError_t b_lp_finish(const BTable* t, BOut* out, BTune g, cudaStream_t s) {
  k_b_update<<<g.blocks, g.threads, 0, s>>>(t);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 0);
  k_b_norm<<<g.blocks, g.threads, 0, s>>>(t, out, 1);
  k_b_reqsum<<<g.blocks, 256, 0, s>>>(t, out, 1);
  return cudaGetLastError();
}

}  // namespace mc
