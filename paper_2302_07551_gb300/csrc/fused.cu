// Several staircase sweeps (Algorithm 2, repeated) in one persistent launch.
//
// Work units are (sweep k, half-sweep h, level l), claimed in that order from
// one queue counter.  Half-sweep 1 of sweep k (the diagonal-only stair rows)
// reads its neighbours as left by half-sweep 2 of sweep k-1; half-sweep 2
// reads its neighbours as left by half-sweep 1 of sweep k.  So each unit
// depends on exactly two earlier units, the neighbour levels l-1 and l+1, and
// waits for them through per-level completion counters instead of a launch
// boundary: the grid streams through all K sweeps with one ramp-up and one
// tail, and the queue balances the load across warps and SMs.
//
// The vector is updated in place (W).  A unit overwrites level l only after
// both units that read the old value of level l (its neighbours' previous
// updates) have completed, which is exactly the condition it waits for.  The
// last sweep writes Z instead, so that W keeps z_{K-1} for the step error.
//
// Progress: a warp handles its claimed units in increasing queue order and
// every unit depends only on units earlier in the queue, all claimed by
// running warps, so the earliest unfinished unit can always proceed.  Each
// wait is still bounded (FusedArgs::wait_ns of the GPU's global timer); on
// expiry the warp latches MC_ERR_TIMEOUT and carries on, so the launch
// always ends.
//
// Residual of the result (with_resid): P0 more units follow the K sweeps in
// the queue, one per diagonal-only level l.  The last sweep solved
// M z_K = N z_{K-1}, so Q^T z_K = N (z_{K-1} - z_K): zero on the coupled rows
// and T_lo d_{l-1} + T_up d_{l+1} (d = z_K - z_{K-1}) on the diagonal-only
// rows.  A residual unit waits until both neighbours hold z_K, reads z_K from
// Z and z_{K-1} from W (x_in when K = 1) and stores its level's L1 norm; this
// streams the off-diagonal blocks of half the levels once, a third of one
// sweep's bytes in inverse mode, instead of all three blocks of every level.
//
// Values and level sums do not depend on which warp handles which unit, and
// the sums are reduced per level in a fixed order: results are bitwise
// reproducible for any grid.
#include <math.h>

#include "mc_internal.cuh"
#include "sweep_dev.cuh"
#include "wave_dev.cuh"

namespace mc {

namespace {

using namespace dev;

template <int R, bool COUPLED, bool PAIRED>
__global__ void __launch_bounds__(256, Tune<R>::MINB) k_sweeps(FusedArgs a) {
  extern __shared__ double vsh[];
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * R;
  const unsigned long long sweeps = (unsigned long long)a.K * (unsigned long long)a.L;
  const unsigned long long total = sweeps + (a.with_resid ? (unsigned long long)a.P0 : 0ull);
  unsigned long long q0 = claim_unit(a.claim, lane);
  unsigned long long q = __shfl_sync(kFull, q0, 0);
  while (q < total) {
    // claim the next unit now; its index is needed only after this one
    q0 = claim_unit(a.claim, lane);
    if (q >= sweeps) {
      // residual unit of diagonal-only level l: neighbours must hold z_K
      const int64_t u = (int64_t)(q - sweeps);
      const int64_t l = 2 * u + a.par0;
      wait_neighbours(a.ver, l, a.L, (int)a.K, &a.hdr->status, lane, a.wait_ns);
      const double t = level_resid_split<R, PAIRED>(a.RA, a.RB, a.Z, a.prev, l, a.L, a.m, a.ms,
                                                    slice, lane);
      if (lane == 0) a.rsum[u] = t;
      q = __shfl_sync(kFull, q0, 0);
      continue;
    }
    const int64_t k = (int64_t)(q / (unsigned long long)a.L);
    const int64_t r = (int64_t)q - k * a.L;
    const bool h2 = r >= a.P0;
    const int64_t l = h2 ? 2 * (r - a.P0) + (1 - a.par0) : 2 * r + a.par0;
    const bool last = k == a.K - 1;
    double* dst = last ? a.Z : a.W;
    // half-sweep 1 reads z_k (x_in for k = 0); half-sweep 2 reads z_{k+1}
    const double* src = h2 ? dst : (k == 0 ? a.x_in : a.W);
    const int need = (int)(h2 ? k + 1 : k);
    if (need > 0) wait_neighbours(a.ver, l, a.L, need, &a.hdr->status, lane, a.wait_ns);
    // e^T z is needed of the last two sweeps only
    const bool want = k >= a.K - 2;
    const double t = level_sweep2<R, COUPLED, PAIRED, true, true>(
        a.A, a.B, a.C, src, src, dst, l, a.L, a.m, a.ms, slice, lane, 1.0, nullptr, nullptr,
        nullptr, want);
    if (want && lane == 0) a.lsum[(k & 1) * a.L + l] = t;
    publish(a.ver + l, (int)(k + 1), lane);
    q = __shfl_sync(kFull, q0, 0);
  }
}

// Block-banded chains (Algorithm 2 with off-staircase terms, inverse mode):
// every row also adds sum_d T_{l,l+d} x_{l+d} over the far diagonals |d| >= 2
// from the sweep's input, at levels of both parities, so the sweeps cannot
// update in place.  Y_0 = x_in; sweep k reads Y_k and writes Y_{k+1} into W
// (k even) or Z (k odd), over Y_{k-1}.  A unit of sweep k at level l waits
// until every level within the band l - bw .. l + bw has finished sweep k - 1
// (its inputs are ready and every reader of the Y_{k-1} it overwrites is
// done); a coupled-row unit also waits for half-sweep 1 of sweep k at l - 1
// and l + 1.
template <int R>
__global__ void __launch_bounds__(256, Tune<R>::MINB) k_sweeps_banded(FusedArgs a) {
  extern __shared__ double vsh[];
  const int lane = threadIdx.x & 31;
  double* slice = vsh + (threadIdx.x >> 5) * 3 * 32 * R;
  const unsigned long long total = (unsigned long long)a.K * (unsigned long long)a.L;
  unsigned long long q0 = claim_unit(a.claim, lane);
  unsigned long long q = __shfl_sync(kFull, q0, 0);
  while (q < total) {
    q0 = claim_unit(a.claim, lane);
    const int64_t k = (int64_t)(q / (unsigned long long)a.L);
    const int64_t r = (int64_t)q - k * a.L;
    const bool h2 = r >= a.P0;
    const int64_t l = h2 ? 2 * (r - a.P0) + (1 - a.par0) : 2 * r + a.par0;
    const double* y = k == 0 ? a.x_in : ((k & 1) ? a.W : a.Z);   // Y_k
    double* dst = (k & 1) ? a.Z : a.W;                             // Y_{k+1}
    if (k > 0 || h2)
      wait_band(a.ver, l, a.L, a.bw, (int)k, (int)(h2 ? k + 1 : k), &a.hdr->status, lane,
                a.wait_ns);
    const double* near = h2 ? dst : y;
    const bool want = k >= a.K - 2;
    const double t = level_sweep2<R, false, false, true, true>(
        a.A, a.B, a.C, near, near, dst, l, a.L, a.m, a.ms, slice, lane, 1.0, a.far, y, y, want);
    if (want && lane == 0) a.lsum[(k & 1) * a.L + l] = t;
    publish(a.ver + l, (int)(k + 1), lane);
    q = __shfl_sync(kFull, q0, 0);
  }
}

// Block Gauss-Seidel sweeps (Sect. 2 comparison splitting, M = block lower
// triangle of Q^T), all K sweeps of a call in one persistent launch:
// z^{k+1}_l = (-T_dd)^{-1} (T_lo z^{k+1}_{l-1} + T_up z^k_{l+1}) (inverse mode;
// W_lo, W_up when coupled).  Unit (k, l) needs (k, l-1) and (k-1, l+1), so the
// units are claimed in wavefront order (wave_unit): a sweep traverses the
// levels one after the other, each sweep trailing the previous one by two
// levels, and up to min(K, L / 2) units run at once.  In place in W (the
// last sweep writes Z): a unit overwrites z^k_l only after its two readers,
// (k, l-1) and (k-1, l+1), have completed, which is what it waits for.
//
// One block of kBgsWarps warps per unit: the warps split the columns of every
// block product (warp w takes a fixed even-aligned column range and keeps
// partial sums of all rows), and the partials are added in warp order.  A
// unit sits on the wavefront's critical path, so streaming its blocks with
// several warps' loads in flight instead of one shortens that path; the
// launch runs one block per unit in flight.  Four warps measured best (2, 4
// and 8 tried: fewer warps per unit leave more units resident at once).  Warp 0 waits for the two neighbours, the block barrier
// hands the wait on (every warp also acquires both counters), and after its
// stores every thread fences before thread 0 releases the level.  The
// vectors sit in block shared memory with 16 zero doubles of padding, so a
// warp's last column batch may read past its range (those products are with
// zero block entries).
constexpr int kBgsWarps = 4;

__device__ __forceinline__ double bgs_parts(const double* part, int W, int i) {
  if constexpr (kBgsWarps == 8)
    return ((part[i] + part[W + i]) + (part[2 * W + i] + part[3 * W + i])) +
           ((part[4 * W + i] + part[5 * W + i]) + (part[6 * W + i] + part[7 * W + i]));
  else if constexpr (kBgsWarps == 4)
    return (part[i] + part[W + i]) + (part[2 * W + i] + part[3 * W + i]);
  else
    return part[i] + part[W + i];
}

template <int R, bool COUPLED>
__global__ void __launch_bounds__(32 * kBgsWarps, 16 / kBgsWarps) k_bgs_cta(FusedArgs a) {
  constexpr int W = 32 * R, VS = W + 16;
  extern __shared__ double sh[];
  double* v_lo = sh;
  double* v_up = sh + VS;
  double* v_g = sh + 2 * VS;
  double* part = sh + 3 * VS;   // kBgsWarps x W partial sums
  __shared__ double red[kBgsWarps];
  __shared__ unsigned long long s_q;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nt = blockDim.x;
  const int m = a.m;
  const int cw = (((m + kBgsWarps - 1) / kBgsWarps) + 1) & ~1;
  const int j0 = w * cw, j1 = j0 + cw < m ? j0 + cw : m;
  for (int i = threadIdx.x; i < 3 * VS; i += nt) sh[i] = 0.0;   // pads stay zero
  const unsigned long long total = (unsigned long long)a.K * (unsigned long long)a.L;
  while (true) {
    if (threadIdx.x == 0) s_q = atomicAdd(a.claim, 1ull);
    __syncthreads();
    const unsigned long long q = s_q;
    if (q >= total) break;
    int64_t k, l;
    wave_unit(q, a.L, a.K, &k, &l);
    double* dst = k == a.K - 1 ? a.Z : a.W;
    const double* up = k == 0 ? a.x_in : a.W;    // z^k at l + 1
    const bool has_lo = l > 0, has_up = l < a.L - 1;
    if (w == 0)
      wait_neighbours2(a.ver, l, a.L, (int)(k + 1), (int)k, &a.hdr->status, lane, a.wait_ns);
    __syncthreads();
    if (w != 0) {
      if (has_lo) (void)ld_acquire(a.ver + l - 1);
      if (has_up && k > 0) (void)ld_acquire(a.ver + l + 1);
    }
    for (int i = threadIdx.x; i < m; i += nt) {
      v_lo[i] = has_lo ? __ldcg(dst + (l - 1) * m + i) : 0.0;
      v_up[i] = has_up ? __ldcg(up + (l + 1) * m + i) : 0.0;
    }
    __syncthreads();
    double acc[R][Tune<R>::NA];
    zero_acc<R>(acc);
    if (j0 < j1) {
      if (has_lo) gemv_acc_part<R, 0, R>(acc, a.A + (size_t)l * a.ms, v_lo, j0, j1, m, lane);
      if (has_up) gemv_acc_part<R, 0, R>(acc, a.B + (size_t)l * a.ms, v_up, j0, j1, m, lane);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) part[w * W + lane + 32 * r] = fold<R>(acc[r]);
    __syncthreads();
    if (!COUPLED) {
      for (int i = threadIdx.x; i < m; i += nt) v_g[i] = bgs_parts(part, W, i);
      __syncthreads();
      zero_acc<R>(acc);
      if (j0 < j1) gemv_acc_part<R, 0, R>(acc, a.C + (size_t)l * a.ms, v_g, j0, j1, m, lane);
#pragma unroll
      for (int r = 0; r < R; ++r) part[w * W + lane + 32 * r] = fold<R>(acc[r]);
      __syncthreads();
    }
    double ls = 0.0;
    for (int i = threadIdx.x; i < m; i += nt) {
      const double z = bgs_parts(part, W, i);
      dst[l * m + i] = z;
      ls += z;
    }
    if (k >= a.K - 2) {   // e^T z of the last two sweeps only (uniform over the block)
      ls = block_sum(ls, red);
      if (threadIdx.x == 0) a.lsum[(k & 1) * a.L + l] = ls;
    }
    __threadfence();
    __syncthreads();   // every store of z_l, and every read of part, before the release
    if (threadIdx.x == 0) st_release(a.ver + l, (int)(k + 1));
  }
}

// Self-test of the bounded wait: one warp waits for level 1 of a 3-level
// counter array; the counters hold `preset`, the wait needs 1.
__global__ void k_wait_selftest(int preset, unsigned long long wait_ns, Header* hdr, int* ver) {
  const int lane = threadIdx.x & 31;
  if (lane < 3) ver[lane] = preset;
  __syncwarp();
  wait_neighbours(ver, 1, 3, 1, &hdr->status, lane, wait_ns);
}

// e^T z_K and e^T z_{K-1} from the per-level sums, and the residual from the
// per-level residual norms.  FP64 adds run at two lanes per clock per SM
// here, so the sums are spread over kScaleBlocks blocks, each over a fixed
// contiguous range of levels; the last block to finish adds the block
// partials (fixed summation order).
// part: 3 kScaleBlocks doubles of scratch; ticket: zero between launches.
__global__ void __launch_bounds__(256) k_fused_scale(const double* lsum, int64_t L, int64_t K,
                                                     const double* rsum, int64_t P,
                                                     double* part, unsigned* ticket,
                                                     double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double* a = lsum + ((K - 1) & 1) * L;
  const double* b = lsum + ((K - 2) & 1) * L;
  const int64_t chunk = (L + gridDim.x - 1) / gridDim.x;
  const int64_t l0 = blockIdx.x * chunk;
  const int64_t l1 = l0 + chunk < L ? l0 + chunk : L;
  double ta = 0.0, tb = 0.0, tr = 0.0;
  for (int64_t l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
    ta += a[l];
    if (K >= 2) tb += b[l];
  }
  if (rsum) {
    const int64_t pc = (P + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = blockIdx.x * pc;
    const int64_t p1 = p0 + pc < P ? p0 + pc : P;
    for (int64_t u = p0 + threadIdx.x; u < p1; u += blockDim.x) tr += rsum[u];
  }
  ta = block_sum(ta, sh);
  tb = block_sum(tb, sh);
  tr = block_sum(tr, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = ta;
    part[3 * blockIdx.x + 1] = tb;
    part[3 * blockIdx.x + 2] = tr;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // the first warp loads the partials in parallel (lane i: blocks i, i + 32)
  // and adds them with a fixed shuffle tree
  double sa = 0.0, sb = 0.0, sr = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) {
    sa += __ldcg(part + 3 * i);
    sb += __ldcg(part + 3 * i + 1);
    sr += __ldcg(part + 3 * i + 2);
  }
  sa = warp_sum(sa);
  sb = warp_sum(sb);
  sr = warp_sum(sr);
  if (threadIdx.x == 0) {
    out[0] = sa;
    out[1] = K >= 2 ? sb : 1.0;
    out[2] = rsum ? sr : nan("");
    *ticket = 0u;
  }
}

template <int R, bool C, bool P = false>
cudaError_t sweeps_r(const FusedArgs& a, int nb, cudaStream_t s) {
  static bool done = false;
  const size_t smem = (size_t)kWarpsPerBlock * 3 * 32 * R * sizeof(double);
  if (!done && smem > 40 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_sweeps<R, C, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    done = true;
  }
  k_sweeps<R, C, P><<<nb, 256, smem, s>>>(a);
  return cudaGetLastError();
}

// nb: units that can run at once (capped here at the blocks resident at once,
// so every claimed unit belongs to a running block).
template <int R, bool C>
cudaError_t bgs_fused_r(const FusedArgs& a, int nb, cudaStream_t s) {
  static int cap = 0;
  const size_t smem = (size_t)(3 * (32 * R + 16) + kBgsWarps * 32 * R) * sizeof(double);
  if (cap == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bgs_cta<R, C>, 32 * kBgsWarps,
                                                        smem);
    if (e != cudaSuccess) return e;
    cap = (occ < 1 ? 1 : occ) * sms;
  }
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  k_bgs_cta<R, C><<<nb, 32 * kBgsWarps, smem, s>>>(a);
  return cudaGetLastError();
}

template <int R>
cudaError_t banded_r(const FusedArgs& a, int nb, cudaStream_t s) {
  static bool done = false;
  const size_t smem = (size_t)kWarpsPerBlock * 3 * 32 * R * sizeof(double);
  if (!done && smem > 40 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_sweeps_banded<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    done = true;
  }
  k_sweeps_banded<R><<<nb, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool C>
cudaError_t sweeps_dispatch(const FusedArgs& a, int nb, cudaStream_t s) {
  if (a.bgs) {
    if (a.far || a.paired) return cudaErrorInvalidValue;
    switch ((a.m + 31) / 32) {
      case 1: return bgs_fused_r<1, C>(a, nb, s);
      case 2: return bgs_fused_r<2, C>(a, nb, s);
      case 3: return bgs_fused_r<3, C>(a, nb, s);
      case 4: return bgs_fused_r<4, C>(a, nb, s);
      case 5: return bgs_fused_r<5, C>(a, nb, s);
      case 6: return bgs_fused_r<6, C>(a, nb, s);
      case 7: return bgs_fused_r<7, C>(a, nb, s);
      case 8: return bgs_fused_r<8, C>(a, nb, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.far) {
    if (C) return cudaErrorInvalidValue;   // block-banded chains: inverse mode only
    switch ((a.m + 31) / 32) {
      case 1: return banded_r<1>(a, nb, s);
      case 2: return banded_r<2>(a, nb, s);
      case 3: return banded_r<3>(a, nb, s);
      case 4: return banded_r<4>(a, nb, s);
      case 5: return banded_r<5>(a, nb, s);
      case 6: return banded_r<6>(a, nb, s);
      case 7: return banded_r<7>(a, nb, s);
      case 8: return banded_r<8>(a, nb, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.paired && !C) {
    switch (a.m / 32) {
      case 2: return sweeps_r<2, false, true>(a, nb, s);
      case 4: return sweeps_r<4, false, true>(a, nb, s);
      case 6: return sweeps_r<6, false, true>(a, nb, s);
      case 8: return sweeps_r<8, false, true>(a, nb, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch ((a.m + 31) / 32) {
    case 1: return sweeps_r<1, C>(a, nb, s);
    case 2: return sweeps_r<2, C>(a, nb, s);
    case 3: return sweeps_r<3, C>(a, nb, s);
    case 4: return sweeps_r<4, C>(a, nb, s);
    case 5: return sweeps_r<5, C>(a, nb, s);
    case 6: return sweeps_r<6, C>(a, nb, s);
    case 7: return sweeps_r<7, C>(a, nb, s);
    case 8: return sweeps_r<8, C>(a, nb, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_sweeps_fused(const FusedArgs& a, int coupled, int n_blocks, cudaStream_t s) {
  return coupled ? sweeps_dispatch<true>(a, n_blocks, s) : sweeps_dispatch<false>(a, n_blocks, s);
}

cudaError_t launch_wait_selftest(int preset, unsigned long long wait_ns, Header* hdr, int* ver,
                                 cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(preset, wait_ns, hdr, ver);
  return cudaGetLastError();
}

cudaError_t launch_fused_scale(const double* lsum, int64_t L, int64_t K, const double* rsum,
                               int64_t P, double* out, double* part, unsigned* ticket,
                               cudaStream_t s) {
  k_fused_scale<<<kScaleBlocks, 256, 0, s>>>(lsum, L, K, rsum, P, part, ticket, out);
  return cudaGetLastError();
}

}  // namespace mc

namespace {
struct WaitSelftestScratch {
  mc::Header hdr;
  int ver[4];
};
__device__ __align__(256) WaitSelftestScratch g_wait_selftest;
}  // namespace

extern "C" int mc_wait_selftest(void* cuda_stream, int reachable, int64_t wait_ns) {
  if (wait_ns < 0 || wait_ns > 10000000000ll) return MC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_wait_selftest) != cudaSuccess || !p) return MC_ERR_CUDA;
  WaitSelftestScratch* w = (WaitSelftestScratch*)p;
  if (cudaMemsetAsync(w, 0, sizeof(WaitSelftestScratch), s) != cudaSuccess) return MC_ERR_CUDA;
  if (mc::launch_wait_selftest(reachable ? 1 : 0, (unsigned long long)wait_ns, &w->hdr, w->ver,
                               s) != cudaSuccess)
    return MC_ERR_CUDA;
  int status = 0;
  if (cudaMemcpyAsync(&status, &w->hdr.status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MC_ERR_CUDA;
  return status;
}
