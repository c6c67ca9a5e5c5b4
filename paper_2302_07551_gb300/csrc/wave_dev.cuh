// Device helpers of the fused multi-sweep launches (FP64 and low precision):
// per-level completion counters with acquire / release ordering, bounded
// waits on them, and the queue claim.
//
// A unit (sweep k, half-sweep h, level l) waits until its neighbour levels
// l-1 and l+1 have completed `need` writes in the launch, then publishes its
// own level with the next count.  Waits are bounded by the GPU's global timer:
// on expiry the warp latches MC_ERR_TIMEOUT and carries on, so a launch
// always ends.
#pragma once
#include <stdint.h>

#include "mc_internal.cuh"

namespace mc {
namespace dev {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Polling load: relaxed (no ordering, no L1 invalidation as an acquire at
// GPU scope would do on every poll); the acquire follows once the value is
// ready.
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Back-off between polls: 32 ns doubling to 256 ns.  Polls are relaxed loads
// (cheap), while a long sleep keeps a warp idle after its neighbours are
// ready: with block-banded dependencies (a unit waits for a whole band of the
// previous sweep) a 2 us cap left the FP64 pipe idle 16 % of the time.
__device__ __forceinline__ unsigned backoff(unsigned ns) {
  __nanosleep(ns);
  return ns < 256u ? 2u * ns : ns;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until levels l-1 and l+1 (where they exist) have completed `need`
// writes, for at most wait_ns nanoseconds (then MC_ERR_TIMEOUT is latched in
// *status unless it holds an earlier error).  Lane 0 polls with relaxed
// loads; then every lane performs its own acquire of both counters, which
// orders its reads of the neighbour vectors after the producers' writes.
__device__ __forceinline__ void wait_neighbours(const int* ver, int64_t l, int64_t L, int need,
                                                int* status, int lane,
                                                unsigned long long wait_ns) {
  const bool lo = l > 0, up = l < L - 1;
  if (lane == 0) {
    unsigned long long t0 = 0;
    unsigned ns = 32;
    for (int it = 0;; ++it) {
      const bool ok = (!lo || ld_relaxed(ver + l - 1) >= need) &&
                      (!up || ld_relaxed(ver + l + 1) >= need);
      if (ok) break;
      if (it == 0) {
        t0 = global_ns();
      } else if (global_ns() - t0 > wait_ns) {
        atomicCAS(status, 0, (int)MC_ERR_TIMEOUT);
        break;
      }
      ns = backoff(ns);
    }
  }
  __syncwarp();
  if (lo) (void)ld_acquire(ver + l - 1);
  if (up) (void)ld_acquire(ver + l + 1);
}

// As wait_neighbours with separate counts for the two neighbours: level l-1
// must have completed need_lo writes and level l+1 need_up (<= 0: no wait).
__device__ __forceinline__ void wait_neighbours2(const int* ver, int64_t l, int64_t L,
                                                 int need_lo, int need_up, int* status, int lane,
                                                 unsigned long long wait_ns) {
  const bool lo = l > 0 && need_lo > 0, up = l < L - 1 && need_up > 0;
  if (lane == 0) {
    unsigned long long t0 = 0;
    unsigned ns = 32;
    for (int it = 0;; ++it) {
      const bool ok = (!lo || ld_relaxed(ver + l - 1) >= need_lo) &&
                      (!up || ld_relaxed(ver + l + 1) >= need_up);
      if (ok) break;
      if (it == 0) {
        t0 = global_ns();
      } else if (global_ns() - t0 > wait_ns) {
        atomicCAS(status, 0, (int)MC_ERR_TIMEOUT);
        break;
      }
      ns = backoff(ns);
    }
  }
  __syncwarp();
  if (lo) (void)ld_acquire(ver + l - 1);
  if (up) (void)ld_acquire(ver + l + 1);
}

// Wavefront order of the units (sweep k, level l), 0 <= k < K, 0 <= l < L,
// of fused block Gauss-Seidel sweeps: by anti-diagonal t = 2k + l, then k.
// Unit (k, l) needs (k, l-1) and (k-1, l+1), both on diagonal t - 1, so every
// unit depends only on units earlier in the order, and the units of one
// diagonal are independent.  wave_prefix(t) counts the units with 2k + l < t:
// the sweeps k with 2k + L <= t contribute L levels each, those with
// 2k < t < 2k + L contribute t - 2k.
__device__ __forceinline__ int64_t wave_prefix(int64_t t, int64_t L, int64_t K) {
  int64_t a = t >= L ? (t - L) / 2 + 1 : 0;
  if (a > K) a = K;
  int64_t b = (t + 1) / 2;
  if (b > K) b = K;
  return a * L + (b - a) * t - (b - a) * (a + b - 1);
}

// Queue position q (< K L) -> (k, l) in wavefront order: the diagonal by
// bisection on wave_prefix, then the sweep within it.
__device__ __forceinline__ void wave_unit(unsigned long long q, int64_t L, int64_t K, int64_t* k,
                                          int64_t* l) {
  const int64_t qq = (int64_t)q;
  int64_t lo = 0, hi = 2 * (K - 1) + L;   // wave_prefix(lo) <= q < wave_prefix(hi)
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (wave_prefix(mid, L, K) <= qq)
      lo = mid;
    else
      hi = mid;
  }
  const int64_t k0 = lo >= L ? (lo - L + 2) / 2 : 0;   // first sweep on diagonal lo
  *k = k0 + (qq - wave_prefix(lo, L, K));
  *l = lo - 2 * *k;
}

// Block-banded dataflow: wait until every level j in [l - bw, l + bw] has
// completed `need` writes and, when near_need > need, levels l - 1 and l + 1
// have completed near_need; lane i polls level l - bw + i (2 bw + 1 <= 32).
// Afterwards every lane acquires all of them itself (its reads of any of these
// levels are ordered after the producers' writes).  Bounded like
// wait_neighbours.
__device__ __forceinline__ void wait_band(const int* ver, int64_t l, int64_t L, int bw, int need,
                                          int near_need, int* status, int lane,
                                          unsigned long long wait_ns) {
  const int64_t j = l - bw + lane;
  const bool mine = lane <= 2 * bw && j >= 0 && j < L;
  const int nj = (j == l - 1 || j == l + 1) ? near_need : need;
  bool ok = !mine || ld_relaxed(ver + j) >= nj;
  if (!__all_sync(0xffffffffu, ok)) {
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while (true) {
      ns = backoff(ns);
      if (!ok) ok = ld_relaxed(ver + j) >= nj;
      if (__all_sync(0xffffffffu, ok)) break;
      if (__any_sync(0xffffffffu, global_ns() - t0 > wait_ns)) {
        if (lane == 0) atomicCAS(status, 0, (int)MC_ERR_TIMEOUT);
        break;
      }
    }
  }
  for (int64_t i = l - bw; i <= l + bw; ++i)
    if (i >= 0 && i < L) (void)ld_acquire(ver + i);
}

// Wait until the `count` (<= 32) levels first, first + stride, ... (those in
// [0, L)) have completed `need` writes; lane i polls level first + stride i.
// Afterwards every lane acquires all of them itself.  Bounded like
// wait_neighbours.
__device__ __forceinline__ void wait_levels(const int* ver, int64_t first, int stride, int count,
                                            int64_t L, int need, int* status, int lane,
                                            unsigned long long wait_ns) {
  const int64_t j = first + (int64_t)stride * lane;
  const bool mine = lane < count && j >= 0 && j < L;
  bool ok = !mine || ld_relaxed(ver + j) >= need;
  if (!__all_sync(0xffffffffu, ok)) {
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while (true) {
      ns = backoff(ns);
      if (!ok) ok = ld_relaxed(ver + j) >= need;
      if (__all_sync(0xffffffffu, ok)) break;
      if (__any_sync(0xffffffffu, global_ns() - t0 > wait_ns)) {
        if (lane == 0) atomicCAS(status, 0, (int)MC_ERR_TIMEOUT);
        break;
      }
    }
  }
  for (int i = 0; i < count; ++i) {
    const int64_t jj = first + (int64_t)stride * i;
    if (jj >= 0 && jj < L) (void)ld_acquire(ver + jj);
  }
}

// Levels first, first + stride, ... (count <= 32) now hold version v: every
// lane's stores are made visible before lane i releases level
// first + stride i.
__device__ __forceinline__ void publish_levels(int* ver, int64_t first, int stride, int count,
                                               int v, int lane) {
  __threadfence();
  __syncwarp();
  if (lane < count) st_release(ver + first + (int64_t)stride * lane, v);
}

// Level l now holds its version v: every lane's stores of z_l are made
// visible before the counter.
__device__ __forceinline__ void publish(int* ver, int v, int lane) {
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release(ver, v);
}

// Next queue position for the whole warp (lane 0 claims).
__device__ __forceinline__ unsigned long long claim_unit(unsigned long long* q, int lane) {
  return lane == 0 ? atomicAdd(q, 1ull) : 0ull;
}

}  // namespace dev
}  // namespace mc
