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
// *status unless it holds an earlier error).  Lane 0 polls; then
// every lane performs its own acquire of both counters, which orders its
// reads of the neighbour vectors after the producers' writes.
__device__ __forceinline__ void wait_neighbours(const int* ver, int64_t l, int64_t L, int need,
                                                int* status, int lane,
                                                unsigned long long wait_ns) {
  const bool lo = l > 0, up = l < L - 1;
  if (lane == 0) {
    unsigned long long t0 = 0;
    for (int it = 0;; ++it) {
      const bool ok = (!lo || ld_acquire(ver + l - 1) >= need) &&
                      (!up || ld_acquire(ver + l + 1) >= need);
      if (ok) break;
      if (it == 0) {
        t0 = global_ns();
      } else if (global_ns() - t0 > wait_ns) {
        atomicCAS(status, 0, (int)MC_ERR_TIMEOUT);
        break;
      }
      __nanosleep(128);
    }
  }
  __syncwarp();
  if (lo) (void)ld_acquire(ver + l - 1);
  if (up) (void)ld_acquire(ver + l + 1);
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
  bool ok = !mine || ld_acquire(ver + j) >= nj;
  if (!__all_sync(0xffffffffu, ok)) {
    const unsigned long long t0 = global_ns();
    while (true) {
      __nanosleep(128);
      if (!ok) ok = ld_acquire(ver + j) >= nj;
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
