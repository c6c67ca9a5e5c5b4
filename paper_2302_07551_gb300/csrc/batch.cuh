// Batched (multi-request) sweep: descriptors shared by batch.cu and server.cu.
//
// All active requests of the solve server advance together: one fused
// persistent launch per block-size bucket covers every level of every
// request for all sweeps of a chunk (details below).  The request
// table lives in device memory and is rewritten by the host between chunks,
// so one captured CUDA graph serves any active set.  Requests are ordered by
// size class (m <= 32, m <= 64, m <= 128, m <= 256: rows per lane R <= 1, 2,
// 4, 8); a bucket is a run of classes launched as one kernel sized for its
// largest block, so that register use follows the bucket.  Where the bucket
// edges lie is a tuning choice (BTune::split64).
//
// Every reduction is per level first (one partial per level), then per
// request in level order: a request's iterates do not depend on which other
// requests share the launch, nor on any choice of the autotuner (grid,
// levels per unit, bucket edges, load depth).
//
// The sweeps of a chunk run fused (as the single-chain fused sweeps): one
// persistent launch per bucket for all sweeps of the chunk, units claimed in
// order, each waiting for its neighbour levels through the request's
// completion counters.  A unit covers G adjacent levels of one half-sweep of
// one request (levels l0, l0 + 2, ..., l0 + 2 (G - 1); G per request, from
// the table's G and the request's size class): one claim, one wait for the
// G + 1 neighbour levels, one completion fence.  Counters grow across
// chunks: a chunk with epoch E writes E + k + 1 after its sweep k, so counters
// never need resetting (new requests start at zero <= E); the claim counters
// live in the table and are reset by the table copy that starts every chunk.
#pragma once
#include "mc_internal.cuh"

namespace mc {

constexpr int kMaxReq = 1024;

struct BReq {
  const double* A;      // FP64 sweep operators: T_lo / W_lo
  const double* B;      // T_up / W_up
  const double* C;      // (-T_dd)^{-1} (inverse mode)
  const double* TLO;    // residual blocks
  const double* TDD;
  const double* TUP;
  const double* NINV;
  const void* lA;       // low-precision operators (dtype MC_F32 / MC_BF16)
  const void* lB;
  const float* lC;
  const float* sc;
  float* d;             // correction (low precision)
  float* q;             // (-T_dd)^{-1} r
  double* x;            // iterate pi
  double* z;            // unnormalised sweep output
  double* xb;           // pi + d before renormalisation
  double* lsum;         // one partial per level
  double* lsum2;        // fused sweeps: [2][L] level sums of the last two sweeps
  int* ver;             // fused sweeps: per-level completion counters
  int64_t L;
  int32_t m, ms, R, p1;  // p1: 0-based parity of the diagonal-only rows
  int32_t G, pad;        // levels per unit of this request (the table's G scaled by size class)
  int64_t lp_bs, lp_cbs;
};

// Size classes of the request table: m <= 32, 64, 128, 256.
constexpr int kClasses = 4;
__host__ __device__ inline int size_class(int m) { return m <= 32 ? 0 : m <= 64 ? 1 : m <= 128 ? 2 : 3; }
// Levels per unit of a request: the table's G times 4, 2, 1, 1 by size class
// (at most 16), so that a unit of small blocks carries about as many bytes as
// one of m <= 128 and the claim, the wait and the fence are paid less often.
__host__ __device__ inline int class_group(int G, int m) {
  const int c = size_class(m);
  const int g = G * (c == 0 ? 4 : c == 1 ? 2 : 1);
  return g > 16 ? 16 : g;
}

struct BTable {
  int32_t n;            // active requests, ordered by size class
  int32_t cls_end[kClasses];     // requests [0, cls_end[c]) have size class <= c
  int32_t epoch;        // completion-counter base of this chunk
  int32_t G;            // levels per unit of the fused sweep launches (1, 2 or 4), scaled
                        // per request by class_group
  int32_t pad;
  unsigned long long claim[kClasses];   // queue counters of one chunk's buckets (0 in t_host)
  int64_t off_h1[kMaxReq + 1];   // prefix counts of half-sweep-1 units (groups of G levels)
  int64_t off_h2[kMaxReq + 1];   // prefix counts of half-sweep-2 units
  int64_t off_lv[kMaxReq + 1];   // prefix counts of all levels
  BReq r[kMaxReq];
};

struct BOut {
  double s, step, resid;
  double s_last, s_prev;   // fused FP64 chunk: e^T z of its last two sweeps (s_prev = 1 for one)
  int32_t status;
  int32_t pad;
};

// Launch configuration of a chunk, chosen per batch signature by the server's
// autotuner from live chunk timings.  The levels per unit G travel in the
// request table (its unit prefix counts depend on G).
struct BTune {
  int blocks, threads;  // persistent grid of the fused launches
  int split64;          // 1: m <= 64 in a launch of its own (kernel for R <= 2);
                        // 0: m <= 128 in one launch (kernel for R <= 4)
  int deep;             // low-precision blocks of m <= 64: 16 (1) or 8 (0) loads in flight
};

// The buckets (runs of size classes launched as one kernel) of a tuning:
// FP64 and low precision alike, [c0[i], c1[i]) for i < n.
struct BBuckets {
  int n;
  int c0[kClasses], c1[kClasses];
};
inline BBuckets buckets_of(int split64) {
  BBuckets b{};
  if (split64) {
    b.n = 3;
    b.c0[0] = 0, b.c1[0] = 2;
    b.c0[1] = 2, b.c1[1] = 3;
    b.c0[2] = 3, b.c1[2] = 4;
  } else {
    b.n = 2;
    b.c0[0] = 0, b.c1[0] = 3;
    b.c0[1] = 3, b.c1[1] = 4;
  }
  return b;
}

// K FP64 sweeps of every request (fused launches, no normalisation in
// between); then (b_sweeps_finish) e^T z, normalisation and the step error of
// the last sweep.  t_claim: the device table's claim counters.  coupled:
// server-wide apply mode.
cudaError_t b_sweeps(const BTable* t, unsigned long long* t_claim, BOut* out, int coupled, int K,
                     BTune g, cudaStream_t s);
cudaError_t b_sweeps_finish(const BTable* t, BOut* out, int K, BTune g, cudaStream_t s);
// Direct residual of every request's iterate (with_q: also q for refinement).
cudaError_t b_resid(const BTable* t, BOut* out, int with_q, BTune g, cudaStream_t s);
// Mixed precision: d = 0 (b_lp_zero); `inner` fused correction sweeps
// (b_lp_sweeps); pi <- (pi + d)/e^T(pi + d) with the step error (b_lp_finish).
cudaError_t b_lp_zero(const BTable* t, BTune g, cudaStream_t s);
cudaError_t b_lp_sweeps(const BTable* t, unsigned long long* t_claim, BOut* out, int bf16,
                        int coupled, int inner, BTune g, cudaStream_t s);
cudaError_t b_lp_finish(const BTable* t, BOut* out, BTune g, cudaStream_t s);

}  // namespace mc
