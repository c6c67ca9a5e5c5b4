// Batched (multi-request) sweep: descriptors shared by batch.cu and server.cu.
//
// All active requests of the solve server advance together: one fused
// persistent launch per block-size bucket covers every level of every
// request for all sweeps of a chunk (details below).  The request
// table lives in device memory and is rewritten by the host between chunks,
// so one captured CUDA graph serves any active set.  Requests are ordered
// small blocks first (m <= 128: rows per lane R <= 4) and large blocks after
// (m <= 256: R = 8); each bucket has its own kernel so that register use
// follows the bucket.  The low-precision kernels split the small bucket once
// more: m <= 64 (16-byte-load path, few registers, more resident warps) and
// 64 < m <= 128.
//
// Every reduction is per level first (one partial per level), then per
// request in level order: a request's iterates do not depend on which other
// requests share the launch, nor on the grid shape the autotuner picks.
//
// The sweeps of a chunk run fused (as the single-chain fused sweeps): one
// persistent launch per bucket for all sweeps of the chunk, units claimed in
// order, each waiting for its neighbour levels through the request's
// completion counters.  Counters grow across chunks: a chunk with epoch E
// writes E + k + 1 after its sweep k, so counters never need resetting (new
// requests start at zero <= E); the two claim counters live in the table and
// are reset by the table copy that starts every chunk.
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
  int64_t lp_bs, lp_cbs;
};

struct BTable {
  int32_t n;            // active requests
  int32_t n_small;      // requests [0, n_small) have m <= 128
  int32_t n_tiny;       // requests [0, n_tiny) have m <= 64 (low-precision kernels only)
  int32_t epoch;        // completion-counter base of this chunk
  unsigned long long claim[3];   // queue counters of the buckets of one chunk (0 in t_host)
  int64_t off_h1[kMaxReq + 1];   // prefix counts of half-sweep-1 levels
  int64_t off_h2[kMaxReq + 1];   // prefix counts of half-sweep-2 levels
  int64_t off_lv[kMaxReq + 1];   // prefix counts of all levels
  BReq r[kMaxReq];
};

struct BOut {
  double s, step, resid;
  double s_last, s_prev;   // fused FP64 chunk: e^T z of its last two sweeps (s_prev = 1 for one)
  int32_t status;
  int32_t pad;
};

struct BGrid {
  int blocks, threads;
};

// K FP64 sweeps of every request (fused, no normalisation in between), then
// e^T z, normalisation and the step error of the last sweep.  t_claim: the
// device table's claim counters.  coupled: server-wide apply mode.
cudaError_t b_sweeps(const BTable* t, unsigned long long* t_claim, BOut* out, int coupled, int K,
                     BGrid g, cudaStream_t s);
// Direct residual of every request's iterate (with_q: also q for refinement).
cudaError_t b_resid(const BTable* t, BOut* out, int with_q, BGrid g, cudaStream_t s);
// Mixed precision: d = 0; `inner` correction sweeps; pi <- (pi + d)/e^T(pi + d).
cudaError_t b_lp_step(const BTable* t, unsigned long long* t_claim, BOut* out, int bf16,
                      int coupled, int inner, BGrid g, cudaStream_t s);

}  // namespace mc
