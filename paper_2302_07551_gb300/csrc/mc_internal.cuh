// Internal declarations shared by the libmc translation units.
//
// Workspace layout (all regions 256-byte aligned, offsets in bytes):
//   [hdr]      Header: status latch, last-block tickets, stats.
//   [planes]   n_planes planes; plane p holds L blocks, block l at
//              p*plane_bytes + l*ms*8, each block m x m doubles COLUMN-major
//              (entry (i, j) of the Q^T block at j*m + i), ms = m*m rounded up
//              to 32 doubles.  Column-major Q^T blocks are row-major Q blocks,
//              so the layout step is a plain copy.
//   [vectors]  z (sweep output before normalisation), xa, xb (iterate ping-pong
//              of mc_solve / mc_sweep), each N doubles rounded to 32.
//   [partials] per-warp level-sum partials of the two half-sweeps, per-block
//              step-error partials, per-warp residual partials.
//   [fused]    per-level sums of the last two sweeps and the queue / per-level
//              counters of the fused multi-sweep launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mc.h"

namespace mc {

constexpr int kMaxM = 256;
constexpr int kWarpsPerBlock = 8;          // sweep / residual kernels: 256 threads
constexpr int kMaxWarps = 8192;            // bound on the persistent sweep grid
constexpr int kMaxNormBlocks = 2048;
constexpr int kNormThreads = 256;

struct Header {
  int32_t status;        // first device-side error (mc_status), 0 = none
  uint32_t ticket[7];    // last-block-done counters (0 between launches): [0] normalise,
                         // [1] residual, [2] half-sweep 2, [3] low-precision update,
                         // [4] fused scale
  double stats[4];       // [e^T z, step_l1, resid_l1, spare]
};

// Off-staircase block diagonals |d| >= 2 of a block-banded Q^T (device
// resident in the workspace header region).
constexpr int kMaxFar = 8;
struct FarDesc {
  int32_t n;
  int32_t off[kMaxFar];           // d: the Q^T block (l, l + d)
  const double* plane[kMaxFar];   // L blocks, column-major, stride ms
};
constexpr size_t kFarDescOffset = 512;   // byte offset inside the 4 KB header

// Plane indices match mc_plane.
constexpr int kPlaneTLO = 0, kPlaneTUP = 1, kPlaneTDD = 2, kPlaneLU = 3, kPlaneNINV = 4,
              kPlaneWLO = 5, kPlaneWUP = 6;

struct Layout {
  int64_t L, N;
  int m, ms;             // block size and padded block stride (doubles)
  int n_planes;
  int nfar;              // off-staircase diagonals (block-banded chains)
  int far_off[kMaxFar];
  int far_base;          // plane index of the first far diagonal
  size_t plane_bytes, vec_bytes;
  size_t off_hdr, off_planes, off_z, off_xa, off_xb, off_wpart, off_dpart, off_rpart, total;
  // fused multi-sweep launches: per-level sums of the last two sweeps, the
  // per-level residual sums, the scales, queue counter + per-level completion
  // counters
  size_t off_fsum, off_fver;
  // low-precision storage (dtype MC_F32 / MC_BF16)
  int lp;                // 0: none, 1: FP32, 2: BF16
  int64_t lp_bs;         // elements per stored block of the A/B planes
  int64_t lp_cbs;        // floats per block of the FP32 (-T_dd)^{-1} plane
  size_t off_lpA, off_lpB, off_lpC, off_sc, off_q, off_d, off_bpart;
};

Layout make_layout(const mc_desc& d);

// Arguments of one half-sweep (Algorithm 2, step 1+2 or step 3).
struct PhaseArgs {
  const double* A;       // first operator plane (TLO, or WLO when coupled)
  const double* B;       // second operator plane (TUP, or WUP when coupled)
  const double* C;       // NINV plane (inverse mode), unused when coupled
  const double* src;     // vector read at neighbour levels l-1, l+1
  const double* src_up;  // if set: vector read at level l+1 instead (block Gauss-Seidel)
  const FarDesc* far;    // if set: off-staircase diagonals, read from xfar
  const double* xfar;    // the sweep's input x (far terms of both half-sweeps)
  double* dst;           // z, written at this half-sweep's levels
  double* wpart;         // one level-sum partial per warp
  Header* hdr;
  int64_t L, P;          // levels, levels in this half-sweep
  int m, ms;
  int parity;            // level of unit u is stride * u + parity
  int stride;            // 2: stair half-sweep, 1: all levels (block Jacobi)
  int reduce_s;          // last block sums the n_wpart partials into hdr->stats[0]
  int n_wpart;           // partials of both half-sweeps (reduce_s only)
};

// Several sweeps in one persistent launch (Algorithm 2 repeated K times):
// the units (sweep k, half-sweep h, level l) are claimed in that order from a
// queue counter; a unit waits until its two neighbour levels hold the values
// it reads (per-level completion counters), so no launch boundary or grid
// barrier separates half-sweeps or sweeps.  The sweeps are not normalised in
// between: z_{k+1} = M^{-1} N z_k, z_0 = x_in; e^T z of the last two sweeps is
// kept per level for the final normalisation.
struct FusedArgs {
  const double* A;       // TLO / WLO plane
  const double* B;       // TUP / WUP plane
  const double* C;       // NINV plane (inverse mode)
  const double* x_in;    // z_0 (read by the first half-sweep only)
  double* W;             // z_1 .. z_{K-1}, in place
  double* Z;             // z_K
  double* lsum;          // [2][L]: e^T of level l of sweep k in slot k & 1
  int* ver;              // [L]: completed writes of level l in this launch (zeroed before)
  unsigned long long* claim;   // queue position (zeroed before)
  Header* hdr;
  int64_t L, K;          // levels, sweeps
  int64_t P0;            // levels of half-sweep 1 (parity par0)
  int m, ms;
  int par0;              // 0: STAIR1, 1: STAIR2
  int paired;
  unsigned long long wait_ns;   // bound of one wait for a neighbour level
  // block-banded chains: off-staircase diagonals (NULL: block-tridiagonal) and
  // the band half-width bw = max |d|; the sweeps then alternate between W and
  // Z (sweep k writes W for even k, Z for odd k) instead of updating in place
  const FarDesc* far;
  int bw;
  // residual of z_K from the splitting (block-tridiagonal stair splittings):
  // with_resid adds P0 units after the K sweeps, one per diagonal-only level
  // l, each storing ||T_lo (z_K - z_{K-1})_{l-1} + T_up (z_K - z_{K-1})_{l+1}||_1
  // into rsum[(l - par0) / 2] (Q^T z_K = N (z_{K-1} - z_K) is zero on the
  // coupled rows).  RA, RB: the T_lo, T_up planes; prev: z_{K-1} (W, or x_in
  // when K = 1).
  int with_resid;
  // block Gauss-Seidel instead of a stair splitting (block-tridiagonal, not
  // paired): units in wavefront order, in place (k_bgs_cta)
  int bgs;
  const double* RA;
  const double* RB;
  const double* prev;
  double* rsum;
};

struct NormArgs {
  const double* r;       // NULL, or ||Q^T z||_1 (stats[2] = *r / e^T z)
  const double* z;
  const double* x_old;   // NULL: no step error (the previous iterate was not stored)
  const double* s_old;   // NULL: x_old is normalised; else x_old / *s_old is the iterate
  double* x_new;
  const double* s;       // e^T z (hdr->stats[0], written by half-sweep 2)
  double* dpart;         // one per block
  Header* hdr;
  double* stats_out;     // optional extra copy of [s, step, NaN]
  int64_t N;
};

struct ResidArgs {
  const double* TLO;
  const double* TDD;
  const double* TUP;
  const double* NINV;    // with q: (-T_dd)^{-1} plane
  float* q;              // optional output q = (-T_dd)^{-1} r (FP32)
  const double* x;
  double* rpart;         // one per warp
  Header* hdr;
  double* out;           // optional copy of the residual (device)
  int64_t L;
  int m, ms;
  int paired;
  const FarDesc* far;
};

// Launchers (return cudaGetLastError()).
cudaError_t launch_layout(const double* dn, const double* loc, const double* up, double* planes,
                          const Layout& lay, Header* hdr, cudaStream_t s);
// Q^T diagonal d into a plane: plane[l] = diag[l + d] (row-major Q block =
// column-major Q^T block), zero where l + d is outside [0, L).
cudaError_t launch_layout_diag(const double* diag, int d, double* plane, const Layout& lay,
                               cudaStream_t s);
cudaError_t launch_factor(double* planes, const Layout& lay, Header* hdr, int coupled,
                          int num_sms, cudaStream_t s);
cudaError_t launch_phase(const PhaseArgs& a, int coupled, int n_blocks, cudaStream_t s);
// Block Gauss-Seidel step: one warp walks the levels in order (z_{l-1} fresh,
// x_{l+1} old); e^T z into hdr->stats[0].
cudaError_t launch_bgs(const PhaseArgs& a, int coupled, cudaStream_t s);
int phase_blocks_per_sm(int m);   // resident 256-thread blocks of k_phase per SM
cudaError_t launch_normalise(const NormArgs& a, int n_blocks, cudaStream_t s);
cudaError_t launch_sweeps_fused(const FusedArgs& a, int coupled, int n_blocks, cudaStream_t s);
// One warp waits (at most wait_ns) for counters preset to `preset` to reach 1;
// MC_ERR_TIMEOUT is latched in hdr when they never do.
cudaError_t launch_wait_selftest(int preset, unsigned long long wait_ns, Header* hdr, int* ver,
                                 cudaStream_t s);
// out[0] = e^T z_K, out[1] = e^T z_{K-1} (1 when K = 1), out[2] = the sum of
// rsum[0..P) (NaN when rsum is NULL), fixed summation order; part:
// 3 kScaleBlocks doubles of scratch, ticket: a counter that is zero.
constexpr int kScaleBlocks = 64;
cudaError_t launch_fused_scale(const double* lsum, int64_t L, int64_t K, const double* rsum,
                               int64_t P, double* out, double* part, unsigned* ticket,
                               cudaStream_t s);
cudaError_t launch_residual(const ResidArgs& a, int n_blocks, cudaStream_t s);
cudaError_t launch_fill(double* x, int64_t n, double v, cudaStream_t s);
// Latch MC_ERR_ARG unless the paired zero quadrants of TLO / TUP are zero.
cudaError_t launch_check_paired(const double* tlo, const double* tup, const Layout& lay,
                                Header* hdr, cudaStream_t s);
cudaError_t launch_check_scale(const double* x0, double* x, int64_t n, Header* hdr,
                               double* dpart, cudaStream_t s);

cudaError_t launch_lp_convert(const double* src, void* dst, int bf16, float* sc, int sc_stride,
                              const Layout& lay, int64_t dbs, cudaStream_t s);
// All K correction sweeps of a refinement step in one launch (ver, claim:
// zeroed counters as for launch_sweeps_fused; parity of half-sweep 1); lpu:
// levels per claimed unit (1, 2 or 4); bps: resident blocks per SM (0: the
// kernel's occupancy).
cudaError_t launch_sweeps_lp(const void* A, const void* B, const float* C, const float* sc,
                             float* d, const float* q, int64_t L, int m, int parity, int64_t abs_,
                             int64_t cbs, int bf16, int coupled, int64_t K, int* ver,
                             unsigned long long* claim, Header* hdr, unsigned long long wait_ns,
                             int num_sms, int lpu, int bps, cudaStream_t s);
cudaError_t launch_update(const double* pi, const float* d, double* out, int64_t N, double* bpart,
                          int nb, Header* hdr, double* s_out, cudaStream_t s);

// Latch an error code into the header (first error wins).
__device__ __forceinline__ void latch(Header* h, int code) { atomicCAS(&h->status, 0, code); }

}  // namespace mc
