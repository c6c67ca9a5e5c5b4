/*
 * mc.h -- C ABI of libmc: the block staircase stationary iteration for the
 * stationary vector of a Markov chain on one NVIDIA GB300 (sm_103a).
 *
 * Method (Besozzi, Della Bartola, Gemignani, arXiv 2302.07551):
 *   Eq. (1)      find pi with Q^T pi = 0, pi >= 0, e^T pi = 1 for an
 *                irreducible generator Q;
 *   Sect. 2      regular splitting Q^T = M - N with M a stair matrix;
 *   Eq. (2)      M x_{k+1} = N x_k, then x_{k+1} <- x_{k+1} / e^T x_{k+1};
 *   Algorithm 2  one sweep in two data-parallel steps over block rows;
 *   Sect. 3      stopping rule ||x_k - x_{k+1}||_1 <= eps or k >= maxit.
 *
 * Scope: block-tridiagonal Q^T (QBD-like generators) with L levels of m
 * phases each, N = L*m, and block-banded Q^T through mc_create_banded.
 * Level l (0-based) is block row l+1 of the paper.
 *
 * Conventions for every entry point
 *   - Device pointers are CUDA device addresses on the current device; all
 *     work is enqueued on the stream given to mc_create (NULL = legacy
 *     default stream).  Entry points marked "async" return before the GPU
 *     finishes; entry points marked "syncs" block on that stream.
 *   - The library never allocates device memory: the caller passes one
 *     workspace of at least mc_workspace_bytes() bytes, 256-byte aligned,
 *     which must outlive the handle.  The handle itself is host memory owned
 *     by the library (free it with mc_destroy).
 *   - Every call returns an mc_status; none aborts, traps or hangs.  Host
 *     side argument errors are reported before any GPU work.  Errors found
 *     on the device are latched into a status word in the workspace and are
 *     returned by the next syncing call (mc_factor, mc_solve, mc_residual,
 *     mc_sweep_host, mc_sync), which also clears the latch.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MC_OK = 0,
  MC_ERR_ARG = 1,             /* invalid argument (checked on the host)        */
  MC_ERR_WORKSPACE = 2,       /* workspace NULL, misaligned or too small       */
  MC_ERR_CUDA = 3,            /* a CUDA runtime call failed                    */
  MC_ERR_SINGULAR_BLOCK = 4,  /* a diagonal block has a zero/non-finite pivot  */
  MC_ERR_NOT_FACTORED = 5,    /* sweep/solve before a successful mc_factor     */
  MC_ERR_BREAKDOWN = 6,       /* e^T z <= 0 or not finite during normalisation */
  MC_ERR_NO_CONVERGENCE = 7,  /* mc_solve reached maxit                        */
  MC_ERR_TIMEOUT = 8          /* a bounded device-side wait gave up            */
} mc_status;

/*
 * Storage type of the blocks streamed by mc_solve's sweeps.
 *   MC_F64: plain FP64 staircase iteration of Eq. (2) (Algorithm 2).
 *   MC_F32, MC_BF16: mixed-precision iterative refinement (a library design,
 *     not in the paper): each outer step forms r = Q^T pi and
 *     q = (-T_dd)^{-1} r in FP64, runs check_every staircase sweeps of the
 *     correction equation Q^T d = -r (d <- M^{-1}(N d - r), Eq. (2) with a
 *     right-hand side) in FP32 arithmetic on blocks stored in FP32, or in BF16
 *     with one power-of-two scale per block, then updates
 *     pi <- (pi + d) / e^T(pi + d) in FP64.  (-T_dd)^{-1} is stored in FP32.
 *     Requires m % 4 == 0.  The FP64 blocks stay resident for the residual.
 */
typedef enum { MC_F64 = 0, MC_F32 = 1, MC_BF16 = 2 } mc_dtype;

/*
 * How the diagonal-block solves Q_{i,i}^{-1} of Algorithm 2 (steps 2 and 3)
 * are applied.  Both are computed from the LU factors of mc_factor and give
 * the same iterates up to rounding.
 *   MC_APPLY_INVERSE: store (-Q_{i,i})^{-1} (entrywise >= 0, Q^T being a
 *     singular M-matrix up to sign) and apply it as a dense product after
 *     the neighbour products: 3 m^2 FP64 multiply-adds and 24 m^2 bytes per
 *     level and sweep.
 *   MC_APPLY_COUPLED: store W_lo = (-Q_{i,i})^{-1} Q_{i,i-1} and
 *     W_up = (-Q_{i,i})^{-1} Q_{i,i+1} (both >= 0), so that each level is
 *     one product z_i = W_lo v_{i-1} + W_up v_{i+1}: 2 m^2 multiply-adds
 *     and 16 m^2 bytes per level and sweep.
 */
typedef enum { MC_APPLY_INVERSE = 0, MC_APPLY_COUPLED = 1 } mc_apply;

/* Planes of stored blocks, for mc_export. */
typedef enum {
  MC_PLANE_TLO = 0,   /* Q^T block (l, l-1)  = (Q_{l-1,l})^T; zero at l = 0     */
  MC_PLANE_TUP = 1,   /* Q^T block (l, l+1)  = (Q_{l+1,l})^T; zero at l = L-1   */
  MC_PLANE_TDD = 2,   /* Q^T block (l, l)    = (Q_{l,l})^T                      */
  MC_PLANE_LU = 3,    /* LU of TDD: unit L strictly below, U on/above diagonal  */
  MC_PLANE_NINV = 4,  /* (-TDD)^{-1}                                           */
  MC_PLANE_WLO = 5,   /* (-TDD)^{-1} TLO   (MC_APPLY_COUPLED only)                */
  MC_PLANE_WUP = 6    /* (-TDD)^{-1} TUP   (MC_APPLY_COUPLED only)                */
} mc_plane;

typedef struct {
  int64_t L;       /* number of levels (block rows), L >= 2                     */
  int32_t m;       /* phases per level (block size), 1 <= m <= 256              */
  int32_t stair;   /* 1: stair matrix of type 1 (default), 2: type 2 (Sect. 2);
                      3: block Jacobi, 4: block Gauss-Seidel (the comparison
                      splittings of Sect. 2; FP64, paired = 0).  Block
                      Gauss-Seidel on block-tridiagonal chains runs all sweeps
                      of a call in one launch in wavefront order (sweep k at
                      level l after sweep k at l-1 and sweep k-1 at l+1, up to
                      min(sweeps, L/2) levels at once); on block-banded chains
                      one warp walks the levels of one sweep at a time.         */
  int32_t apply;   /* mc_apply                                                  */
  int32_t dtype;   /* mc_dtype (MC_F32 / MC_BF16 need m % 4 == 0)               */
  int32_t paired;  /* 0, or 1: levels are pairs {2J, 2J+1} of a block-pentadiagonal
                      chain (jumps of +-1, +-2 levels), so the Q^T block (J, J-1) is
                      zero in rows m/2.. x columns ..m/2 and the block (J, J+1) in
                      rows ..m/2 x columns m/2..; the FP64 sweep and residual skip
                      those quadrants.  Needs m % 64 == 0; mc_factor checks that the
                      quadrants are zero (MC_ERR_ARG otherwise).                 */
  int32_t lower;   /* block bandwidths of the generator: Q_{l,l+e} may be nonzero */
  int32_t upper;   /* only for -lower <= e <= upper (0 means 1, block tridiagonal).
                      Wider bands (block Hessenberg / banded, up to 5 each side)
                      need mc_create_banded, apply = MC_APPLY_INVERSE, MC_F64 and
                      paired = 0; the sweeps then carry Algorithm 2's
                      off-staircase terms |k - i| >= 2, read from the sweep's
                      input vector.                                                 */
} mc_desc;

typedef struct {
  int64_t sweeps;       /* sweeps performed                                    */
  double residual_l1;   /* ||Q^T pi||_1 of the returned pi (direct, FP64)      */
  double step_l1;       /* ||x_k - x_{k-1}||_1 of the last sweep (Sect. 3)     */
  double contraction;   /* (step_k / step_{k-c})^(1/c) over the last check     */
  int32_t converged;    /* 1 if a stopping test other than maxit fired         */
} mc_result;

typedef struct mc_chain mc_chain;

/* Bytes of device workspace needed for desc (0 if desc is invalid). */
size_t mc_workspace_bytes(const mc_desc* desc);

/*
 * Create a chain from the generator blocks of Q (Eq. (1); the blocks Q_{i,j}
 * of Sect. 2 are the blocks of Q^T, formed here by transposition).
 *   dn, loc, up: device pointers to L blocks each of m x m doubles, row-major,
 *     contiguous ([L][m][m]): dn[l] = Q_{l,l-1}, loc[l] = Q_{l,l} (diagonal
 *     included), up[l] = Q_{l,l+1}.  dn[0] and up[L-1] are ignored.  8-byte
 *     aligned.  They are copied into the workspace during this call's stream
 *     work and may be freed once that work has completed.
 *   workspace, ws_bytes: caller-owned device memory (see conventions).
 *   cuda_stream: cudaStream_t on which all work of this handle is enqueued.
 *   out: receives the handle.
 * Async.  Errors: MC_ERR_ARG (bad desc, NULL pointers, misaligned blocks),
 * MC_ERR_WORKSPACE, MC_ERR_CUDA.
 */
int mc_create(const mc_desc* desc, const double* dn, const double* loc, const double* up,
              void* workspace, size_t ws_bytes, void* cuda_stream, mc_chain** out);

/*
 * As mc_create for a block-banded generator (desc->lower, desc->upper):
 * diags[e + lower], e = -lower..upper, are device pointers to L blocks of
 * m x m doubles, row-major, diags[e + lower][l] = Q_{l,l+e} (e = 0: the
 * diagonal blocks with their diagonal).  Blocks whose level l+e lies outside
 * [0, L) are ignored.  The Q^T block (l, l+d) is (Q_{l+d,l})^T (Sect. 2).
 * Async.  Errors as mc_create.
 */
int mc_create_banded(const mc_desc* desc, const double* const* diags, void* workspace,
                     size_t ws_bytes, void* cuda_stream, mc_chain** out);

/*
 * Factor the diagonal blocks Q_{i,i} (as blocks of Q^T) by batched LU without
 * pivoting (the blocks of a generator's transpose are strictly diagonally
 * dominant by columns, so no row exchange is ever needed) and form the
 * operators that apply Q_{i,i}^{-1} in Algorithm 2 steps 2 and 3 (see
 * mc_apply).  Syncs once.  Errors: MC_ERR_SINGULAR_BLOCK if a pivot is zero
 * or not finite (the handle stays unfactored), MC_ERR_CUDA.
 */
int mc_factor(mc_chain* chain);

/*
 * nsweeps sweeps of Eq. (2) with M the stair matrix of desc.stair, each as in
 * Algorithm 2: for the diagonal-only block rows (0-based even levels for
 * type 1) z_l = Q_{l,l}^{-1}(-Q_{l,l-1} x_{l-1} - Q_{l,l+1} x_{l+1}); then for
 * the coupled rows z_l = Q_{l,l}^{-1}(-Q_{l,l-1} z_{l-1} - Q_{l,l+1} z_{l+1});
 * then x <- z / e^T z and step = ||x_new - x_old||_1.
 *   x_in, x_out: device vectors of N doubles (x_in is not modified unless it
 *     equals x_out; in-place is allowed).  x_in should satisfy e^T x_in = 1
 *     for step to be the paper's step error.  (desc.stair 3 and 4 run block
 *     Jacobi and block Gauss-Seidel sweeps with the same interface.)
 *   nsweeps >= 1.
 *   stats_dev: NULL or device array of 3 doubles receiving, for the last
 *     sweep, [e^T z, ||x_new - x_old||_1, ||Q^T x_out||_1].  The residual
 *     (Eq. (1)) of a block-tridiagonal stair chain comes from the splitting:
 *     the last sweep solved M z = N x, so Q^T z = N (x - z), which is zero on
 *     the coupled block rows and T_lo d_{l-1} + T_up d_{l+1} (d = z - x) on
 *     the diagonal-only rows; it costs one pass over the two off-diagonal
 *     blocks of half the levels (a third of a sweep's bytes in inverse mode)
 *     at the end of the last fused launch.  Other chains (block-banded,
 *     block Jacobi / Gauss-Seidel) compute the direct residual.  With
 *     stats_dev == NULL no residual is formed.
 * Stair splittings (desc.stair 1 or 2, block-tridiagonal or banded) and block
 * Gauss-Seidel on block-tridiagonal chains run the nsweeps sweeps as one
 * persistent launch per 1024 sweeps, with no normalisation between the sweeps
 * of a launch (the scale of the iterate does not change the next one, Eq. (2)
 * up to rounding); x_out is normalised and stats refer to the last sweep as
 * above.  Block Jacobi (and banded block Gauss-Seidel) run one launch per
 * sweep.  Results are bitwise reproducible for equal calls and independent of
 * the launch configuration (mc_set_tuning); a run split into several calls
 * agrees up to rounding.
 * Async.  Errors: MC_ERR_ARG, MC_ERR_NOT_FACTORED, MC_ERR_CUDA; a breakdown
 * (e^T z <= 0 or not finite) is latched on the device (MC_ERR_BREAKDOWN);
 * MC_ERR_TIMEOUT if a bounded device-side wait of the fused launch gave up
 * (never expected: every wait is for work already claimed by a running warp).
 */
int mc_sweep(mc_chain* chain, const double* x_in, double* x_out, int64_t nsweeps,
             double* stats_dev);

/*
 * As mc_sweep but with HOST vectors (pinned memory recommended): returns the
 * result in x_out_host and the stats of mc_sweep (3 doubles, residual
 * included; NULL: no stats, and neither the residual nor the step error is
 * formed, so the input is not read a second time) in stats_host.  Stair chains
 * read a page-locked x_in_host (cudaHostAlloc / cudaHostRegister) in place
 * from the kernels over the CPU-GPU link, and when x_out_host is page-locked
 * and the sweeps run as one fused launch, the normalisation stores the
 * result into it directly; pageable buffers are copied.  x_in_host may equal
 * x_out_host.  Syncs.
 */
int mc_sweep_host(mc_chain* chain, const double* x_in_host, double* x_out_host, int64_t nsweeps,
                  double* stats_host);

/*
 * Self-test of the bounded device-side wait used between the units of a fused
 * sweep launch (no counterpart in the paper: it checks this library's
 * guarantee that a wait which can never be satisfied ends with an error
 * instead of hanging the GPU).  One warp waits for two completion counters
 * that are set (reachable != 0) or never set (reachable == 0), for at most
 * wait_ns nanoseconds (0 <= wait_ns <= 1e10).  Uses a small static device
 * buffer (not thread-safe across concurrent calls).  Syncs cuda_stream.
 * Returns MC_OK (reached) or MC_ERR_TIMEOUT (gave up), MC_ERR_ARG, MC_ERR_CUDA.
 */
int mc_wait_selftest(void* cuda_stream, int reachable, int64_t wait_ns);

/*
 * Diagnostics: for FP64 chains exactly mc_sweep(x_in, x_out, nsweeps, stats)
 * with the stats kept in the handle (block-tridiagonal stair chains form the
 * residual from the splitting at the end of the last fused launch, as one
 * chunk of mc_solve does);
 * for low-precision chains (MC_F32 / MC_BF16) the correction sweeps of one
 * refinement step from x_in (r and q of x_in, then nsweeps correction sweeps
 * from d = 0 in one fused launch; x_out = x_in).  CUDA events are recorded on
 * the handle's stream; ms_host (5 doubles, host) receives device times in
 * milliseconds and the number of kernel launches:
 *   fused sweeps (ms_host[4] = 1): [0] the fused sweep kernel(s) with their
 *     counter reset, [1] the reduction of e^T z, [2] the normalisation (both
 *     0 for low-precision chains), [3] launches;
 *   comparison splittings, desc.stair 3 or 4 (ms_host[4] = 0): [0] the
 *     sweeps, [1] 0, [2] the normalisations, summed over the sweeps,
 *     [3] launches.
 * 1 <= nsweeps <= 2^20.  Syncs.
 */
int mc_profile(mc_chain* chain, const double* x_in, double* x_out, int64_t nsweeps,
               double* ms_host);

/*
 * Solve Eq. (1) by iterating Eq. (2) (Algorithm 2 loop).
 *   x0: NULL (start from the uniform vector 1/N) or a device vector of N
 *     doubles, entries >= 0 with positive sum (normalised on entry).
 *   pi: device output, N doubles.
 *   tol: stop when ||Q^T pi||_1 <= tol, evaluated every check_every sweeps
 *     and at maxit; tol <= 0 disables.  Block-tridiagonal stair chains take
 *     the residual from the splitting inside the chunk's last fused launch
 *     (see mc_sweep) and confirm it with the direct FP64 residual before
 *     stopping (if the direct one is still above tol, rounding near the
 *     floor, the iteration continues); other chains evaluate the direct
 *     residual every check.  res->residual_l1 is always the direct residual
 *     of the returned pi.
 *   eps: stop when the step error of Sect. 3 is <= eps (evaluated every
 *     check_every sweeps); eps <= 0 disables.
 *   maxit: sweep limit (>= 1).  check_every >= 1: sweeps per check; the
 *     sweeps between checks run as one CUDA graph.
 *   res: receives the result (may be NULL).
 * Syncs once per check.  Errors: MC_ERR_ARG (bad sizes, x0 with a negative
 * entry or zero sum), MC_ERR_NOT_FACTORED, MC_ERR_BREAKDOWN,
 * MC_ERR_NO_CONVERGENCE (maxit reached with tol or eps enabled; pi and res
 * still hold the last iterate), MC_ERR_CUDA.
 */
int mc_solve(mc_chain* chain, const double* x0, double* pi, double tol, double eps, int64_t maxit,
             int32_t check_every, mc_result* res);

/*
 * ||Q^T pi||_1 (Eq. (1)) computed directly from the stored FP64 blocks.
 *   pi: device vector of N doubles.  resid_l1_host: host output.
 * Syncs.  Errors: MC_ERR_ARG, MC_ERR_CUDA.
 */
int mc_residual(mc_chain* chain, const double* pi, double* resid_l1_host);

/*
 * Copy count stored blocks of a plane, levels [level0, level0+count), to
 * dst_dev as count packed m x m blocks in COLUMN-major order (entry (i, j) of
 * a block of Q^T at j*m + i).  Async.  Errors: MC_ERR_ARG (range, plane not
 * stored for this desc.apply, LU/NINV/W* before mc_factor), MC_ERR_CUDA.
 */
int mc_export(mc_chain* chain, int32_t plane, int64_t level0, int64_t count, double* dst_dev);

/*
 * Direct residual ||Q^T pi||_1 for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a library service.  Code
 * running inside a CUDA graph capture, a serving loop whose device memory is
 * owned by another allocator or budget, or a plug-in that only holds device
 * pointers to someone else's data may be unable to call cudaMalloc or to
 * provide an mc_create workspace; this entry point needs neither and
 * allocates nothing.
 *   dn, loc, up: device generator blocks exactly as for mc_create
 *     ([L][m][m] doubles, row-major, 8-byte aligned).
 *   pi: device vector of N = L*m doubles.  resid_dev: device output (1 double).
 *   L: 2 <= L <= 65536 (larger L is rejected with MC_ERR_ARG: the library's
 *     scratch holds one partial sum per level).  m: 1 <= m <= 256.
 *   cuda_stream: stream for the work (NULL = legacy default stream).
 * Scratch: one static device array of 65536 doubles plus a counter (about
 * 512 KB), kept by every GPU that loads the library until the process exits.
 * All calls share it and a call leaves its contents behind, so calls whose
 * work overlaps on the GPU (other streams or threads) race: serialise them.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call outside any stream capture.
 * Async (the result is in resid_dev when the stream reaches it).
 * Errors: MC_ERR_ARG, MC_ERR_CUDA.
 */
int mc_residual_noalloc(const double* dn, const double* loc, const double* up, int64_t L,
                        int32_t m, const double* pi, double* resid_dev, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Solve server: continuous batching of many independent chains.  A library
 * service around the method (the paper solves one chain at a time).
 *
 * Requests (generator blocks as for mc_create, but in HOST memory) are
 * admitted into one caller-owned device arena while their workspace fits
 * (mc_server_request_bytes each) and at most max_active are running.  Each
 * mc_server_step runs check_every sweeps (dtype MC_F64) or one refinement
 * step of check_every correction sweeps (MC_F32 / MC_BF16) for ALL active
 * requests in shared fused persistent launches (one per block-size bucket
 * for all sweeps of the step), then every request's FP64 residual; requests with residual <= tol
 * (or a latched error, or maxit sweeps) are retired, their pi copied to host
 * memory and their arena memory freed.  Requests submitted between steps
 * join the next chunk.  A request's iterates are bitwise independent of the
 * other requests in the batch and of every launch configuration.  With
 * autotune = 1 the first chunks of every new batch signature time candidate
 * configurations (persistent grid, levels per claimed unit, block-size
 * bucketing, load depth) on the live requests and keep the fastest
 * (mc_server_trials lists the search).
 * --------------------------------------------------------------------------- */
typedef struct mc_server mc_server;

typedef struct {
  int32_t dtype;        /* mc_dtype of every request                           */
  int32_t apply;        /* mc_apply                                            */
  int32_t stair;        /* 1 or 2                                              */
  int32_t check_every;  /* sweeps per step (>= 1)                              */
  double tol;           /* retire when ||Q^T pi||_1 <= tol (tol <= 0: never)    */
  int64_t maxit;        /* retire (MC_ERR_NO_CONVERGENCE) after this many sweeps */
  int32_t max_active;   /* 1..1024 requests in flight                          */
  int32_t autotune;     /* 0 or 1                                              */
} mc_server_desc;

/*
 * arena: caller-owned device memory (256-byte aligned) holding the request
 * table and every admitted request; it must outlive the server.  Syncs no.
 * Errors: MC_ERR_ARG, MC_ERR_WORKSPACE (arena too small), MC_ERR_CUDA.
 */
int mc_server_create(const mc_server_desc* desc, void* arena, size_t arena_bytes,
                     void* cuda_stream, mc_server** out);

/* Arena bytes one request of L levels and block size m occupies (0 if invalid). */
size_t mc_server_request_bytes(const mc_server* server, int64_t L, int32_t m);

/*
 * Admit a request: dn, loc, up are HOST arrays of L blocks of m x m doubles
 * (row-major, as for mc_create), copied during the call.  tag identifies
 * the result.  Returns MC_OK, MC_ERR_WORKSPACE when the arena or the slot
 * count has no room now (retry after a step retires requests), MC_ERR_ARG,
 * MC_ERR_CUDA.  Low-precision servers need m % 4 == 0.  Start: uniform 1/N.
 */
int mc_server_submit(mc_server* server, int64_t tag, int64_t L, int32_t m, const double* dn,
                     const double* loc, const double* up);

/* One chunk for all active requests (syncs); returns active and finished counts. */
int mc_server_step(mc_server* server, int32_t* n_active, int32_t* n_done);

/*
 * Pop the oldest finished request: tag, pi (host, n_cap >= its N; pi_host may
 * be NULL to discard), result and status (MC_OK, MC_ERR_NO_CONVERGENCE,
 * MC_ERR_SINGULAR_BLOCK, MC_ERR_BREAKDOWN; MC_ERR_CUDA or MC_ERR_ARG when its
 * pi could not be copied out at retirement, and then pi_host is left as is).
 * MC_ERR_ARG when none is finished.
 */
int mc_server_fetch(mc_server* server, int64_t* tag, double* pi_host, int64_t n_cap,
                    mc_result* res, int32_t* status);

/* Launch grid in use and the number of tuned batch signatures. */
int mc_server_grid(const mc_server* server, int32_t* blocks, int32_t* threads,
                   int32_t* n_tuned);

/*
 * One timed chunk of the autotuner (autotune = 1).  For every new batch
 * signature the server times one live chunk per candidate configuration in a
 * coordinate search -- the persistent grid (1, 2, 3, 4, 6, 8 resident
 * 256-thread blocks per SM), then 2 and 4 levels per claimed unit (scaled up
 * for small blocks, see levels_per_unit below), then the
 * other block-size bucketing, then (low precision with blocks of m <= 64)
 * the other load depth -- and keeps the fastest.  The paper trades block
 * size against thread count by hand (Sect. 3); here the trade is measured on
 * the live request mix.
 */
typedef struct {
  uint64_t signature;       /* bit c set: requests of size class c present (m <= 32, 64,
                               128, 256); bits 8..: ceil(log2(total levels)) / 2      */
  int32_t blocks_per_sm;    /* resident 256-thread blocks per SM of the fused launches  */
  int32_t levels_per_unit;  /* adjacent same-parity levels per claimed unit (1, 2, 4)
                               for m > 64; x2 for m <= 64, x4 for m <= 32 (at most 16) */
  int32_t split64;          /* 1: blocks of m <= 64 in a launch of their own            */
  int32_t deep;             /* 1: 16 loads in flight per lane for low-precision m <= 64 */
  int32_t chosen;           /* 1: the configuration kept for this signature            */
  double chunk_ms;          /* the whole chunk (sweeps, reductions, residuals)         */
  double sweep_ms;          /* the fused sweep launches of the chunk (CUDA events)     */
  double sweep_bytes;       /* algorithmic bytes those launches stream                 */
} mc_server_tuning;

/* Copy up to cap timed chunks of the autotuner into out; *n = how many exist. */
int mc_server_trials(const mc_server* server, mc_server_tuning* out, int32_t cap, int32_t* n);

/* Release the server (requests still active are dropped). */
void mc_server_destroy(mc_server* server);

/*
 * Launch configuration of a chain's fused persistent launches: the trade
 * between block size and parallelism that the paper tunes by hand (Sect. 3),
 * chosen here by measurement.
 *   blocks_per_sm: resident 256-thread blocks per SM (0: all the kernel's
 *     occupancy allows, the default);
 *   levels_per_unit: adjacent same-parity levels per claimed work unit of the
 *     low-precision correction sweeps (1, 2 or 4; one claim, one neighbour
 *     wait and one completion fence per unit); FP64 sweeps use 1.
 * Neither changes any result: every level is computed the same way.
 */
typedef struct {
  int32_t blocks_per_sm;
  int32_t levels_per_unit;
} mc_tuning;

/* Set the configuration (MC_ERR_ARG for values outside the ranges above). */
int mc_set_tuning(mc_chain* chain, const mc_tuning* tuning);
int mc_get_tuning(const mc_chain* chain, mc_tuning* tuning);

/*
 * Autotune the chain: time nsweeps (1..1024) fused sweeps from the device
 * vector x (FP64 chains: stair or block Gauss-Seidel sweeps with their
 * residual units, blocks_per_sm in {0, 1, 2}; low-precision chains: the
 * correction sweeps of one refinement step from x, blocks_per_sm in
 * {0, 2, 3, 4} x levels_per_unit in {1, 2, 4}), each candidate once to warm up
 * and once timed with CUDA events, and keep the fastest.  x is only read;
 * the chain's scratch vectors are overwritten.  best, best_ms (may be NULL)
 * receive the choice and its time.  Syncs.  Errors: MC_ERR_ARG,
 * MC_ERR_NOT_FACTORED, MC_ERR_CUDA.
 */
int mc_tune(mc_chain* chain, const double* x, int64_t nsweeps, mc_tuning* best,
            double* best_ms);

/* Wait for the handle's stream and return (and clear) the device status. */
int mc_sync(mc_chain* chain);

/* Release the handle (host memory only; the workspace stays the caller's). */
void mc_destroy(mc_chain* chain);

/* Static description of a status code. */
const char* mc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* MC_H */
