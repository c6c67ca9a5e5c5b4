// The chain handle (host memory) and the internal entry points shared by the
// C ABI (api.cu) and the solve server (server.cu).
#pragma once
#include "mc_internal.cuh"

struct mc_chain {
  mc_desc d;
  mc::Layout lay;
  char* ws;
  cudaStream_t user;         // caller's stream: every enqueue goes here
  cudaStream_t cap;          // private stream used only to capture graphs
  int num_sms;
  int factored;
  int nb_phase, nw;          // persistent sweep grid (blocks, warps)
  int nb_norm, nb_resid;
  mc::Header* hdr;           // device header inside the workspace
  mc::Header* hh;            // pinned host copy of the header
  double *planes, *z, *xa, *xb, *wpart, *dpart, *rpart;
  double* flsum;             // fused launches: [2][L] level sums, 2 scales, block partials
  int* fver;                 // [L] completion counters, after the queue counter
  unsigned long long* fclaim;
  int nb_fused;              // grid of the fused multi-sweep kernel
  int tune_bps;              // blocks per SM of the fused launches (0: default)
  int tune_lpu;              // levels per unit of the low-precision fused launches
  cudaGraphExec_t gexec;     // cached chunk graph of mc_solve
  int g_chunk, g_resid;
};

namespace mc {

// Validate desc and set up a handle on workspace ws (no GPU work).
int chain_init(const mc_desc* desc, void* workspace, size_t ws_bytes, cudaStream_t stream,
               mc_chain** out);
// Enqueue the factorisation (LU, inverse, optional coupled and low-precision
// operators) without waiting; errors are latched in the chain's header.
int chain_factor_async(mc_chain* c);
// Enqueue the direct residual of x (and q = (-T_dd)^{-1} r when q != NULL).
int chain_residual_async(mc_chain* c, const double* x, cudaStream_t s, float* q);
const void* chain_lpA(mc_chain* c);
const void* chain_lpB(mc_chain* c);
const float* chain_lpC(mc_chain* c);
const float* chain_lpSc(mc_chain* c);
float* chain_lpQ(mc_chain* c);
float* chain_lpD(mc_chain* c);

}  // namespace mc
