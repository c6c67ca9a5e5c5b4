// Host side of the libmc C ABI (declarations and contracts in include/mc.h).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "chain.cuh"


namespace mc {

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static bool desc_ok(const mc_desc* d) {
  return d && d->L >= 2 && d->L <= (int64_t)1 << 31 && d->m >= 1 && d->m <= kMaxM &&
         (d->stair >= 1 && d->stair <= 4) &&
         (d->stair <= 2 || (d->dtype == MC_F64 && d->paired == 0)) &&
         (d->apply == MC_APPLY_INVERSE || d->apply == MC_APPLY_COUPLED) &&
         (d->dtype == MC_F64 || ((d->dtype == MC_F32 || d->dtype == MC_BF16) && d->m % 4 == 0)) &&
         (d->paired == 0 || (d->paired == 1 && d->m % 64 == 0)) &&
         d->lower >= 0 && d->lower <= 5 && d->upper >= 0 && d->upper <= 5 &&
         ((d->lower <= 1 && d->upper <= 1) ||
          (d->apply == MC_APPLY_INVERSE && d->dtype == MC_F64 && d->paired == 0));
}

Layout make_layout(const mc_desc& d) {
  Layout y{};
  y.L = d.L;
  y.m = d.m;
  y.N = d.L * d.m;
  y.ms = (int)round_up((size_t)d.m * d.m, 32);
  y.n_planes = d.apply == MC_APPLY_COUPLED ? 7 : 5;
  // off-staircase diagonals of Q^T: offsets -upper..-2 and 2..lower (the
  // Q^T block (l, l+d) is (Q_{l+d,l})^T, so Q's upper band is Q^T's lower)
  const int lo = d.lower > 1 ? d.lower : 1, up = d.upper > 1 ? d.upper : 1;
  y.nfar = 0;
  y.far_base = y.n_planes;
  for (int o = -up; o <= -2; ++o) y.far_off[y.nfar++] = o;
  for (int o = 2; o <= lo; ++o) y.far_off[y.nfar++] = o;
  y.n_planes += y.nfar;
  y.plane_bytes = (size_t)d.L * y.ms * sizeof(double);
  y.vec_bytes = round_up((size_t)y.N, 32) * sizeof(double);
  size_t o = 0;
  y.off_hdr = o;
  o += 4096;
  y.off_planes = o;
  o += y.plane_bytes * y.n_planes;
  y.off_z = o;
  o += y.vec_bytes;
  y.off_xa = o;
  o += y.vec_bytes;
  y.off_xb = o;
  o += y.vec_bytes;
  y.off_wpart = o;
  o += round_up(2 * kMaxWarps * sizeof(double), 256);
  y.off_dpart = o;
  o += round_up(kMaxNormBlocks * sizeof(double), 256);
  y.off_rpart = o;
  o += round_up(kMaxWarps * sizeof(double), 256);
  y.off_fsum = o;
  // [2][L] level sums of e^T z, [L] residual sums, 4 scale slots, partials
  o += round_up((3 * (size_t)d.L + 4 + 3 * kScaleBlocks) * sizeof(double), 256);
  y.off_fver = o;
  o += round_up(sizeof(unsigned long long) + (size_t)d.L * sizeof(int), 256);
  y.lp = d.dtype == MC_F32 ? 1 : d.dtype == MC_BF16 ? 2 : 0;
  if (y.lp) {
    const size_t es = y.lp == 1 ? 4 : 2;
    const size_t mm = (size_t)d.m * d.m;
    y.lp_bs = (int64_t)(round_up(mm * es, 256) / es);
    y.lp_cbs = (int64_t)(round_up(mm * 4, 256) / 4);
    y.off_lpA = o;
    o += round_up((size_t)d.L * y.lp_bs * es, 256);
    y.off_lpB = o;
    o += round_up((size_t)d.L * y.lp_bs * es, 256);
    y.off_lpC = o;
    if (d.apply == MC_APPLY_INVERSE) o += round_up((size_t)d.L * y.lp_cbs * 4, 256);
    y.off_sc = o;
    o += round_up((size_t)d.L * 2 * sizeof(float), 256);
    y.off_q = o;
    o += round_up((size_t)y.N * 4, 256);
    y.off_d = o;
    o += round_up((size_t)y.N * 4, 256);
    y.off_bpart = o;
    o += round_up(kMaxNormBlocks * sizeof(double), 256);
  }
  y.total = o;
  return y;
}

}  // namespace mc

using namespace mc;

#define CK(call)                                   \
  do {                                             \
    if ((call) != cudaSuccess) return MC_ERR_CUDA; \
  } while (0)

// One sweep of a comparison splitting of Sect. 2 (the stair splittings run
// fused): block Jacobi (every level from x, one launch) or block Gauss-Seidel
// (levels in order, one warp), then the normalisation into dst with the step
// error.  ev (optional) = 4 events recorded before the sweep, twice after it,
// and after the normalisation.
static int enqueue_sweep(mc_chain* c, const double* src, double* dst, double* stats_out,
                         cudaStream_t s, cudaEvent_t* ev = nullptr) {
  const bool coupled = c->d.apply == MC_APPLY_COUPLED;
  const size_t pe = c->lay.plane_bytes / sizeof(double);
  PhaseArgs a{};
  a.A = c->planes + (coupled ? kPlaneWLO : kPlaneTLO) * pe;
  a.B = c->planes + (coupled ? kPlaneWUP : kPlaneTUP) * pe;
  a.C = c->planes + kPlaneNINV * pe;
  a.L = c->lay.L;
  a.m = c->lay.m;
  a.ms = c->lay.ms;
  a.far = c->lay.nfar ? (const FarDesc*)((const char*)c->hdr + kFarDescOffset) : nullptr;
  a.xfar = src;
  a.src = src;
  a.src_up = src;
  a.dst = c->z;
  a.wpart = c->wpart;
  a.hdr = c->hdr;
  a.parity = 0;
  a.stride = 1;
  a.P = c->lay.L;
  a.reduce_s = 1;
  a.n_wpart = c->nw;
  if (ev) CK(cudaEventRecord(ev[0], s));
  if (c->d.stair == 3) {
    CK(launch_phase(a, coupled, c->nb_phase, s));
  } else {
    CK(launch_bgs(a, coupled, s));
  }
  if (ev) CK(cudaEventRecord(ev[1], s));
  if (ev) CK(cudaEventRecord(ev[2], s));
  NormArgs n{};
  n.z = c->z;
  n.x_old = src;
  n.x_new = dst;
  n.s = &c->hdr->stats[0];
  n.dpart = c->dpart;
  n.hdr = c->hdr;
  n.stats_out = stats_out;
  n.N = c->lay.N;
  CK(launch_normalise(n, c->nb_norm, s));
  if (ev) CK(cudaEventRecord(ev[3], s));
  return MC_OK;
}

// Sweeps per fused launch: bounds the launch and keeps the unnormalised
// iterates of one launch far from the FP64 range limits.
constexpr int64_t kMaxFusedSweeps = 1024;
// Bound of one wait for a neighbour level in a fused launch.  A wait is for a
// unit that a running warp has already claimed, normally well under a
// millisecond even at m = 256; two seconds only catches a broken invariant.
constexpr unsigned long long kFusedWaitNs = 2000000000ull;

// Stair splittings run fused (block-tridiagonal in place, block-banded with
// alternating buffers), and so does block Gauss-Seidel on block-tridiagonal
// chains (wavefront order); block Jacobi and banded block Gauss-Seidel one
// sweep at a time.
static bool fused_ok(const mc_chain* c) {
  return c->d.stair <= 2 || (c->d.stair == 4 && c->lay.nfar == 0 && !c->d.paired);
}

// Block-tridiagonal stair splittings get the residual of a fused launch's
// result from the splitting (residual units at the end of the launch); other
// chains use the direct residual.
static bool split_resid_ok(const mc_chain* c) { return c->d.stair <= 2 && c->lay.nfar == 0; }

// n stair sweeps src -> dst (in place allowed) as fused launches of at most
// kMaxFusedSweeps sweeps, each followed by the normalisation (with the step
// error after the last).  With resid (block-tridiagonal chains only) the last
// launch also forms ||Q^T dst||_1 from the splitting into stats[2].  ev
// (optional, 4 events): before the first launch, after the last fused kernel,
// after its scale reduction, after the last normalisation.
static int enqueue_sweeps_fused(mc_chain* c, const double* src, double* dst, int64_t n,
                                double* stats_out, cudaStream_t s, cudaEvent_t* ev,
                                bool resid, bool step) {
  const bool coupled = c->d.apply == MC_APPLY_COUPLED;
  const size_t pe = c->lay.plane_bytes / sizeof(double);
  const int64_t L = c->lay.L;
  const size_t cnt_bytes = sizeof(unsigned long long) + (size_t)L * sizeof(int);
  double* rsum = c->flsum + 2 * L;
  double* scale = c->flsum + 3 * L;
  const bool banded = c->lay.nfar > 0;
  int bw = 1;
  for (int i = 0; i < c->lay.nfar; ++i) {
    const int o = c->lay.far_off[i] < 0 ? -c->lay.far_off[i] : c->lay.far_off[i];
    if (o > bw) bw = o;
  }
  if (ev) CK(cudaEventRecord(ev[0], s));
  const double* in = src;
  for (int64_t done = 0; done < n;) {
    const int64_t K = n - done < kMaxFusedSweeps ? n - done : kMaxFusedSweeps;
    const bool final = done + K == n;
    FusedArgs a{};
    a.A = c->planes + (coupled ? kPlaneWLO : kPlaneTLO) * pe;
    a.B = c->planes + (coupled ? kPlaneWUP : kPlaneTUP) * pe;
    a.C = c->planes + kPlaneNINV * pe;
    a.x_in = in;
    a.W = c->xb;
    a.Z = c->z;
    a.lsum = c->flsum;
    a.ver = c->fver;
    a.claim = c->fclaim;
    a.hdr = c->hdr;
    a.L = L;
    a.K = K;
    a.par0 = c->d.stair == 1 ? 0 : 1;
    a.P0 = (L - a.par0 + 1) / 2;
    a.m = c->lay.m;
    a.ms = c->lay.ms;
    a.paired = c->d.paired && !coupled;
    a.wait_ns = kFusedWaitNs;
    a.far = banded ? (const FarDesc*)((const char*)c->hdr + kFarDescOffset) : nullptr;
    a.bw = bw;
    a.bgs = c->d.stair == 4;
    const bool with_resid = resid && final && !banded && !a.bgs;
    if (with_resid) {
      a.with_resid = 1;
      a.RA = c->planes + kPlaneTLO * pe;
      a.RB = c->planes + kPlaneTUP * pe;
      a.prev = K == 1 ? in : c->xb;
      a.rsum = rsum;
    }
    // block Gauss-Seidel runs at most min(K, L/2) units at once (one per sweep
    // in flight), one block per unit; the launcher caps the grid at the blocks
    // resident at once
    int nb = c->nb_fused;
    if (a.bgs) {
      const int64_t par = K < (L + 1) / 2 ? K : (L + 1) / 2;
      nb = par < (1 << 30) ? (int)par : (1 << 30);
    }
    if (c->tune_bps > 0 && c->tune_bps * c->num_sms < nb) nb = c->tune_bps * c->num_sms;
    CK(cudaMemsetAsync(c->fclaim, 0, cnt_bytes, s));
    CK(launch_sweeps_fused(a, coupled, nb, s));
    if (ev && final) CK(cudaEventRecord(ev[1], s));
    CK(launch_fused_scale(c->flsum, L, K, with_resid ? rsum : nullptr, a.P0, scale, scale + 4,
                          &c->hdr->ticket[4], s));
    if (ev && final) CK(cudaEventRecord(ev[2], s));
    NormArgs nn{};
    nn.r = with_resid ? scale + 2 : nullptr;
    // step error of the last sweep: z_K / s_K against z_{K-1} / s_{K-1}
    // (block-tridiagonal: z_K in Z, z_{K-1} in W; block-banded: z_k in W for
    // odd k, in Z for even k >= 2)
    const double* last = banded ? ((K & 1) ? c->xb : c->z) : c->z;
    const double* prev = banded ? ((K & 1) ? c->z : c->xb) : c->xb;
    nn.z = last;
    nn.x_old = (final && step) ? (K == 1 ? in : prev) : nullptr;
    nn.s_old = scale + 1;
    nn.x_new = dst;
    nn.s = scale;
    nn.dpart = c->dpart;
    nn.hdr = c->hdr;
    nn.stats_out = final ? stats_out : nullptr;
    nn.N = c->lay.N;
    CK(launch_normalise(nn, c->nb_norm, s));
    in = dst;
    done += K;
  }
  if (ev) CK(cudaEventRecord(ev[3], s));
  return MC_OK;
}

// nsweeps sweeps src -> dst (in place allowed).  Stair splittings run as
// fused launches; the comparison splittings one sweep at a time, each
// normalised.  resid: form ||Q^T dst||_1 from the splitting (stats[2]) where
// split_resid_ok.  step = false: a fused call skips the step error of its
// last sweep (stats[1] = 0) and never reads the previous iterate again.
static int enqueue_sweeps(mc_chain* c, const double* src, double* dst, int64_t n,
                          double* stats_out, cudaStream_t s, cudaEvent_t* ev = nullptr,
                          bool resid = false, bool step = true) {
  if (fused_ok(c)) return enqueue_sweeps_fused(c, src, dst, n, stats_out, s, ev, resid, step);
  for (int64_t k = 0; k < n; ++k) {
    const int rc = enqueue_sweep(c, k == 0 ? src : dst, dst, k == n - 1 ? stats_out : nullptr, s,
                                 ev ? ev + 4 * k : nullptr);
    if (rc != MC_OK) return rc;
  }
  return MC_OK;
}

static int enqueue_residual(mc_chain* c, const double* x, cudaStream_t s, float* q = nullptr,
                            double* out = nullptr) {
  const size_t pe = c->lay.plane_bytes / sizeof(double);
  ResidArgs r{};
  r.TLO = c->planes + kPlaneTLO * pe;
  r.TDD = c->planes + kPlaneTDD * pe;
  r.TUP = c->planes + kPlaneTUP * pe;
  r.NINV = c->planes + kPlaneNINV * pe;
  r.q = q;
  r.x = x;
  r.rpart = c->rpart;
  r.hdr = c->hdr;
  r.out = out;
  r.L = c->lay.L;
  r.m = c->lay.m;
  r.ms = c->lay.ms;
  r.paired = c->d.paired;
  r.far = c->lay.nfar ? (const FarDesc*)((const char*)c->hdr + kFarDescOffset) : nullptr;
  CK(launch_residual(r, c->nb_resid, s));
  return MC_OK;
}

// ---- mixed-precision refinement (dtype MC_F32 / MC_BF16) -------------------------
static const void* lpA(mc_chain* c) { return c->ws + c->lay.off_lpA; }
static const void* lpB(mc_chain* c) { return c->ws + c->lay.off_lpB; }
static const float* lpC(mc_chain* c) { return (const float*)(c->ws + c->lay.off_lpC); }
static float* lpSc(mc_chain* c) { return (float*)(c->ws + c->lay.off_sc); }
static float* lpQ(mc_chain* c) { return (float*)(c->ws + c->lay.off_q); }
static float* lpD(mc_chain* c) { return (float*)(c->ws + c->lay.off_d); }

// One correction sweep d <- M^{-1}(N d - r) in low precision (two launches).
// One outer step on the iterate xa: `inner` correction sweeps from d = 0 (q
// must hold (-T_dd)^{-1} r for the current xa), pi <- (pi + d)/e^T(pi + d)
// with the step error, then r and q of the new iterate.
static int enqueue_lp_sweeps_fused(mc_chain* c, int64_t K, cudaStream_t s) {
  const size_t cnt_bytes = sizeof(unsigned long long) + (size_t)c->lay.L * sizeof(int);
  CK(cudaMemsetAsync(c->fclaim, 0, cnt_bytes, s));
  CK(launch_sweeps_lp(lpA(c), lpB(c), lpC(c), lpSc(c), lpD(c), lpQ(c), c->lay.L, c->lay.m,
                      c->d.stair == 1 ? 0 : 1, c->lay.lp_bs, c->lay.lp_cbs, c->lay.lp == 2,
                      c->d.apply == MC_APPLY_COUPLED, K, c->fver, c->fclaim, c->hdr, kFusedWaitNs,
                      c->num_sms, c->tune_lpu, c->tune_bps, s));
  return MC_OK;
}

static int enqueue_refine_step(mc_chain* c, int inner, cudaStream_t s) {
  CK(cudaMemsetAsync(lpD(c), 0, (size_t)c->lay.N * sizeof(float), s));
  const int rc = enqueue_lp_sweeps_fused(c, inner, s);
  if (rc != MC_OK) return rc;
  double* bpart = (double*)(c->ws + c->lay.off_bpart);
  CK(launch_update(c->xa, lpD(c), c->xb, c->lay.N, bpart, c->nb_norm, c->hdr, &c->hdr->stats[0],
                   s));
  NormArgs n{};
  n.z = c->xb;
  n.x_old = c->xa;
  n.x_new = c->xa;
  n.s = &c->hdr->stats[0];
  n.dpart = c->dpart;
  n.hdr = c->hdr;
  n.stats_out = nullptr;
  n.N = c->lay.N;
  CK(launch_normalise(n, c->nb_norm, s));
  return enqueue_residual(c, c->xa, s, lpQ(c));
}

int mc::chain_residual_async(mc_chain* c, const double* x, cudaStream_t s, float* q) {
  return enqueue_residual(c, x, s, q);
}
const void* mc::chain_lpA(mc_chain* c) { return lpA(c); }
const void* mc::chain_lpB(mc_chain* c) { return lpB(c); }
const float* mc::chain_lpC(mc_chain* c) { return lpC(c); }
const float* mc::chain_lpSc(mc_chain* c) { return lpSc(c); }
float* mc::chain_lpQ(mc_chain* c) { return lpQ(c); }
float* mc::chain_lpD(mc_chain* c) { return lpD(c); }

// Wait for the stream, fetch the header, clear a latched status.
static int sync_header(mc_chain* c) {
  CK(cudaMemcpyAsync(c->hh, c->hdr, sizeof(Header), cudaMemcpyDeviceToHost, c->user));
  CK(cudaStreamSynchronize(c->user));
  const int st = c->hh->status;
  if (st != 0) {
    CK(cudaMemsetAsync(&c->hdr->status, 0, sizeof(int32_t), c->user));
    CK(cudaStreamSynchronize(c->user));
  }
  return st;
}

int mc::chain_init(const mc_desc* desc, void* workspace, size_t ws_bytes, cudaStream_t stream,
                   mc_chain** out) {
  if (!out) return MC_ERR_ARG;
  *out = nullptr;
  if (!desc_ok(desc)) return MC_ERR_ARG;
  const Layout lay = make_layout(*desc);
  if (!workspace || ((uintptr_t)workspace & 255u) || ws_bytes < lay.total) return MC_ERR_WORKSPACE;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  mc_chain* c = new (std::nothrow) mc_chain();
  if (!c) return MC_ERR_ARG;
  c->d = *desc;
  c->lay = lay;
  c->ws = (char*)workspace;
  c->user = stream;
  c->num_sms = sms;
  c->hdr = (Header*)(c->ws + lay.off_hdr);
  c->planes = (double*)(c->ws + lay.off_planes);
  c->z = (double*)(c->ws + lay.off_z);
  c->xa = (double*)(c->ws + lay.off_xa);
  c->xb = (double*)(c->ws + lay.off_xb);
  c->wpart = (double*)(c->ws + lay.off_wpart);
  c->dpart = (double*)(c->ws + lay.off_dpart);
  c->rpart = (double*)(c->ws + lay.off_rpart);
  c->flsum = (double*)(c->ws + lay.off_fsum);
  c->fclaim = (unsigned long long*)(c->ws + lay.off_fver);
  c->fver = (int*)(c->ws + lay.off_fver + sizeof(unsigned long long));
  // persistent grids: the full resident grid of the kernel's occupancy (a
  // multiple of the SM count) once there is at least one unit per SM, else one
  // warp per unit
  const int64_t pmax = (lay.L + 1) / 2;
  const int64_t wps = (int64_t)kWarpsPerBlock * phase_blocks_per_sm(lay.m);
  int64_t w = wps * sms;
  if (pmax < sms) w = pmax;
  if (w > kMaxWarps) w = kMaxWarps;
  c->nb_phase = (int)((w + kWarpsPerBlock - 1) / kWarpsPerBlock);
  c->nw = c->nb_phase * kWarpsPerBlock;
  int64_t wr = wps * sms;
  if (lay.L < sms) wr = lay.L;
  if (wr > kMaxWarps) wr = kMaxWarps;
  c->nb_resid = (int)((wr + kWarpsPerBlock - 1) / kWarpsPerBlock);
  // fused launches claim units dynamically: the full resident grid, but no
  // more warps than levels
  int64_t wf = wps * sms;
  if (wf > lay.L) wf = lay.L;
  c->nb_fused = (int)((wf + kWarpsPerBlock - 1) / kWarpsPerBlock);
  c->tune_bps = 0;
  c->tune_lpu = 1;
  int64_t nbn = (lay.N + 4 * kNormThreads - 1) / (4 * kNormThreads);
  if (nbn > 8 * sms) nbn = 8 * sms;
  if (nbn > kMaxNormBlocks) nbn = kMaxNormBlocks;
  c->nb_norm = (int)(nbn < 1 ? 1 : nbn);
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return MC_ERR_CUDA;
  }
  if (cudaHostAlloc((void**)&c->hh, sizeof(Header), cudaHostAllocDefault) != cudaSuccess) {
    cudaStreamDestroy(c->cap);
    delete c;
    return MC_ERR_CUDA;
  }
  memset(c->hh, 0, sizeof(Header));
  int rc = MC_OK;
  if (cudaMemsetAsync(c->ws + lay.off_hdr, 0, 4096, c->user) != cudaSuccess) rc = MC_ERR_CUDA;
  if (rc != MC_OK) {
    mc_destroy(c);
    return rc;
  }
  *out = c;
  return MC_OK;
}


extern "C" {

size_t mc_workspace_bytes(const mc_desc* desc) {
  if (!desc_ok(desc)) return 0;
  return make_layout(*desc).total;
}

int mc_create(const mc_desc* desc, const double* dn, const double* loc, const double* up,
              void* workspace, size_t ws_bytes, void* cuda_stream, mc_chain** out) {
  if (!out) return MC_ERR_ARG;
  *out = nullptr;
  if (!desc_ok(desc) || !dn || !loc || !up) return MC_ERR_ARG;
  if (desc->lower > 1 || desc->upper > 1) return MC_ERR_ARG;
  if (((uintptr_t)dn | (uintptr_t)loc | (uintptr_t)up) & 7u) return MC_ERR_ARG;
  mc_chain* c = nullptr;
  const int rc = chain_init(desc, workspace, ws_bytes, (cudaStream_t)cuda_stream, &c);
  if (rc != MC_OK) return rc;
  if (launch_layout(dn, loc, up, c->planes, c->lay, c->hdr, c->user) != cudaSuccess) {
    mc_destroy(c);
    return MC_ERR_CUDA;
  }
  *out = c;
  return MC_OK;
}

int mc_create_banded(const mc_desc* desc, const double* const* diags, void* workspace,
                     size_t ws_bytes, void* cuda_stream, mc_chain** out) {
  if (!out) return MC_ERR_ARG;
  *out = nullptr;
  if (!desc_ok(desc) || !diags) return MC_ERR_ARG;
  const int lo = desc->lower > 1 ? desc->lower : 1, up = desc->upper > 1 ? desc->upper : 1;
  for (int e = -lo; e <= up; ++e)
    if (!diags[e + lo] || ((uintptr_t)diags[e + lo] & 7u)) return MC_ERR_ARG;
  mc_chain* c = nullptr;
  int rc = chain_init(desc, workspace, ws_bytes, (cudaStream_t)cuda_stream, &c);
  if (rc != MC_OK) return rc;
  const Layout& y = c->lay;
  const size_t pe = y.plane_bytes / sizeof(double);
  // near diagonals as in mc_create: Q^T (l, l-1) <- Q_{l-1,l} (e = +1),
  // (l, l+1) <- Q_{l+1,l} (e = -1), (l, l) <- Q_{l,l}
  if (launch_layout(diags[lo - 1], diags[lo], diags[lo + 1], c->planes, y, c->hdr, c->user) !=
      cudaSuccess)
    rc = MC_ERR_CUDA;
  FarDesc fd{};
  fd.n = y.nfar;
  for (int j = 0; j < y.nfar && rc == MC_OK; ++j) {
    const int d = y.far_off[j];
    double* plane = c->planes + (size_t)(y.far_base + j) * pe;
    fd.off[j] = d;
    fd.plane[j] = plane;
    if (launch_layout_diag(diags[-d + lo], d, plane, y, c->user) != cudaSuccess) rc = MC_ERR_CUDA;
  }
  if (rc == MC_OK && cudaMemcpyAsync((char*)c->hdr + kFarDescOffset, &fd, sizeof(fd),
                                     cudaMemcpyHostToDevice, c->user) != cudaSuccess)
    rc = MC_ERR_CUDA;
  if (rc == MC_OK && cudaStreamSynchronize(c->user) != cudaSuccess) rc = MC_ERR_CUDA;
  if (rc != MC_OK) {
    mc_destroy(c);
    return rc;
  }
  *out = c;
  return MC_OK;
}

int mc_factor(mc_chain* c) {
  if (!c) return MC_ERR_ARG;
  const int rc = chain_factor_async(c);
  if (rc != MC_OK) return rc;
  const int st = sync_header(c);
  if (st != MC_OK) return st;
  c->factored = 1;
  return MC_OK;
}

}  // extern "C"

int mc::chain_factor_async(mc_chain* c) {
  c->factored = 0;
  if (c->d.paired) {
    const size_t pe = c->lay.plane_bytes / sizeof(double);
    CK(launch_check_paired(c->planes + kPlaneTLO * pe, c->planes + kPlaneTUP * pe, c->lay, c->hdr,
                           c->user));
  }
  CK(launch_factor(c->planes, c->lay, c->hdr, c->d.apply == MC_APPLY_COUPLED, c->num_sms,
                   c->user));
  if (c->lay.lp) {
    const size_t pe = c->lay.plane_bytes / sizeof(double);
    const int bf16 = c->lay.lp == 2;
    const bool coupled = c->d.apply == MC_APPLY_COUPLED;
    CK(launch_lp_convert(c->planes + (coupled ? kPlaneWLO : kPlaneTLO) * pe, c->ws + c->lay.off_lpA,
                         bf16, lpSc(c), 2, c->lay, c->lay.lp_bs, c->user));
    CK(launch_lp_convert(c->planes + (coupled ? kPlaneWUP : kPlaneTUP) * pe, c->ws + c->lay.off_lpB,
                         bf16, lpSc(c) + 1, 2, c->lay, c->lay.lp_bs, c->user));
    if (!coupled)
      CK(launch_lp_convert(c->planes + kPlaneNINV * pe, c->ws + c->lay.off_lpC, 0, nullptr, 0,
                           c->lay, c->lay.lp_cbs, c->user));
  }
  return MC_OK;
}

extern "C" {

int mc_sweep(mc_chain* c, const double* x_in, double* x_out, int64_t nsweeps, double* stats_dev) {
  if (!c || !x_in || !x_out || nsweeps < 1) return MC_ERR_ARG;
  if (((uintptr_t)x_in | (uintptr_t)x_out) & 7u) return MC_ERR_ARG;
  if (!c->factored) return MC_ERR_NOT_FACTORED;
  const bool split = split_resid_ok(c);
  const int rc = enqueue_sweeps(c, x_in, x_out, nsweeps, stats_dev, c->user, nullptr,
                                stats_dev != nullptr && split);
  if (rc != MC_OK || !stats_dev || split) return rc;
  return enqueue_residual(c, x_out, c->user, nullptr, stats_dev + 2);
}

int mc_profile(mc_chain* c, const double* x_in, double* x_out, int64_t nsweeps, double* ms_host) {
  if (!c || !x_in || !x_out || !ms_host || nsweeps < 1 || nsweeps > (1 << 20)) return MC_ERR_ARG;
  if (((uintptr_t)x_in | (uintptr_t)x_out) & 7u) return MC_ERR_ARG;
  if (!c->factored) return MC_ERR_NOT_FACTORED;
  // low-precision chains: the correction sweeps of refinement, always fused
  const bool fused = c->lay.lp || fused_ok(c);
  const size_t ne = fused ? 4 : 4 * (size_t)nsweeps;
  cudaEvent_t* ev = (cudaEvent_t*)calloc(ne, sizeof(cudaEvent_t));
  if (!ev) return MC_ERR_ARG;
  int rc = MC_OK;
  size_t made = 0;
  for (; made < ne; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) { rc = MC_ERR_CUDA; break; }
  if (c->lay.lp) {
    // low-precision chains: time the correction sweeps of refinement, with
    // r and q of x_in (the FP64 x_out is left equal to x_in)
    if (cudaMemcpyAsync(c->xa, x_in, (size_t)c->lay.N * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->user) != cudaSuccess ||
        cudaMemsetAsync(lpD(c), 0, (size_t)c->lay.N * sizeof(float), c->user) != cudaSuccess ||
        cudaMemcpyAsync(x_out, x_in, (size_t)c->lay.N * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->user) != cudaSuccess)
      rc = MC_ERR_CUDA;
    if (rc == MC_OK) rc = enqueue_residual(c, c->xa, c->user, lpQ(c));
    if (rc == MC_OK && cudaEventRecord(ev[0], c->user) != cudaSuccess) rc = MC_ERR_CUDA;
    if (rc == MC_OK) rc = enqueue_lp_sweeps_fused(c, nsweeps, c->user);
    for (int q = 1; q < 4 && rc == MC_OK; ++q)
      if (cudaEventRecord(ev[q], c->user) != cudaSuccess) rc = MC_ERR_CUDA;
  } else {
    rc = enqueue_sweeps(c, x_in, x_out, nsweeps, nullptr, c->user, ev, split_resid_ok(c));
  }
  double t[3] = {0.0, 0.0, 0.0};
  if (rc == MC_OK && cudaStreamSynchronize(c->user) != cudaSuccess) rc = MC_ERR_CUDA;
  for (int64_t k = 0; k < (fused ? 1 : nsweeps) && rc == MC_OK; ++k)
    for (int q = 0; q < 3; ++q) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ev[4 * k + q], ev[4 * k + q + 1]) != cudaSuccess) {
        rc = MC_ERR_CUDA;
        break;
      }
      t[q] += ms;
    }
  for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  free(ev);
  if (rc != MC_OK) return rc;
  ms_host[0] = t[0];
  ms_host[1] = t[1];
  ms_host[2] = t[2];
  // kernel launches: fused chains 3 per launch of up to kMaxFusedSweeps
  // sweeps (sweeps, scale, normalisation); the comparison splittings 2 per
  // sweep
  if (c->lay.lp)
    ms_host[3] = 2.0;   // residual (r, q) + the fused correction sweeps
  else if (fused)
    ms_host[3] = 3.0 * (double)((nsweeps + kMaxFusedSweeps - 1) / kMaxFusedSweeps);
  else
    ms_host[3] = 2.0 * (double)nsweeps;   // comparison splitting sweep + normalisation
  ms_host[4] = fused ? 1.0 : 0.0;
  return sync_header(c);
}

// Device address of a page-locked host buffer (16-byte aligned), or NULL for
// pageable memory.  Kernels read and write such buffers directly over the
// CPU-GPU link (NVLink-C2C on Grace-Blackwell), so no staging copy is needed.
static const double* mapped(const double* h) {
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (pa.type == cudaMemoryTypeHost && pa.devicePointer && ((uintptr_t)pa.devicePointer & 15u) == 0)
    return (const double*)pa.devicePointer;
  return nullptr;
}

int mc_sweep_host(mc_chain* c, const double* x_in_host, double* x_out_host, int64_t nsweeps,
                  double* stats_host) {
  if (!c || !x_in_host || !x_out_host || nsweeps < 1) return MC_ERR_ARG;
  if (!c->factored) return MC_ERR_NOT_FACTORED;
  const size_t bytes = (size_t)c->lay.N * sizeof(double);
  // page-locked input: the first half-sweep (and the step error) read it in
  // place; page-locked output: the final normalisation stores the result
  // straight into it (one fused launch).  Pageable buffers are copied.
  const double* in_dev = fused_ok(c) ? mapped(x_in_host) : nullptr;
  double* out_dev = (fused_ok(c) && nsweeps <= kMaxFusedSweeps) ? (double*)mapped(x_out_host)
                                                                 : nullptr;
  if (!in_dev) CK(cudaMemcpyAsync(c->xa, x_in_host, bytes, cudaMemcpyHostToDevice, c->user));
  const bool split = split_resid_ok(c);
  double* res_dev = out_dev ? out_dev : c->xa;
  int rc = enqueue_sweeps(c, in_dev ? in_dev : c->xa, res_dev, nsweeps, nullptr, c->user, nullptr,
                          stats_host != nullptr && split, stats_host != nullptr);
  if (rc == MC_OK && stats_host && !split) rc = enqueue_residual(c, res_dev, c->user);
  if (rc != MC_OK) return rc;
  if (!out_dev)
    CK(cudaMemcpyAsync(x_out_host, c->xa, bytes, cudaMemcpyDeviceToHost, c->user));
  const int st = sync_header(c);
  if (stats_host) {
    stats_host[0] = c->hh->stats[0];
    stats_host[1] = c->hh->stats[1];
    stats_host[2] = c->hh->stats[2];
  }
  return st;
}

// Residual of a chunk of mc_solve: none, direct (k_residual after the sweeps)
// or from the splitting inside the last fused launch.
enum { kResidNone = 0, kResidDirect = 1, kResidSplit = 3 };

// The sweeps (and residual) of one chunk of mc_solve on xa, in place.
static int enqueue_chunk(mc_chain* c, int64_t chunk, int resid_mode, cudaStream_t s) {
  int rc = enqueue_sweeps(c, c->xa, c->xa, chunk, nullptr, s, nullptr, resid_mode == kResidSplit);
  if (rc == MC_OK && resid_mode == kResidDirect) rc = enqueue_residual(c, c->xa, s);
  return rc;
}

static int capture_chunk(mc_chain* c, int chunk, int resid_mode) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_chunk(c, chunk, resid_mode, c->cap);
  if (rc == MC_OK &&
      cudaMemcpyAsync(c->hh, c->hdr, sizeof(Header), cudaMemcpyDeviceToHost, c->cap) != cudaSuccess)
    rc = MC_ERR_CUDA;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (rc != MC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return MC_ERR_CUDA;
  }
  const cudaError_t e2 = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    c->gexec = nullptr;
    return MC_ERR_CUDA;
  }
  c->g_chunk = chunk;
  c->g_resid = resid_mode;
  return MC_OK;
}

// Mixed-precision solve: outer FP64 refinement steps of check_every
// low-precision correction sweeps each; the iterate is xa (already set).
static int solve_refine(mc_chain* c, double* pi, double tol, double eps, int64_t maxit,
                        int32_t inner, mc_result* res) {
  const int64_t N = c->lay.N;
  int rc = enqueue_residual(c, c->xa, c->user, lpQ(c));
  if (rc != MC_OK) return rc;
  int st = sync_header(c);
  if (st != MC_OK) return st;
  double r = c->hh->stats[2], d = NAN, d_prev = NAN, kappa = NAN;
  int64_t k = 0;
  int converged = (tol > 0.0 && r <= tol);
  while (!converged && k < maxit) {
    const int64_t chunk = (maxit - k < inner) ? (maxit - k) : inner;
    if (chunk == inner) {
      if (!c->gexec || c->g_chunk != inner || c->g_resid != 2) {
        if (c->gexec) {
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_refine_step(c, inner, c->cap);
        if (rc == MC_OK && cudaMemcpyAsync(c->hh, c->hdr, sizeof(Header), cudaMemcpyDeviceToHost,
                                           c->cap) != cudaSuccess)
          rc = MC_ERR_CUDA;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        if (rc != MC_OK || e != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          return MC_ERR_CUDA;
        }
        const cudaError_t e2 = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
          c->gexec = nullptr;
          return MC_ERR_CUDA;
        }
        c->g_chunk = inner;
        c->g_resid = 2;
      }
      CK(cudaGraphLaunch(c->gexec, c->user));
      CK(cudaStreamSynchronize(c->user));
    } else {
      rc = enqueue_refine_step(c, (int)chunk, c->user);
      if (rc != MC_OK) return rc;
      CK(cudaMemcpyAsync(c->hh, c->hdr, sizeof(Header), cudaMemcpyDeviceToHost, c->user));
      CK(cudaStreamSynchronize(c->user));
    }
    k += chunk;
    st = c->hh->status;
    if (st != 0) {
      CK(cudaMemsetAsync(&c->hdr->status, 0, sizeof(int32_t), c->user));
      CK(cudaStreamSynchronize(c->user));
      return st;
    }
    d = c->hh->stats[1];
    r = c->hh->stats[2];
    if (d_prev > 0.0 && d > 0.0) kappa = pow(d / d_prev, 1.0 / (double)chunk);
    d_prev = d;
    if ((tol > 0.0 && r <= tol) || (eps > 0.0 && d <= eps)) converged = 1;
  }
  CK(cudaMemcpyAsync(pi, c->xa, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, c->user));
  CK(cudaStreamSynchronize(c->user));
  if (res) {
    res->sweeps = k;
    res->residual_l1 = r;
    res->step_l1 = d;
    res->contraction = kappa;
    res->converged = converged;
  }
  if (!converged && (tol > 0.0 || eps > 0.0)) return MC_ERR_NO_CONVERGENCE;
  return MC_OK;
}

int mc_solve(mc_chain* c, const double* x0, double* pi, double tol, double eps, int64_t maxit,
             int32_t check_every, mc_result* res) {
  if (!c || !pi || maxit < 1 || check_every < 1) return MC_ERR_ARG;
  if (((uintptr_t)pi | (uintptr_t)x0) & 7u) return MC_ERR_ARG;
  if (!c->factored) return MC_ERR_NOT_FACTORED;
  const int64_t N = c->lay.N;
  if (x0) {
    CK(launch_check_scale(x0, c->xa, N, c->hdr, c->dpart, c->user));
  } else {
    CK(launch_fill(c->xa, N, 1.0 / (double)N, c->user));
  }
  int st = sync_header(c);
  if (st != MC_OK) return st;
  if (c->lay.lp) return solve_refine(c, pi, tol, eps, maxit, check_every, res);
  // residual test every chunk: from the splitting inside the chunk's last
  // fused launch (block-tridiagonal stair splittings; confirmed once by the
  // direct residual before stopping) or the direct residual
  const int mode = tol > 0.0 ? (split_resid_ok(c) ? kResidSplit : kResidDirect) : kResidNone;
  int64_t k = 0;
  double d = NAN, d_prev = NAN, r = NAN, kappa = NAN;
  int converged = 0;
  bool direct = mode == kResidDirect;   // r is the direct residual of xa
  while (k < maxit) {
    const int64_t chunk = (maxit - k < check_every) ? (maxit - k) : check_every;
    direct = mode == kResidDirect;
    if (chunk == check_every) {
      if (!c->gexec || c->g_chunk != check_every || c->g_resid != mode) {
        const int rc = capture_chunk(c, check_every, mode);
        if (rc != MC_OK) return rc;
      }
      CK(cudaGraphLaunch(c->gexec, c->user));
      CK(cudaStreamSynchronize(c->user));
    } else {
      const int rc = enqueue_chunk(c, chunk, mode, c->user);
      if (rc != MC_OK) return rc;
      CK(cudaMemcpyAsync(c->hh, c->hdr, sizeof(Header), cudaMemcpyDeviceToHost, c->user));
      CK(cudaStreamSynchronize(c->user));
    }
    k += chunk;
    st = c->hh->status;
    if (st != 0) {
      CK(cudaMemsetAsync(&c->hdr->status, 0, sizeof(int32_t), c->user));
      CK(cudaStreamSynchronize(c->user));
      return st;
    }
    d = c->hh->stats[1];
    if (mode != kResidNone) r = c->hh->stats[2];
    if (d_prev > 0.0 && d > 0.0) kappa = pow(d / d_prev, 1.0 / (double)chunk);
    d_prev = d;
    if (mode == kResidSplit && r <= tol) {
      // confirm with the direct residual of the stored iterate (the two agree
      // to rounding; near the rounding floor the direct one decides)
      const int rc = enqueue_residual(c, c->xa, c->user);
      if (rc != MC_OK) return rc;
      st = sync_header(c);
      if (st != MC_OK) return st;
      r = c->hh->stats[2];
      direct = true;
    }
    if ((mode != kResidNone && r <= tol) || (eps > 0.0 && d <= eps)) {
      converged = 1;
      break;
    }
  }
  CK(cudaMemcpyAsync(pi, c->xa, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, c->user));
  if (!direct) {
    // the reported residual is always the direct one of the returned pi
    const int rc = enqueue_residual(c, c->xa, c->user);
    if (rc != MC_OK) return rc;
    st = sync_header(c);
    if (st != MC_OK) return st;
    r = c->hh->stats[2];
  } else {
    CK(cudaStreamSynchronize(c->user));
  }
  if (res) {
    res->sweeps = k;
    res->residual_l1 = r;
    res->step_l1 = d;
    res->contraction = kappa;
    res->converged = converged;
  }
  if (!converged && (tol > 0.0 || eps > 0.0)) return MC_ERR_NO_CONVERGENCE;
  return MC_OK;
}

int mc_residual(mc_chain* c, const double* pi, double* resid_l1_host) {
  if (!c || !pi || !resid_l1_host || ((uintptr_t)pi & 7u)) return MC_ERR_ARG;
  const int rc = enqueue_residual(c, pi, c->user);
  if (rc != MC_OK) return rc;
  const int st = sync_header(c);
  *resid_l1_host = c->hh->stats[2];
  return st;
}

int mc_export(mc_chain* c, int32_t plane, int64_t level0, int64_t count, double* dst_dev) {
  if (!c || !dst_dev || plane < 0 || plane >= c->lay.n_planes || level0 < 0 || count < 0 ||
      level0 + count > c->lay.L)
    return MC_ERR_ARG;
  if (plane >= kPlaneLU && !c->factored) return MC_ERR_ARG;
  if (count == 0) return MC_OK;
  const size_t pe = c->lay.plane_bytes / sizeof(double);
  const size_t mm = (size_t)c->lay.m * c->lay.m;
  const double* src = c->planes + plane * pe + (size_t)level0 * c->lay.ms;
  CK(cudaMemcpy2DAsync(dst_dev, mm * sizeof(double), src, (size_t)c->lay.ms * sizeof(double),
                       mm * sizeof(double), (size_t)count, cudaMemcpyDeviceToDevice, c->user));
  return MC_OK;
}

int mc_set_tuning(mc_chain* c, const mc_tuning* t) {
  if (!c || !t || t->blocks_per_sm < 0 || t->blocks_per_sm > 16 ||
      (t->levels_per_unit != 1 && t->levels_per_unit != 2 && t->levels_per_unit != 4) ||
      (!c->lay.lp && t->levels_per_unit != 1))
    return MC_ERR_ARG;
  c->tune_bps = t->blocks_per_sm;
  c->tune_lpu = t->levels_per_unit;
  return MC_OK;
}

int mc_get_tuning(const mc_chain* c, mc_tuning* t) {
  if (!c || !t) return MC_ERR_ARG;
  t->blocks_per_sm = c->tune_bps;
  t->levels_per_unit = c->tune_lpu;
  return MC_OK;
}

int mc_tune(mc_chain* c, const double* x, int64_t nsweeps, mc_tuning* best, double* best_ms) {
  if (!c || !x || ((uintptr_t)x & 7u) || nsweeps < 1 || nsweeps > kMaxFusedSweeps)
    return MC_ERR_ARG;
  if (!c->factored) return MC_ERR_NOT_FACTORED;
  if (!c->lay.lp && !fused_ok(c)) return MC_ERR_ARG;
  const int64_t N = c->lay.N;
  // candidates: blocks per SM (0 = the kernel's occupancy) x levels per unit
  static const int kBpsF64[] = {0, 1, 2};
  static const int kBpsLp[] = {0, 2, 3, 4};
  static const int kLpu[] = {1, 2, 4};
  const int nb = c->lay.lp ? 4 : 3, nl = c->lay.lp ? 3 : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return MC_ERR_CUDA;
  }
  const int bps0 = c->tune_bps, lpu0 = c->tune_lpu;
  int rc = MC_OK;
  // low precision: the correction sweeps of one refinement step from x (r and
  // q of x, d from zero); FP64: the fused sweeps from x into the scratch
  // iterate, with the residual units of a solve chunk.  x is only read.
  if (c->lay.lp) {
    if (cudaMemcpyAsync(c->xa, x, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->user) != cudaSuccess)
      rc = MC_ERR_CUDA;
    if (rc == MC_OK) rc = enqueue_residual(c, c->xa, c->user, lpQ(c));
  }
  float best_t = 1e30f;
  mc_tuning bt{bps0, lpu0};
  for (int bi = 0; bi < nb && rc == MC_OK; ++bi)
    for (int li = 0; li < nl && rc == MC_OK; ++li) {
      c->tune_bps = c->lay.lp ? kBpsLp[bi] : kBpsF64[bi];
      c->tune_lpu = kLpu[li];
      for (int rep = 0; rep < 2 && rc == MC_OK; ++rep) {   // the first run warms up
        if (c->lay.lp &&
            cudaMemsetAsync(lpD(c), 0, (size_t)N * sizeof(float), c->user) != cudaSuccess)
          rc = MC_ERR_CUDA;
        if (rc == MC_OK && cudaEventRecord(e0, c->user) != cudaSuccess) rc = MC_ERR_CUDA;
        if (rc == MC_OK)
          rc = c->lay.lp ? enqueue_lp_sweeps_fused(c, nsweeps, c->user)
                         : enqueue_sweeps(c, x, c->xa, nsweeps, nullptr, c->user, nullptr,
                                          split_resid_ok(c));
        if (rc == MC_OK && cudaEventRecord(e1, c->user) != cudaSuccess) rc = MC_ERR_CUDA;
      }
      float ms = 0.0f;
      if (rc == MC_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = MC_ERR_CUDA;
      if (rc == MC_OK && ms < best_t) {
        best_t = ms;
        bt.blocks_per_sm = c->tune_bps;
        bt.levels_per_unit = c->tune_lpu;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tune_bps = rc == MC_OK ? bt.blocks_per_sm : bps0;
  c->tune_lpu = rc == MC_OK ? bt.levels_per_unit : lpu0;
  if (rc != MC_OK) return rc;
  const int st = sync_header(c);
  if (st != MC_OK) return st;
  if (best) *best = bt;
  if (best_ms) *best_ms = best_t;
  return MC_OK;
}

int mc_sync(mc_chain* c) {
  if (!c) return MC_ERR_ARG;
  return sync_header(c);
}

void mc_destroy(mc_chain* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->hh) cudaFreeHost(c->hh);
  delete c;
}

const char* mc_status_string(int s) {
  switch (s) {
    case MC_OK: return "ok";
    case MC_ERR_ARG: return "invalid argument";
    case MC_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case MC_ERR_CUDA: return "CUDA runtime error";
    case MC_ERR_SINGULAR_BLOCK: return "diagonal block with zero or non-finite pivot";
    case MC_ERR_NOT_FACTORED: return "chain not factored";
    case MC_ERR_BREAKDOWN: return "normalisation breakdown (e^T z <= 0 or not finite)";
    case MC_ERR_NO_CONVERGENCE: return "no convergence within maxit";
    case MC_ERR_TIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
  }
}

}  // extern "C"
