// Continuous-batching solve server (C ABI in include/mc.h, mc_server_*).
//
// Requests (independent chains of any L and m <= 256) are admitted into a
// caller-owned device arena as long as their workspace fits; each step runs
// one chunk of check_every sweeps for ALL active requests with the batched
// kernels of batch.cu (one fused persistent launch per block-size bucket for
// all sweeps of the chunk), then reads every request's residual and retires the converged
// ones.  New requests join at the next chunk, so their work overlaps with the
// requests already running.  A chunk is one CUDA graph, captured once per
// (grid, chunk length) and replayed: the kernels read the request table from
// device memory, which the graph itself refreshes from pinned host memory.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "batch.cuh"
#include "chain.cuh"

using namespace mc;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Req {
  int64_t tag;
  mc_chain* chain;
  size_t off, bytes;
  double* lsum;
  int64_t sweeps;
  double step_prev;
  bool fresh;           // factor status not yet checked
};

struct Done {
  int64_t tag;
  double* pi;           // host copy of the result (malloc), N doubles
  int64_t N;
  mc_result res;
  int status;
};

}  // namespace

struct mc_server {
  mc_server_desc d;
  char* arena;
  size_t arena_bytes;
  cudaStream_t user;
  int num_sms;
  std::map<size_t, size_t> free_;   // offset -> size, coalesced
  BTable* t_dev;
  BOut* out_dev;
  BTable* t_host;                   // pinned
  BOut* out_host;                   // pinned
  std::vector<Req*> active;
  std::deque<Done> done;
  cudaStream_t cap;
  cudaGraphExec_t gexec;
  BTune g_tune;          // configuration of the captured graph
  int g_chunk;
  int G;                 // levels per unit of the table being built
  std::map<uint64_t, BTune> tuned;
  std::map<uint64_t, int> tuned_G;
  // autotuner results: (signature, candidate, ms per chunk) of every timed chunk
  std::vector<mc_server_tuning> trials;
  int64_t chunks;
  int32_t epoch_next;   // completion-counter base of the next chunk
};

namespace {

bool alloc(mc_server* s, size_t bytes, size_t* off) {
  for (auto it = s->free_.begin(); it != s->free_.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t start = it->first + bytes;
      s->free_.erase(it);
      if (rest) s->free_[start] = rest;
      return true;
    }
  }
  return false;
}

void release(mc_server* s, size_t off, size_t bytes) {
  auto it = s->free_.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_.erase(nx);
  }
  if (it != s->free_.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_.erase(it);
    }
  }
}

mc_desc request_desc(const mc_server* s, int64_t L, int32_t m) {
  mc_desc d{};
  d.L = L;
  d.m = m;
  d.stair = s->d.stair;
  d.apply = s->d.apply;
  d.dtype = s->d.dtype;
  return d;
}

size_t request_bytes(const mc_server* s, int64_t L, int32_t m) {
  const mc_desc d = request_desc(s, L, m);
  const size_t ws = mc_workspace_bytes(&d);
  if (!ws) return 0;
  return align_up(ws) + align_up((size_t)L * sizeof(double));
}

void fill_req(const mc_server* s, const Req* r, BReq* q) {
  mc_chain* c = r->chain;
  const size_t pe = c->lay.plane_bytes / sizeof(double);
  const bool coupled = s->d.apply == MC_APPLY_COUPLED;
  memset(q, 0, sizeof(*q));
  q->A = c->planes + (coupled ? kPlaneWLO : kPlaneTLO) * pe;
  q->B = c->planes + (coupled ? kPlaneWUP : kPlaneTUP) * pe;
  q->C = c->planes + kPlaneNINV * pe;
  q->TLO = c->planes + kPlaneTLO * pe;
  q->TDD = c->planes + kPlaneTDD * pe;
  q->TUP = c->planes + kPlaneTUP * pe;
  q->NINV = c->planes + kPlaneNINV * pe;
  if (c->lay.lp) {
    q->lA = chain_lpA(c);
    q->lB = chain_lpB(c);
    q->lC = chain_lpC(c);
    q->sc = chain_lpSc(c);
    q->d = chain_lpD(c);
    q->q = chain_lpQ(c);
    q->lp_bs = c->lay.lp_bs;
    q->lp_cbs = c->lay.lp_cbs;
  }
  q->x = c->xa;
  q->z = c->z;
  q->xb = c->xb;
  q->lsum = r->lsum;
  q->lsum2 = c->flsum;
  q->ver = c->fver;
  q->L = c->lay.L;
  q->m = c->lay.m;
  q->ms = c->lay.ms;
  q->R = (c->lay.m + 31) / 32;
  q->p1 = s->d.stair == 1 ? 0 : 1;
}

// Retire request i of the active list: copy pi to the host, free its memory.
int retire(mc_server* s, size_t i, int status, double resid, double step, double kappa,
           int converged) {
  Req* r = s->active[i];
  Done dn{};
  dn.tag = r->tag;
  dn.N = r->chain->lay.N;
  dn.status = status;
  dn.pi = (double*)malloc(sizeof(double) * (size_t)dn.N);
  int rc = MC_OK;
  if (!dn.pi) rc = MC_ERR_ARG;
  if (rc == MC_OK && cudaMemcpy(dn.pi, r->chain->xa, sizeof(double) * (size_t)dn.N,
                                cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = MC_ERR_CUDA;
  dn.res.sweeps = r->sweeps;
  dn.res.residual_l1 = resid;
  dn.res.step_l1 = step;
  dn.res.contraction = kappa;
  dn.res.converged = converged;
  // a result that could not be copied out is reported as failed, without pi
  if (rc != MC_OK) {
    free(dn.pi);
    dn.pi = nullptr;
    if (dn.status == MC_OK) dn.status = rc;
    dn.res.converged = 0;
  }
  s->done.push_back(dn);
  mc_destroy(r->chain);
  release(s, r->off, r->bytes);
  delete r;
  s->active.erase(s->active.begin() + (long)i);
  return rc;
}

// The next chunk (about to run) uses the current counter base; the one after
// it starts c higher.  Called before each execution of a chunk (a direct
// enqueue or a graph launch), while no chunk is in flight.  Before the 32-bit
// counters could wrap, every active request's counters are zeroed (stream
// ordered before the chunk) and the base restarts at 0.
int begin_chunk(mc_server* s, int c) {
  if (s->epoch_next > (1 << 30)) {
    for (Req* r : s->active)
      if (cudaMemsetAsync(r->chain->fver, 0, (size_t)r->chain->lay.L * sizeof(int), s->user) !=
          cudaSuccess)
        return MC_ERR_CUDA;
    s->epoch_next = 0;
  }
  s->t_host->epoch = s->epoch_next;
  s->epoch_next += c;
  return MC_OK;
}

// Chunk body on stream st: c fused sweeps (FP64) or one refinement step of c
// fused correction sweeps (low precision), then every request's residual.
// ev (optional, 2 events): recorded around the fused sweep launches.
int enqueue_chunk(mc_server* s, BTune g, int c, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  const bool lp = s->d.dtype != MC_F64;
  const int coupled = s->d.apply == MC_APPLY_COUPLED;
  if (cudaMemcpyAsync(s->t_dev, s->t_host, sizeof(BTable), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(s->out_dev, 0, sizeof(BOut) * kMaxReq, st) != cudaSuccess)
    return MC_ERR_CUDA;
  unsigned long long* claim = &s->t_dev->claim[0];
  if (lp && b_lp_zero(s->t_dev, g, st) != cudaSuccess) return MC_ERR_CUDA;
  if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return MC_ERR_CUDA;
  if (lp) {
    if (b_lp_sweeps(s->t_dev, claim, s->out_dev, s->d.dtype == MC_BF16, coupled, c, g, st) !=
        cudaSuccess)
      return MC_ERR_CUDA;
  } else {
    if (b_sweeps(s->t_dev, claim, s->out_dev, coupled, c, g, st) != cudaSuccess)
      return MC_ERR_CUDA;
  }
  if (ev && cudaEventRecord(ev[1], st) != cudaSuccess) return MC_ERR_CUDA;
  if (lp) {
    if (b_lp_finish(s->t_dev, s->out_dev, g, st) != cudaSuccess) return MC_ERR_CUDA;
  } else {
    if (b_sweeps_finish(s->t_dev, s->out_dev, c, g, st) != cudaSuccess) return MC_ERR_CUDA;
  }
  if (b_resid(s->t_dev, s->out_dev, lp ? 1 : 0, g, st) != cudaSuccess) return MC_ERR_CUDA;
  if (cudaMemcpyAsync(s->out_host, s->out_dev, sizeof(BOut) * kMaxReq, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess)
    return MC_ERR_CUDA;
  return MC_OK;
}

// Algorithmic bytes the fused sweep launches of one chunk stream: per level
// and sweep the stored operator blocks once plus the neighbour vectors read
// and the level written (FP64: 24 m^2 + 16 m inverse, 16 m^2 + 16 m coupled;
// low precision: 2 e m^2 for the two off-diagonal blocks of e-byte entries,
// + 4 m^2 for the FP32 inverse, + 16 m for the FP32 vectors d and q).
double chunk_sweep_bytes(const mc_server* s, int c) {
  const bool inv = s->d.apply == MC_APPLY_INVERSE;
  double b = 0.0;
  for (const Req* r : s->active) {
    const double m = r->chain->lay.m, L = (double)r->chain->lay.L;
    double lvl;
    if (s->d.dtype == MC_F64) {
      lvl = (inv ? 24.0 : 16.0) * m * m + 16.0 * m;
    } else {
      const double e = s->d.dtype == MC_F32 ? 4.0 : 2.0;
      lvl = 2.0 * e * m * m + (inv ? 4.0 * m * m : 0.0) + 16.0 * m;
    }
    b += lvl * L * c;
  }
  return b;
}

// Autotuner: for each batch signature (size classes present, size class of
// the total level count) time one live chunk per candidate configuration
// (real work, counted as such: results do not depend on the configuration)
// and keep the fastest.  Coordinate search: the persistent grid (1, 2, 3, 4,
// 6, 8 resident 256-thread blocks per SM) with one level per unit, then 2
// and 4 levels per unit, then the other bucket edge, then (low precision
// with m <= 64 present) the other load depth.
uint64_t signature(const mc_server* s) {
  const BTable* t = s->t_host;
  const int64_t lv = t->off_lv[t->n];
  int lg = 0;
  while ((1LL << lg) < lv && lg < 62) ++lg;
  uint64_t sig = (uint64_t)(lg / 2) << 8;
  for (int c = 0; c < kClasses; ++c)
    if (t->cls_end[c] > (c ? t->cls_end[c - 1] : 0)) sig |= 1ull << c;
  return sig;
}

// Factor status of newly admitted requests (one sync when there are any).
int check_fresh(mc_server* s) {
  bool any = false;
  for (Req* r : s->active) any |= r->fresh;
  if (!any) return MC_OK;
  if (cudaStreamSynchronize(s->user) != cudaSuccess) return MC_ERR_CUDA;
  for (size_t i = 0; i < s->active.size();) {
    Req* r = s->active[i];
    if (!r->fresh) {
      ++i;
      continue;
    }
    int32_t st = 0;
    if (cudaMemcpy(&st, &r->chain->hdr->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
      return MC_ERR_CUDA;
    r->fresh = false;
    r->chain->factored = st == 0;
    if (st != 0) {
      retire(s, i, st, NAN, NAN, NAN, 0);
      continue;
    }
    ++i;
  }
  return MC_OK;
}

// Fill the pinned request table from the active list (small blocks first);
// returns the table order.
std::vector<Req*> build_table(mc_server* s) {
  // size classes m <= 32, 64, 128, 256, in that order
  auto cls = [](const Req* r) { return size_class(r->chain->lay.m); };
  std::stable_sort(s->active.begin(), s->active.end(),
                   [&](const Req* a, const Req* b) { return cls(a) < cls(b); });
  BTable* t = s->t_host;
  t->n = (int32_t)s->active.size();
  for (int c = 0; c < kClasses; ++c) t->cls_end[c] = 0;
  t->G = s->G;
  t->off_h1[0] = t->off_h2[0] = t->off_lv[0] = 0;
  const int p1 = s->d.stair == 1 ? 0 : 1;
  for (int i = 0; i < t->n; ++i) {
    const Req* r = s->active[(size_t)i];
    const int64_t L = r->chain->lay.L;
    for (int c = cls(r); c < kClasses; ++c) t->cls_end[c] = i + 1;
    fill_req(s, r, &t->r[i]);
    const int64_t G = class_group(s->G, r->chain->lay.m);
    t->r[i].G = (int32_t)G;
    // units: groups of G levels of each half-sweep
    const int64_t P1 = (L - p1 + 1) / 2, P2 = (L - (1 - p1) + 1) / 2;
    t->off_h1[i + 1] = t->off_h1[i] + (P1 + G - 1) / G;
    t->off_h2[i + 1] = t->off_h2[i] + (P2 + G - 1) / G;
    t->off_lv[i + 1] = t->off_lv[i] + L;
  }
  return std::vector<Req*>(s->active.begin(), s->active.end());
}

// After a chunk: count its sweeps and retire converged, failed and exhausted
// requests (out_host is indexed by table position).  Returns retirements.
int process_outputs(mc_server* s, const std::vector<Req*>& order, int c) {
  s->chunks++;
  int nd = 0;
  for (size_t k = 0; k < order.size(); ++k) {
    const BOut& o = s->out_host[k];
    Req* r = order[k];
    r->sweeps += c;
    const size_t i =
        (size_t)(std::find(s->active.begin(), s->active.end(), r) - s->active.begin());
    const double kap =
        (r->step_prev > 0 && o.step > 0) ? pow(o.step / r->step_prev, 1.0 / c) : NAN;
    r->step_prev = o.step;
    if (o.status != 0) {
      retire(s, i, o.status, o.resid, o.step, kap, 0);
      ++nd;
    } else if (s->d.tol > 0 && o.resid <= s->d.tol) {
      retire(s, i, MC_OK, o.resid, o.step, kap, 1);
      ++nd;
    } else if (r->sweeps >= s->d.maxit) {
      retire(s, i, MC_ERR_NO_CONVERGENCE, o.resid, o.step, kap, 0);
      ++nd;
    }
  }
  return nd;
}

}  // namespace

extern "C" {

int mc_server_create(const mc_server_desc* desc, void* arena, size_t arena_bytes,
                     void* cuda_stream, mc_server** out) {
  if (!out) return MC_ERR_ARG;
  *out = nullptr;
  if (!desc || desc->check_every < 1 || desc->maxit < 1 || desc->max_active < 1 ||
      desc->max_active > kMaxReq || (desc->stair != 1 && desc->stair != 2) ||
      (desc->apply != MC_APPLY_INVERSE && desc->apply != MC_APPLY_COUPLED) ||
      (desc->dtype != MC_F64 && desc->dtype != MC_F32 && desc->dtype != MC_BF16))
    return MC_ERR_ARG;
  const size_t head = align_up(sizeof(BTable)) + align_up(sizeof(BOut) * kMaxReq);
  if (!arena || ((uintptr_t)arena & (kAlign - 1)) || arena_bytes < head + kAlign)
    return MC_ERR_WORKSPACE;
  mc_server* s = new (std::nothrow) mc_server();
  if (!s) return MC_ERR_ARG;
  s->d = *desc;
  s->arena = (char*)arena;
  s->arena_bytes = arena_bytes;
  s->user = (cudaStream_t)cuda_stream;
  s->t_dev = (BTable*)s->arena;
  s->out_dev = (BOut*)(s->arena + align_up(sizeof(BTable)));
  s->free_[head] = (arena_bytes - head) / kAlign * kAlign;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaHostAlloc((void**)&s->t_host, sizeof(BTable), cudaHostAllocDefault) != cudaSuccess) {
    delete s;
    return MC_ERR_CUDA;
  }
  if (cudaHostAlloc((void**)&s->out_host, sizeof(BOut) * kMaxReq, cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFreeHost(s->t_host);
    delete s;
    return MC_ERR_CUDA;
  }
  memset(s->t_host, 0, sizeof(BTable));
  s->g_tune = BTune{2 * s->num_sms, 256, desc->dtype != MC_F64 ? 1 : 0, 0};
  s->G = 1;
  *out = s;
  return MC_OK;
}

size_t mc_server_request_bytes(const mc_server* s, int64_t L, int32_t m) {
  if (!s) return 0;
  return request_bytes(s, L, m);
}

int mc_server_submit(mc_server* s, int64_t tag, int64_t L, int32_t m, const double* dn,
                     const double* loc, const double* up) {
  if (!s || !dn || !loc || !up || L < 2 || m < 1 || m > kMaxM) return MC_ERR_ARG;
  const size_t bytes = request_bytes(s, L, m);
  if (!bytes) return MC_ERR_ARG;
  if ((int)s->active.size() >= s->d.max_active) return MC_ERR_WORKSPACE;
  size_t off = 0;
  if (!alloc(s, bytes, &off)) return MC_ERR_WORKSPACE;
  const mc_desc d = request_desc(s, L, m);
  const size_t ws = align_up(mc_workspace_bytes(&d));
  mc_chain* c = nullptr;
  int rc = chain_init(&d, s->arena + off, ws, s->user, &c);
  if (rc != MC_OK) {
    release(s, off, bytes);
    return rc;
  }
  // layout of Q^T from the host generator blocks (a row-major Q block is the
  // column-major Q^T block): T_lo[l] = up[l-1], T_up[l] = dn[l+1], T_dd = loc
  const Layout& y = c->lay;
  const size_t pe = y.plane_bytes / sizeof(double), mm = (size_t)m * m;
  const size_t dp = (size_t)y.ms * sizeof(double), sp = mm * sizeof(double);
  double* P = c->planes;
  if (cudaMemsetAsync(P + kPlaneTLO * pe, 0, dp, s->user) != cudaSuccess ||
      cudaMemcpy2DAsync(P + kPlaneTLO * pe + y.ms, dp, up, sp, sp, (size_t)(L - 1),
                        cudaMemcpyHostToDevice, s->user) != cudaSuccess ||
      cudaMemcpy2DAsync(P + kPlaneTUP * pe, dp, dn + mm, sp, sp, (size_t)(L - 1),
                        cudaMemcpyHostToDevice, s->user) != cudaSuccess ||
      cudaMemsetAsync(P + kPlaneTUP * pe + (size_t)(L - 1) * y.ms, 0, dp, s->user) !=
          cudaSuccess ||
      cudaMemcpy2DAsync(P + kPlaneTDD * pe, dp, loc, sp, sp, (size_t)L, cudaMemcpyHostToDevice,
                        s->user) != cudaSuccess)
    rc = MC_ERR_CUDA;
  if (rc == MC_OK &&
      cudaMemsetAsync(c->fver, 0, (size_t)L * sizeof(int), s->user) != cudaSuccess)
    rc = MC_ERR_CUDA;
  if (rc == MC_OK) rc = chain_factor_async(c);
  if (rc == MC_OK && launch_fill(c->xa, y.N, 1.0 / (double)y.N, s->user) != cudaSuccess)
    rc = MC_ERR_CUDA;
  if (rc == MC_OK && y.lp) rc = chain_residual_async(c, c->xa, s->user, chain_lpQ(c));
  if (rc != MC_OK) {
    mc_destroy(c);
    release(s, off, bytes);
    return rc;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) {
    mc_destroy(c);
    release(s, off, bytes);
    return MC_ERR_ARG;
  }
  r->tag = tag;
  r->chain = c;
  r->off = off;
  r->bytes = bytes;
  r->lsum = (double*)(s->arena + off + ws);
  r->sweeps = 0;
  r->step_prev = NAN;
  r->fresh = true;
  s->active.push_back(r);
  return MC_OK;
}

int mc_server_step(mc_server* s, int32_t* n_active, int32_t* n_done) {
  if (!s) return MC_ERR_ARG;
  const int c = s->d.check_every;
  int rc = check_fresh(s);
  if (rc != MC_OK) return rc;
  if (!s->active.empty()) {
    const bool lp = s->d.dtype != MC_F64;
    s->G = 1;
    std::vector<Req*> order = build_table(s);
    const uint64_t sig = signature(s);
    auto it = s->tuned.find(sig);
    if (it == s->tuned.end() && s->d.autotune) {
      // candidate list: grids first (G = 1, default edges and depth), then
      // the other knobs around the best so far
      const BTune base{2 * s->num_sms, 256, lp ? 1 : 0, 0};
      BTune best = base;
      int bestG = 1;
      float best_ms = 1e30f;
      cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
      for (cudaEvent_t& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return MC_ERR_CUDA;
      const bool small_lp = lp && (sig & 3ull) != 0;
      static const int kGrid[] = {1, 2, 3, 4, 6, 8};
      bool stop = false;
      for (int stage = 0; stage < 4 && !stop && rc == MC_OK; ++stage) {
        const int ncand = stage == 0 ? 6 : stage == 1 ? 2 : (stage == 3 && !small_lp) ? 0 : 1;
        for (int ci = 0; ci < ncand && !stop && rc == MC_OK; ++ci) {
          BTune g = best;
          int G = bestG;
          if (stage == 0) g.blocks = kGrid[ci] * s->num_sms;
          if (stage == 1) G = ci == 0 ? 2 : 4;
          if (stage == 2) g.split64 = 1 - best.split64;
          if (stage == 3) g.deep = 1 - best.deep;
          s->G = G;
          order = build_table(s);
          if (cudaEventRecord(ev[0], s->user) != cudaSuccess) rc = MC_ERR_CUDA;
          if (rc == MC_OK) rc = begin_chunk(s, c);
          if (rc == MC_OK) rc = enqueue_chunk(s, g, c, s->user, ev + 1);
          if (rc == MC_OK && cudaEventRecord(ev[3], s->user) != cudaSuccess) rc = MC_ERR_CUDA;
          if (rc == MC_OK && cudaEventSynchronize(ev[3]) != cudaSuccess) rc = MC_ERR_CUDA;
          float ms = 0.0f, sw = 0.0f;
          if (rc == MC_OK && (cudaEventElapsedTime(&ms, ev[0], ev[3]) != cudaSuccess ||
                              cudaEventElapsedTime(&sw, ev[1], ev[2]) != cudaSuccess))
            rc = MC_ERR_CUDA;
          if (rc != MC_OK) break;
          mc_server_tuning tr{};
          tr.signature = sig;
          tr.blocks_per_sm = g.blocks / s->num_sms;
          tr.levels_per_unit = G;
          tr.split64 = g.split64;
          tr.deep = g.deep;
          tr.chunk_ms = ms;
          tr.sweep_ms = sw;
          tr.sweep_bytes = chunk_sweep_bytes(s, c);
          s->trials.push_back(tr);
          if (ms < best_ms) {
            best_ms = ms;
            best = g;
            bestG = G;
          }
          stop = process_outputs(s, order, c) > 0 || s->active.empty();
        }
      }
      for (cudaEvent_t e : ev) cudaEventDestroy(e);
      if (rc != MC_OK) return rc;
      s->tuned[sig] = best;
      s->tuned_G[sig] = bestG;
      for (mc_server_tuning& tr : s->trials)
        if (tr.signature == sig)
          tr.chosen = tr.blocks_per_sm == best.blocks / s->num_sms && tr.levels_per_unit == bestG &&
                      tr.split64 == best.split64 && tr.deep == best.deep;
    } else {
      BTune g{2 * s->num_sms, 256, lp ? 1 : 0, 0};
      int G = 1;
      if (it != s->tuned.end()) {
        g = it->second;
        G = s->tuned_G[sig];
      }
      if (G != s->G) {
        s->G = G;
        order = build_table(s);
      }
      if (!s->gexec || s->g_chunk != c || s->g_tune.blocks != g.blocks ||
          s->g_tune.threads != g.threads || s->g_tune.split64 != g.split64 ||
          s->g_tune.deep != g.deep) {
        if (s->gexec) {
          cudaGraphExecDestroy(s->gexec);
          s->gexec = nullptr;
        }
        if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return MC_ERR_CUDA;
        rc = enqueue_chunk(s, g, c, s->cap);
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s->cap, &gr);
        if (rc != MC_OK || e != cudaSuccess) {
          if (gr) cudaGraphDestroy(gr);
          cudaGetLastError();
          return MC_ERR_CUDA;
        }
        const cudaError_t e2 = cudaGraphInstantiate(&s->gexec, gr, 0);
        cudaGraphDestroy(gr);
        if (e2 != cudaSuccess) {
          s->gexec = nullptr;
          return MC_ERR_CUDA;
        }
        s->g_chunk = c;
        s->g_tune = g;
      }
      rc = begin_chunk(s, c);
      if (rc != MC_OK) return rc;
      if (cudaGraphLaunch(s->gexec, s->user) != cudaSuccess ||
          cudaStreamSynchronize(s->user) != cudaSuccess)
        return MC_ERR_CUDA;
      process_outputs(s, order, c);
    }
  }
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_done) *n_done = (int32_t)s->done.size();
  return MC_OK;
}

int mc_server_fetch(mc_server* s, int64_t* tag, double* pi_host, int64_t n_cap, mc_result* res,
                    int32_t* status) {
  if (!s || s->done.empty()) return MC_ERR_ARG;
  Done dn = s->done.front();
  if (pi_host && n_cap < dn.N) return MC_ERR_ARG;
  s->done.pop_front();
  if (tag) *tag = dn.tag;
  if (pi_host && dn.pi) memcpy(pi_host, dn.pi, sizeof(double) * (size_t)dn.N);
  if (res) *res = dn.res;
  if (status) *status = dn.status;
  free(dn.pi);
  return MC_OK;
}

int mc_server_grid(const mc_server* s, int32_t* blocks, int32_t* threads, int32_t* n_tuned) {
  if (!s) return MC_ERR_ARG;
  if (blocks) *blocks = s->g_tune.blocks;
  if (threads) *threads = s->g_tune.threads;
  if (n_tuned) *n_tuned = (int32_t)s->tuned.size();
  return MC_OK;
}

int mc_server_trials(const mc_server* s, mc_server_tuning* out, int32_t cap, int32_t* n) {
  if (!s || cap < 0 || (cap > 0 && !out)) return MC_ERR_ARG;
  const int32_t total = (int32_t)s->trials.size();
  for (int32_t i = 0; i < total && i < cap; ++i) out[i] = s->trials[(size_t)i];
  if (n) *n = total;
  return MC_OK;
}

void mc_server_destroy(mc_server* s) {
  if (!s) return;
  cudaStreamSynchronize(s->user);
  while (!s->active.empty()) {
    Req* r = s->active.back();
    mc_destroy(r->chain);
    delete r;
    s->active.pop_back();
  }
  for (Done& dn : s->done) free(dn.pi);
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->t_host) cudaFreeHost(s->t_host);
  if (s->out_host) cudaFreeHost(s->out_host);
  delete s;
}

}  // extern "C"
