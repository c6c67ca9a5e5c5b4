// Mixed-precision staircase sweeps for iterative refinement.
//
// Outer step (FP64): r = Q^T pi (direct, from the FP64 blocks), q = (-T_dd)^{-1} r.
// Inner sweeps (FP32 arithmetic): the staircase step of Algorithm 2 applied to
// the correction equation T d = -r, i.e. d <- M^{-1}(N d - r), which on every
// block row reads
//     d_l = (-T_dd)^{-1}(T_lo d_{l-1} + T_up d_{l+1}) + q_l
//  (inverse mode)  or  W_lo d_{l-1} + W_up d_{l+1} + q_l  (coupled mode),
// half-sweep 1 on the diagonal-only rows, half-sweep 2 on the coupled rows,
// in place on one FP32 vector d that starts at zero; all sweeps of a step run
// as one fused launch.
// Update (FP64): pi <- (pi + d) / e^T(pi + d).
//
// Storage of the streamed blocks: FP32, or BF16 with one power-of-two scale per
// block (B = 2^e * B', max |B'| < 1), applied to the input vector in FP32.
// (-T_dd)^{-1} of the inverse mode is stored in FP32.  Lane loads are 8 bytes:
// V = 2 FP32 or 4 BF16 consecutive rows per lane, groups of 32 V rows.
#include <cuda_bf16.h>
#include <math.h>

#include "mc_internal.cuh"
#include "lowprec_dev.cuh"
#include "wave_dev.cuh"

namespace mc {

namespace {

using namespace dev;

struct LpArgs {
  const void* A;       // T_lo or W_lo plane (element type T)
  const void* B;       // T_up or W_up plane
  const float* C;      // (-T_dd)^{-1} in FP32 (inverse mode)
  const float* sc;     // per level: scale of A, scale of B
  float* d;            // iterate, updated in place
  const float* q;      // (-T_dd)^{-1} r
  int64_t L;
  int m, parity;        // parity: levels of half-sweep 1
  int64_t abs_, cbs;   // block strides in elements (A/B planes, C plane)
};

// All `K` correction sweeps of one refinement step in one persistent launch:
// units (sweep k, half-sweep h, levels l0, l0 + 2, ..., at most lpu adjacent
// levels of the half-sweep) claimed in order, each waiting for its
// neighbour levels through per-level completion counters (as the FP64 fused
// sweeps): one claim, one wait for the lpu + 1 neighbours and one completion
// fence per unit.  d is updated in place; a unit overwrites its levels only
// after the units that read their previous values (the neighbours' previous
// updates) have completed, which is the condition it waits for.
template <typename T>
struct SmallOf {
  using type = unsigned short;   // BF16 bits
};
template <>
struct SmallOf<float> {
  using type = float;
};

// SMALL = 16, 32 or 64: blocks of at most SMALL rows through
// level_sweep_lp_small; 0: level_sweep_lp.
template <typename T, int G, int GF, bool COUPLED, int SMALL = 0>
__global__ void __launch_bounds__(256) k_sweeps_lp(LpArgs a, int64_t K, int lpu, int* ver,
                                                   unsigned long long* claim, Header* hdr,
                                                   unsigned long long wait_ns) {
  extern __shared__ float fsh[];
  constexpr int SL = LpSlice<T, G, GF>::SL;
  const int lane = threadIdx.x & 31;
  float* slice = fsh + (threadIdx.x >> 5) * 3 * SL;
  const T* Ap = reinterpret_cast<const T*>(a.A);
  const T* Bp = reinterpret_cast<const T*>(a.B);
  const int64_t P0 = (a.L - a.parity + 1) / 2;   // levels of half-sweep 1
  const int64_t P1 = a.L - P0;
  const int64_t U0 = (P0 + lpu - 1) / lpu, U1 = (P1 + lpu - 1) / lpu;   // units per half-sweep
  const unsigned long long per = (unsigned long long)(U0 + U1);
  const unsigned long long total = (unsigned long long)K * per;
  unsigned long long q0 = claim_unit(claim, lane);
  unsigned long long q = __shfl_sync(0xffffffffu, q0, 0);
  while (q < total) {
    q0 = claim_unit(claim, lane);
    const int64_t k = (int64_t)(q / per);
    const int64_t r = (int64_t)q - k * (int64_t)per;
    const bool h2 = r >= U0;
    const int64_t g = h2 ? r - U0 : r;
    const int64_t l0 = 2 * lpu * g + (h2 ? 1 - a.parity : a.parity);
    const int64_t left = (h2 ? P1 : P0) - (int64_t)lpu * g;
    const int n = left < lpu ? (int)left : lpu;
    const int need = (int)(h2 ? k + 1 : k);
    if (need > 0) wait_levels(ver, l0 - 1, 2, n + 1, a.L, need, &hdr->status, lane, wait_ns);
    for (int i = 0; i < n; ++i) {
    const int64_t l = l0 + 2 * i;
    if constexpr (SMALL > 0) {
      using S = typename SmallOf<T>::type;
      // BF16: 16 loads in flight (single chains; the batched kernel keeps 8,
      // its register budget buys more resident warps there)
      constexpr int BW = sizeof(S) == 2 ? 16 : 8;
      level_sweep_lp_small<S, SMALL, COUPLED, true, BW>(reinterpret_cast<const S*>(a.A),
                                                    reinterpret_cast<const S*>(a.B), a.C, a.sc,
                                                    a.d, a.q, l, a.L, a.m, a.abs_, a.cbs, slice,
                                                    lane);
    } else {
      level_sweep_lp<T, G, GF, COUPLED, true>(Ap, Bp, a.C, a.sc, a.d, a.q, l, a.L, a.m, a.abs_,
                                              a.cbs, slice, lane);
    }
    }
    publish_levels(ver, l0, 2, n, (int)(k + 1), lane);
    q = __shfl_sync(0xffffffffu, q0, 0);
  }
}

// Convert one FP64 block (column-major, stride ms) to FP32 or to BF16 with a
// power-of-two scale: one CTA per (level, block).
template <typename T>
__global__ void __launch_bounds__(256) k_lp_convert(const double* __restrict__ src, T* dst,
                                                    float* sc, int sc_stride, int64_t L, int m,
                                                    int ms, int64_t dbs) {
  __shared__ double red[8];
  const int64_t l = blockIdx.x;
  if (l >= L) return;
  const double* s = src + (size_t)l * ms;
  const int mm = m * m;
  double mx = 0.0;
  for (int e = threadIdx.x; e < mm; e += blockDim.x) mx = fmax(mx, fabs(s[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
  int ex = 0;
  if (sizeof(T) == 2 && mx > 0.0) frexp(mx, &ex);   // mx = f 2^ex, f in [0.5, 1)
  const double inv = ldexp(1.0, -ex);
  for (int e = threadIdx.x; e < mm; e += blockDim.x) {
    if constexpr (sizeof(T) == 2) {
      dst[(size_t)l * dbs + e] = __double2bfloat16(s[e] * inv);
    } else {
      dst[(size_t)l * dbs + e] = (T)s[e];
    }
  }
  if (threadIdx.x == 0 && sc) sc[(size_t)l * sc_stride] = (float)ldexp(1.0, ex);
}

// pi_tmp = pi + d (FP64) with the sum reduced by the last block into s_out.
__global__ void __launch_bounds__(256) k_update(const double* __restrict__ pi,
                                                const float* __restrict__ d, double* out,
                                                int64_t N, double* bpart, Header* hdr,
                                                double* s_out) {
  __shared__ double sh[32];
  __shared__ bool last;
  double t = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = pi[i] + (double)d[i];
    out[i] = v;
    t += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += sh[w];
    bpart[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(&hdr->ticket[3], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(bpart + b);
    *s_out = s;
    hdr->ticket[3] = 0u;
  }
}

struct LpFused {
  int64_t K;
  int* ver;
  unsigned long long* claim;
  Header* hdr;
  unsigned long long wait_ns;
  int lpu;             // levels per unit (1, 2, 4)
  int bps;             // resident blocks per SM (0: all the kernel's occupancy allows)
};

// Grid: bps blocks per SM, by default every block the kernel's occupancy
// allows (the correction sweeps are memory-latency bound, so more resident
// warps help), but no more warps than units of one half-sweep.
template <typename T, int G, int GF, bool C, int SMALL = 0>
cudaError_t lp_fused_launch(const LpArgs& a, const LpFused& f, int num_sms, cudaStream_t s) {
  const size_t smem = (size_t)kWarpsPerBlock * 3 * LpSlice<T, G, GF>::SL * sizeof(float);
  static int occ = 0;
  if (occ == 0) {
    if (smem > 40 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(
          k_sweeps_lp<T, G, GF, C, SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int o = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &o, k_sweeps_lp<T, G, GF, C, SMALL>, 256, smem);
    if (e != cudaSuccess) return e;
    occ = o < 1 ? 1 : o;
  }
  const int bps = (f.bps > 0 && f.bps < occ) ? f.bps : occ;
  int64_t nb = (int64_t)bps * num_sms;
  const int64_t units = (a.L + f.lpu - 1) / f.lpu;
  const int64_t need = (units + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (nb > need) nb = need;
  k_sweeps_lp<T, G, GF, C, SMALL><<<(int)nb, 256, smem, s>>>(a, f.K, f.lpu, f.ver, f.claim, f.hdr,
                                                              f.wait_ns);
  return cudaGetLastError();
}

template <typename T, bool C>
cudaError_t lp_dispatch(const LpArgs& a, const LpFused& f, int nb, cudaStream_t s) {
  // nb: the number of SMs
  constexpr int V = Pack<T>::V;
  const int G = (a.m + 32 * V - 1) / (32 * V);
  const int GF = (a.m + 63) / 64;
  // at most 64 rows: 16-byte lane loads (BF16 columns must be 16-byte aligned)
  if (GF == 1 && (sizeof(typename SmallOf<T>::type) == 4 || a.m % 8 == 0)) {
    if (a.m <= 16) return lp_fused_launch<T, 1, 1, C, 16>(a, f, nb, s);
    if (a.m <= 32) return lp_fused_launch<T, 1, 1, C, 32>(a, f, nb, s);
    return lp_fused_launch<T, 1, 1, C, 64>(a, f, nb, s);
  }
  if (GF == 1) return lp_fused_launch<T, 1, 1, C>(a, f, nb, s);
  if (GF == 2)
    return G == 1 ? lp_fused_launch<T, 1, 2, C>(a, f, nb, s) : lp_fused_launch<T, 2, 2, C>(a, f, nb, s);
  if (GF <= 4) {
    if (G == 1) return lp_fused_launch<T, 1, 4, C>(a, f, nb, s);
    if (G == 2) return lp_fused_launch<T, 2, 4, C>(a, f, nb, s);
    return lp_fused_launch<T, 4, 4, C>(a, f, nb, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_lp_convert(const double* src, void* dst, int bf16, float* sc, int sc_stride,
                              const Layout& lay, int64_t dbs, cudaStream_t s) {
  const int nb = (int)lay.L;
  if (bf16)
    k_lp_convert<__nv_bfloat16><<<nb, 256, 0, s>>>(src, (__nv_bfloat16*)dst, sc, sc_stride, lay.L,
                                                   lay.m, lay.ms, dbs);
  else
    k_lp_convert<float><<<nb, 256, 0, s>>>(src, (float*)dst, sc, sc_stride, lay.L, lay.m, lay.ms,
                                           dbs);
  return cudaGetLastError();
}

cudaError_t launch_sweeps_lp(const void* A, const void* B, const float* C, const float* sc,
                             float* d, const float* q, int64_t L, int m, int parity, int64_t abs_,
                             int64_t cbs, int bf16, int coupled, int64_t K, int* ver,
                             unsigned long long* claim, Header* hdr, unsigned long long wait_ns,
                             int num_sms, int lpu, int bps, cudaStream_t s) {
  if (lpu != 1 && lpu != 2 && lpu != 4) return cudaErrorInvalidValue;
  const int nb = num_sms;
  LpArgs a{};
  a.A = A;
  a.B = B;
  a.C = C;
  a.sc = sc;
  a.d = d;
  a.q = q;
  a.L = L;
  a.m = m;
  a.parity = parity;
  a.abs_ = abs_;
  a.cbs = cbs;
  const LpFused f{K, ver, claim, hdr, wait_ns, lpu, bps};
  if (bf16 && m <= 128)
    return coupled ? lp_dispatch<Bf16x2, true>(a, f, nb, s) : lp_dispatch<Bf16x2, false>(a, f, nb, s);
  if (bf16)
    return coupled ? lp_dispatch<__nv_bfloat16, true>(a, f, nb, s)
                   : lp_dispatch<__nv_bfloat16, false>(a, f, nb, s);
  return coupled ? lp_dispatch<float, true>(a, f, nb, s) : lp_dispatch<float, false>(a, f, nb, s);
}

cudaError_t launch_update(const double* pi, const float* d, double* out, int64_t N, double* bpart,
                          int nb, Header* hdr, double* s_out, cudaStream_t s) {
  k_update<<<nb, 256, 0, s>>>(pi, d, out, N, bpart, hdr, s_out);
  return cudaGetLastError();
}

}  // namespace mc
