// Device helpers of the low-precision (FP32 / BF16 storage, FP32 arithmetic)
// warp-per-level products, shared by the single-chain and batched kernels.
// Lane loads are 8 bytes (4 for BF16 pairs): V consecutive rows per lane,
// groups of 32 V rows.
#pragma once
#include <cuda_bf16.h>

namespace mc {
namespace dev {

template <typename T>
struct Pack;
template <>
struct Pack<float> {
  static constexpr int V = 2;
  using Raw = float2;
  __device__ static __forceinline__ Raw load(const float* p) {
    return __ldcs(reinterpret_cast<const float2*>(p));
  }
  __device__ static __forceinline__ Raw zero() { return make_float2(0.0f, 0.0f); }
  __device__ static __forceinline__ float get(const Raw& r, int e) { return e == 0 ? r.x : r.y; }
};
template <>
struct Pack<__nv_bfloat16> {
  static constexpr int V = 4;
  using Raw = uint2;
  __device__ static __forceinline__ Raw load(const __nv_bfloat16* p) {
    return __ldcs(reinterpret_cast<const uint2*>(p));
  }
  __device__ static __forceinline__ Raw zero() { return make_uint2(0u, 0u); }
  // bf16 -> fp32 is exact: the 16 bits become the high half of the float
  __device__ static __forceinline__ float get(const Raw& r, int e) {
    const unsigned w = (e < 2) ? r.x : r.y;
    return __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
  }
};

// BF16 read two rows per lane (4-byte loads), for blocks of at most 128 rows
// where four-row loads would leave lanes idle.
struct Bf16x2 {
  unsigned short bits;   // one bf16, addressed in pairs
};
template <>
struct Pack<Bf16x2> {
  static constexpr int V = 2;
  using Raw = unsigned int;
  __device__ static __forceinline__ Raw load(const Bf16x2* p) {
    return __ldcs(reinterpret_cast<const unsigned int*>(p));
  }
  __device__ static __forceinline__ Raw zero() { return 0u; }
  __device__ static __forceinline__ float get(const Raw& r, int e) {
    return __uint_as_float(e ? (r & 0xffff0000u) : (r << 16));
  }
};

// acc[g][e] += M(row(g,e), j) * v[j], row(g,e) = 32 V g + V lane + e, for the
// m columns of a column-major block M of element type T.  U columns per
// batch so that U * G = 32 packed 8-byte loads per lane are in flight.
template <typename T, int G>
__device__ __forceinline__ void gemv_lp(float (&acc)[G][Pack<T>::V], const T* __restrict__ M,
                                        const float* v, int m, int lane) {
  constexpr int V = Pack<T>::V, U = (32 / G) < 8 ? 8 : (32 / G);
  using Raw = typename Pack<T>::Raw;
  for (int j0 = 0; j0 < m; j0 += U) {
    Raw t[U][G];
#pragma unroll
    for (int q = 0; q < U; ++q)
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int row = 32 * V * g + V * lane;
        t[q][g] = (j0 + q < m && row < m) ? Pack<T>::load(M + (size_t)(j0 + q) * m + row)
                                          : Pack<T>::zero();
      }
#pragma unroll
    for (int q = 0; q < U; q += 4) {
      const float4 vv = *reinterpret_cast<const float4*>(v + j0 + q);
      const float vq[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
          for (int e = 0; e < V; ++e)
            acc[g][e] = fmaf(Pack<T>::get(t[q + h][g], e), vq[h], acc[g][e]);
    }
  }
}

// Per-warp shared slice (floats per vector) of the low-precision products.
template <typename T, int G, int GF>
struct LpSlice {
  static constexpr int W = 32 * Pack<T>::V * G, WF = 64 * GF;
  static constexpr int SL = W > WF ? W : WF;
};

// One level of a correction half-sweep, in place on d:
//   inverse: d_l = (-T_dd)^{-1} (T_lo d_{l-1} + T_up d_{l+1}) + q_l,
//   coupled: d_l = W_lo d_{l-1} + W_up d_{l+1} + q_l,
// with A/B stored as T (BF16 blocks carry a power-of-two scale sc[2l], sc[2l+1]
// applied to the input vector) and C = (-T_dd)^{-1} in FP32.
// CG: d is also written by other SMs during the launch (L2 reads).
template <typename T, int G, int GF, bool COUPLED, bool CG = false>
__device__ __forceinline__ void level_sweep_lp(const T* A, const T* B, const float* C,
                                               const float* sc, float* d, const float* q,
                                               int64_t l, int64_t L, int m, int64_t abs_,
                                               int64_t cbs, float* slice, int lane) {
  constexpr int V = Pack<T>::V, SL = LpSlice<T, G, GF>::SL;
  float* v_lo = slice;
  float* v_up = slice + SL;
  float* v_g = slice + 2 * SL;
  const bool has_lo = l > 0, has_up = l < L - 1;
  const float s_lo = sc[2 * l], s_up = sc[2 * l + 1];
  for (int i = lane; i < SL; i += 32) {
    if constexpr (CG) {
      v_lo[i] = (has_lo && i < m) ? __ldcg(d + (l - 1) * m + i) * s_lo : 0.0f;
      v_up[i] = (has_up && i < m) ? __ldcg(d + (l + 1) * m + i) * s_up : 0.0f;
    } else {
      v_lo[i] = (has_lo && i < m) ? d[(l - 1) * m + i] * s_lo : 0.0f;
      v_up[i] = (has_up && i < m) ? d[(l + 1) * m + i] * s_up : 0.0f;
    }
  }
  __syncwarp();
  float acc[G][V];
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int e = 0; e < V; ++e) acc[g][e] = 0.0f;
  if (has_lo) gemv_lp<T, G>(acc, A + l * abs_, v_lo, m, lane);
  if (has_up) gemv_lp<T, G>(acc, B + l * abs_, v_up, m, lane);
  if (COUPLED) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int row = 32 * V * g + V * lane;
      if (row < m)
#pragma unroll
        for (int e = 0; e < V; ++e) d[l * m + row + e] = acc[g][e] + q[l * m + row + e];
    }
  } else {
    for (int i = lane; i < SL; i += 32) v_g[i] = 0.0f;
    __syncwarp();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int row = 32 * V * g + V * lane;
      if (row < m)
#pragma unroll
        for (int e = 0; e < V; ++e) v_g[row + e] = acc[g][e];
    }
    __syncwarp();
    float acc2[GF][2];
#pragma unroll
    for (int g = 0; g < GF; ++g) acc2[g][0] = acc2[g][1] = 0.0f;
    gemv_lp<float, GF>(acc2, C + l * cbs, v_g, m, lane);
#pragma unroll
    for (int g = 0; g < GF; ++g) {
      const int row = 64 * g + 2 * lane;
      if (row < m) {
        d[l * m + row] = acc2[g][0] + q[l * m + row];
        d[l * m + row + 1] = acc2[g][1] + q[l * m + row + 1];
      }
    }
  }
  __syncwarp();
}

// ---- blocks of at most ROWS = 16, 32 or 64 rows: 16-byte lane loads -------
// S = float (E = 4 rows per load) or unsigned short (BF16 bits, E = 8; needs
// m % 8 == 0 so that every column starts on a 16-byte boundary).  LPC = ROWS /
// E lanes cover one column (rows E (lane % LPC) ..), CPW = 32 / LPC columns
// per warp load, B loads in flight per lane (at most 64 columns per batch, so
// v is read inside its 64-float slice); lanes of one row group hold partial
// sums over different columns until small_combine adds them.
template <typename S, int ROWS, int BW = 8>
struct SmallLp {
  static constexpr int E = 16 / (int)sizeof(S), LPC = ROWS / E, CPW = 32 / LPC;
  static constexpr int B = 64 / CPW < BW ? 64 / CPW : BW;
};

__device__ __forceinline__ float small_elem(const uint4& t, int e, float) {
  return __uint_as_float(e == 0 ? t.x : e == 1 ? t.y : e == 2 ? t.z : t.w);
}
__device__ __forceinline__ float small_elem(const uint4& t, int e, unsigned short) {
  const unsigned w = (e >> 1) == 0 ? t.x : (e >> 1) == 1 ? t.y : (e >> 1) == 2 ? t.z : t.w;
  return __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
}

// acc[e] += sum over this lane's columns j of M(r0 + e, j) v[j]; v: slice of at
// least 64 floats, zero beyond m.
template <typename S, int ROWS, int BW = 8>
__device__ __forceinline__ void gemv_small(float (&acc)[SmallLp<S, ROWS>::E],
                                           const S* __restrict__ M, const float* v, int m,
                                           int lane) {
  using P = SmallLp<S, ROWS, BW>;
  const int c = lane / P::LPC, r0 = P::E * (lane % P::LPC);
  const bool rok = r0 < m;
  for (int jb = 0; jb < m; jb += P::CPW * P::B) {
    uint4 t[P::B];
#pragma unroll
    for (int b = 0; b < P::B; ++b) {
      const int j = jb + b * P::CPW + c;
      t[b] = (rok && j < m) ? __ldcs(reinterpret_cast<const uint4*>(M + (size_t)j * m + r0))
                            : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int b = 0; b < P::B; ++b) {
      const float vj = v[jb + b * P::CPW + c];
#pragma unroll
      for (int e = 0; e < P::E; ++e) acc[e] = fmaf(small_elem(t[b], e, S()), vj, acc[e]);
    }
  }
}

// Add the CPW partial sums of each row group (fixed shuffle tree); every lane
// ends with the totals of rows r0 ..
template <typename S, int ROWS>
__device__ __forceinline__ void small_combine(float (&acc)[SmallLp<S, ROWS>::E]) {
  using P = SmallLp<S, ROWS>;
#pragma unroll
  for (int o = P::LPC; o < 32; o <<= 1)
#pragma unroll
    for (int e = 0; e < P::E; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
}

// level_sweep_lp for m <= ROWS <= 64 (S as gemv_small; C is FP32); BW: loads
// in flight per lane for the A / B blocks.
template <typename S, int ROWS, bool COUPLED, bool CG = false, int BW = 8>
__device__ __forceinline__ void level_sweep_lp_small(const S* A, const S* B, const float* C,
                                                     const float* sc, float* d, const float* q,
                                                     int64_t l, int64_t L, int m, int64_t abs_,
                                                     int64_t cbs, float* slice, int lane) {
  constexpr int SL = 64, E = SmallLp<S, ROWS>::E, LPC = SmallLp<S, ROWS>::LPC;
  float* v_lo = slice;
  float* v_up = slice + SL;
  float* v_g = slice + 2 * SL;
  const bool has_lo = l > 0, has_up = l < L - 1;
  const float s_lo = sc[2 * l], s_up = sc[2 * l + 1];
  for (int i = lane; i < SL; i += 32) {
    if constexpr (CG) {
      v_lo[i] = (has_lo && i < m) ? __ldcg(d + (l - 1) * m + i) * s_lo : 0.0f;
      v_up[i] = (has_up && i < m) ? __ldcg(d + (l + 1) * m + i) * s_up : 0.0f;
    } else {
      v_lo[i] = (has_lo && i < m) ? d[(l - 1) * m + i] * s_lo : 0.0f;
      v_up[i] = (has_up && i < m) ? d[(l + 1) * m + i] * s_up : 0.0f;
    }
  }
  __syncwarp();
  float acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = 0.0f;
  if (has_lo) gemv_small<S, ROWS, BW>(acc, A + l * abs_, v_lo, m, lane);
  if (has_up) gemv_small<S, ROWS, BW>(acc, B + l * abs_, v_up, m, lane);
  small_combine<S, ROWS>(acc);
  const int r0 = E * (lane % LPC);
  const bool writer = lane < LPC && r0 < m;   // one lane per row group
  if (COUPLED) {
    if (writer)
#pragma unroll
      for (int e = 0; e < E; ++e) d[l * m + r0 + e] = acc[e] + q[l * m + r0 + e];
  } else {
    for (int i = lane; i < SL; i += 32) v_g[i] = 0.0f;
    __syncwarp();
    if (writer)
#pragma unroll
      for (int e = 0; e < E; ++e) v_g[r0 + e] = acc[e];
    __syncwarp();
    constexpr int LPC2 = SmallLp<float, ROWS>::LPC;
    float acc2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    gemv_small<float, ROWS>(acc2, C + l * cbs, v_g, m, lane);
    small_combine<float, ROWS>(acc2);
    const int r2 = 4 * (lane % LPC2);
    if (lane < LPC2 && r2 < m)
#pragma unroll
      for (int e = 0; e < 4; ++e) d[l * m + r2 + e] = acc2[e] + q[l * m + r2 + e];
  }
  __syncwarp();
}

}  // namespace dev
}  // namespace mc
