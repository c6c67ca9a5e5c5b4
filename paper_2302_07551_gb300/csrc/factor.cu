// Set-up kernels: block layout of Q^T, batched LU of the diagonal blocks and
// the operators that apply Q_{l,l}^{-1} in Algorithm 2 (steps 2 and 3).
#include <math.h>

#include "mc_internal.cuh"

namespace mc {

namespace {

// Planes TLO, TUP, TDD from the generator blocks (Sect. 2 block partition of
// Q^T).  A row-major Q block is the column-major storage of its transpose, so
// T_{l,l-1} = (Q_{l-1,l})^T is up[l-1] copied verbatim, T_{l,l+1} =
// (Q_{l+1,l})^T is dn[l+1], T_{l,l} = loc[l].  Missing boundary blocks and
// the padding beyond m*m are zero.
__global__ void k_layout(const double* __restrict__ dn, const double* __restrict__ loc,
                         const double* __restrict__ up, double* __restrict__ tlo,
                         double* __restrict__ tup, double* __restrict__ tdd, int64_t L, int m,
                         int ms) {
  const int64_t mm = (int64_t)m * m;
  const int64_t total = L * ms;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / ms, e = t % ms;
    double a = 0.0, b = 0.0, c = 0.0;
    if (e < mm) {
      if (l > 0) a = up[(l - 1) * mm + e];
      if (l < L - 1) b = dn[(l + 1) * mm + e];
      c = loc[l * mm + e];
    }
    tlo[t] = a;
    tup[t] = b;
    tdd[t] = c;
  }
}

// LU without pivoting of T_dd (column-major, in A), then X = T_dd^{-1} by
// forward and backward substitution on the identity, stored as -X = (-T_dd)^{-1}.
// One CTA per level; A and X live in shared memory (SMEM) or in the LU / NINV
// planes (large m).  Every step ends with a CTA barrier; all loops are bounded.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_lu_inv(const double* tdd, double* lu,
                                                double* ninv, int64_t L, int m, int ms,
                                                Header* hdr) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mm = m * m;
  for (int64_t l = blockIdx.x; l < L; l += gridDim.x) {
    double* A = SMEM ? sm : lu + (size_t)l * ms;
    double* X = SMEM ? sm + mm : ninv + (size_t)l * ms;
    const double* src = tdd + (size_t)l * ms;
    for (int e = tid; e < mm; e += nt) {
      A[e] = src[e];
      X[e] = (e % m == e / m) ? 1.0 : 0.0;
    }
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < m; ++k) {
      const double piv = A[k * m + k];
      if (!(piv != 0.0) || !isfinite(piv)) { bad = true; break; }
      for (int i = k + 1 + tid; i < m; i += nt) A[k * m + i] = A[k * m + i] / piv;
      __syncthreads();
      const int nr = m - k - 1;
      for (int idx = tid; idx < nr * nr; idx += nt) {
        const int i = k + 1 + idx % nr, j = k + 1 + idx / nr;
        A[j * m + i] = fma(-A[k * m + i], A[j * m + k], A[j * m + i]);
      }
      __syncthreads();
    }
    if (bad) {
      if (tid == 0) latch(hdr, MC_ERR_SINGULAR_BLOCK);
      __syncthreads();
      continue;
    }
    // X <- L^{-1} X (unit lower triangular, column oriented)
    for (int k = 0; k < m - 1; ++k) {
      const int nr = m - k - 1;
      for (int idx = tid; idx < nr * m; idx += nt) {
        const int i = k + 1 + idx % nr, c = idx / nr;
        X[c * m + i] = fma(-A[k * m + i], X[c * m + k], X[c * m + i]);
      }
      __syncthreads();
    }
    // X <- U^{-1} X
    for (int k = m - 1; k >= 0; --k) {
      const double ukk = A[k * m + k];
      for (int c = tid; c < m; c += nt) X[c * m + k] = X[c * m + k] / ukk;
      __syncthreads();
      for (int idx = tid; idx < k * m; idx += nt) {
        const int i = idx % k, c = idx / k;
        X[c * m + i] = fma(-A[k * m + i], X[c * m + k], X[c * m + i]);
      }
      __syncthreads();
    }
    double* dlu = lu + (size_t)l * ms;
    double* dni = ninv + (size_t)l * ms;
    for (int e = tid; e < mm; e += nt) {
      if (SMEM) dlu[e] = A[e];
      dni[e] = -X[e];
    }
    __syncthreads();
  }
}

// W = NINV * T for T in {TLO, TUP} (column-major, per level).
__global__ void __launch_bounds__(256) k_coupled(const double* __restrict__ ninv,
                                                 const double* __restrict__ tlo,
                                                 const double* __restrict__ tup,
                                                 double* __restrict__ wlo, double* __restrict__ wup,
                                                 int64_t L, int m, int ms) {
  const int mm = m * m;
  for (int64_t l = blockIdx.x; l < L; l += gridDim.x) {
    const double* Nl = ninv + (size_t)l * ms;
    for (int h = 0; h < 2; ++h) {
      const double* T = (h == 0 ? tlo : tup) + (size_t)l * ms;
      double* W = (h == 0 ? wlo : wup) + (size_t)l * ms;
      for (int e = threadIdx.x; e < mm; e += blockDim.x) {
        const int i = e % m, j = e / m;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(Nl[(size_t)k * m + i], T[(size_t)j * m + k], acc);
        W[e] = acc;
      }
    }
  }
}

}  // namespace

cudaError_t launch_layout(const double* dn, const double* loc, const double* up, double* planes,
                          const Layout& lay, Header*, cudaStream_t s) {
  const size_t pe = lay.plane_bytes / sizeof(double);
  const int64_t total = lay.L * lay.ms;
  int nb = (int)((total + 255) / 256);
  if (nb > 4096) nb = 4096;
  k_layout<<<nb, 256, 0, s>>>(dn, loc, up, planes + kPlaneTLO * pe, planes + kPlaneTUP * pe,
                              planes + kPlaneTDD * pe, lay.L, lay.m, lay.ms);
  return cudaGetLastError();
}

cudaError_t launch_factor(double* planes, const Layout& lay, Header* hdr, int coupled,
                          int num_sms, cudaStream_t s) {
  const size_t pe = lay.plane_bytes / sizeof(double);
  const int m = lay.m;
  int nb = num_sms * 4;
  if (nb > lay.L) nb = (int)lay.L;
  const size_t smem = 2 * sizeof(double) * (size_t)m * m;
  if (m <= 112) {
    cudaError_t e = cudaFuncSetAttribute(k_lu_inv<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_lu_inv<true><<<nb, 256, smem, s>>>(planes + kPlaneTDD * pe, planes + kPlaneLU * pe,
                                         planes + kPlaneNINV * pe, lay.L, m, lay.ms, hdr);
  } else {
    // copy TDD into the LU plane, factor in place in global memory
    cudaError_t e = cudaMemcpyAsync(planes + kPlaneLU * pe, planes + kPlaneTDD * pe,
                                    lay.plane_bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    k_lu_inv<false><<<nb, 256, 0, s>>>(planes + kPlaneLU * pe, planes + kPlaneLU * pe,
                                       planes + kPlaneNINV * pe, lay.L, m, lay.ms, hdr);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !coupled) return e;
  k_coupled<<<nb, 256, 0, s>>>(planes + kPlaneNINV * pe, planes + kPlaneTLO * pe,
                               planes + kPlaneTUP * pe, planes + kPlaneWLO * pe,
                               planes + kPlaneWUP * pe, lay.L, m, lay.ms);
  return cudaGetLastError();
}

}  // namespace mc
