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
// One CTA per level; A and X live in shared memory (m <= 112).  Every step
// ends with a CTA barrier; all loops are bounded.
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

// Blocked LU and inverse for blocks too large for shared memory (m > 112):
// one 512-thread CTA per level, column panels of kB = 32.
//   LU (right-looking): factor the panel (rows p0..m-1) in shared memory,
//   solve U12 = L11^{-1} A12 in shared memory, update the trailing block
//   A22 -= L21 U12 in place.
//   Inverse: X = U^{-1} L^{-1} one identity column panel at a time, kept in
//   shared memory: forward substitution by row panels (triangle by a warp per
//   right-hand side, rows below by a panel product), then backward
//   substitution the same way; the panel is stored as -X = (-T_dd)^{-1}.
constexpr int kB = 32, kLd = 256, kLdU = kB + 1, kBigThreads = 512;

__global__ void __launch_bounds__(kBigThreads, 1) k_factor_big(const double* __restrict__ tdd,
                                                               double* lu, double* ninv,
                                                               int64_t L, int m, int ms,
                                                               Header* hdr) {
  extern __shared__ double sm[];
  double* Pan = sm;                  // panel / right-hand sides: [kB][kLd]
  double* U12 = sm + kB * kLd;       // U12 block: [column][kLdU]
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int nwarp = nt >> 5;
  const int np = (m + kB - 1) / kB;
  for (int64_t l = blockIdx.x; l < L; l += gridDim.x) {
    double* A = lu + (size_t)l * ms;
    double* X = ninv + (size_t)l * ms;
    const double* T = tdd + (size_t)l * ms;
    for (int e = tid; e < m * m; e += nt) A[e] = T[e];
    __syncthreads();
    bool ok = true;
    for (int p = 0; p < np && ok; ++p) {
      const int p0 = p * kB, w = min(kB, m - p0), nr = m - p0;
      for (int e = tid; e < w * nr; e += nt) {
        const int k = e / nr, i = e % nr;
        Pan[k * kLd + i] = A[(size_t)(p0 + k) * m + p0 + i];
      }
      __syncthreads();
      for (int k = 0; k < w; ++k) {
        const double piv = Pan[k * kLd + k];
        if (!(piv != 0.0) || !isfinite(piv)) { ok = false; break; }
        for (int i = k + 1 + tid; i < nr; i += nt) Pan[k * kLd + i] = Pan[k * kLd + i] / piv;
        __syncthreads();
        const int nc = w - k - 1, nrr = nr - k - 1;
        for (int e = tid; e < nc * nrr; e += nt) {
          const int j = k + 1 + e / nrr, i = k + 1 + e % nrr;
          Pan[j * kLd + i] = fma(-Pan[k * kLd + i], Pan[j * kLd + k], Pan[j * kLd + i]);
        }
        __syncthreads();
      }
      if (!ok) break;
      for (int e = tid; e < w * nr; e += nt) {
        const int k = e / nr, i = e % nr;
        A[(size_t)(p0 + k) * m + p0 + i] = Pan[k * kLd + i];
      }
      const int nc2 = m - p0 - w;
      if (nc2 > 0) {
        for (int e = tid; e < w * nc2; e += nt) {
          const int c = e / w, k = e % w;
          U12[c * kLdU + k] = A[(size_t)(p0 + w + c) * m + p0 + k];
        }
        __syncthreads();
        for (int c = tid; c < nc2; c += nt) {
          double* u = U12 + c * kLdU;
          for (int k = 0; k < w; ++k) {
            const double uk = u[k];
            for (int i = k + 1; i < w; ++i) u[i] = fma(-Pan[k * kLd + i], uk, u[i]);
          }
        }
        __syncthreads();
        for (int e = tid; e < w * nc2; e += nt) {
          const int c = e / w, k = e % w;
          A[(size_t)(p0 + w + c) * m + p0 + k] = U12[c * kLdU + k];
        }
        for (int e = tid; e < nc2 * nc2; e += nt) {
          const int i = e % nc2, j = e / nc2;
          double acc = 0.0;
          for (int k = 0; k < w; ++k) acc = fma(Pan[k * kLd + w + i], U12[j * kLdU + k], acc);
          double* a = A + (size_t)(p0 + w + j) * m + p0 + w + i;
          *a = *a - acc;
        }
      }
      __syncthreads();
    }
    if (!ok) {
      if (tid == 0) latch(hdr, MC_ERR_SINGULAR_BLOCK);
      __syncthreads();
      continue;
    }
    for (int c = 0; c < np; ++c) {
      const int c0 = c * kB, wc = min(kB, m - c0);
      double* Y = Pan;
      for (int e = tid; e < wc * m; e += nt) {
        const int j = e / m, i = e % m;
        Y[j * kLd + i] = (i == c0 + j) ? 1.0 : 0.0;
      }
      __syncthreads();
      // forward: L Y = E (rows above c0 stay zero)
      for (int p = c; p < np; ++p) {
        const int p0 = p * kB, w = min(kB, m - p0);
        for (int j = wid; j < wc; j += nwarp) {
          double y = lane < w ? Y[j * kLd + p0 + lane] : 0.0;
          for (int k = 0; k < w; ++k) {
            const double yk = __shfl_sync(0xffffffffu, y, k);
            if (lane > k && lane < w) y = fma(-A[(size_t)(p0 + k) * m + p0 + lane], yk, y);
          }
          if (lane < w) Y[j * kLd + p0 + lane] = y;
        }
        __syncthreads();
        const int nb2 = m - p0 - w;
        for (int e = tid; e < nb2 * wc; e += nt) {
          const int i = e % nb2, j = e / nb2;
          double acc = 0.0;
          for (int k = 0; k < w; ++k)
            acc = fma(A[(size_t)(p0 + k) * m + p0 + w + i], Y[j * kLd + p0 + k], acc);
          Y[j * kLd + p0 + w + i] -= acc;
        }
        __syncthreads();
      }
      // backward: U X = Y
      for (int p = np - 1; p >= 0; --p) {
        const int p0 = p * kB, w = min(kB, m - p0);
        for (int j = wid; j < wc; j += nwarp) {
          double y = lane < w ? Y[j * kLd + p0 + lane] : 0.0;
          for (int k = w - 1; k >= 0; --k) {
            double xk = 0.0;
            if (lane == k) xk = y / A[(size_t)(p0 + k) * m + p0 + k];
            xk = __shfl_sync(0xffffffffu, xk, k);
            if (lane == k) y = xk;
            if (lane < k) y = fma(-A[(size_t)(p0 + k) * m + p0 + lane], xk, y);
          }
          if (lane < w) Y[j * kLd + p0 + lane] = y;
        }
        __syncthreads();
        for (int e = tid; e < p0 * wc; e += nt) {
          const int i = e % p0, j = e / p0;
          double acc = 0.0;
          for (int k = 0; k < w; ++k) acc = fma(A[(size_t)(p0 + k) * m + i], Y[j * kLd + p0 + k], acc);
          Y[j * kLd + i] -= acc;
        }
        __syncthreads();
      }
      for (int e = tid; e < wc * m; e += nt) {
        const int j = e / m, i = e % m;
        X[(size_t)(c0 + j) * m + i] = -Y[j * kLd + i];
      }
      __syncthreads();
    }
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

// Zero quadrants of a paired pentadiagonal chain (column-major blocks):
// TLO rows h.. of columns ..h and TUP rows ..h of columns h.., h = m/2.
__global__ void k_check_paired(const double* __restrict__ tlo, const double* __restrict__ tup,
                               int64_t L, int m, int ms, Header* hdr) {
  const int h = m / 2;
  const int64_t per = (int64_t)h * h;
  const int64_t total = L * per;
  bool bad = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / per, e = t % per;
    const int a = (int)(e / h), b = (int)(e % h);   // column a, row b of the quadrant
    bad |= tlo[(size_t)l * ms + (size_t)a * m + h + b] != 0.0;
    bad |= tup[(size_t)l * ms + (size_t)(h + a) * m + b] != 0.0;
  }
  if (bad) latch(hdr, MC_ERR_ARG);
}

__global__ void k_layout_diag(const double* __restrict__ diag, int d, double* __restrict__ plane,
                              int64_t L, int m, int ms) {
  const int64_t mm = (int64_t)m * m;
  const int64_t total = L * ms;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = t / ms, e = t % ms, k = l + d;
    plane[t] = (e < mm && k >= 0 && k < L) ? diag[k * mm + e] : 0.0;
  }
}

}  // namespace

cudaError_t launch_layout_diag(const double* diag, int d, double* plane, const Layout& lay,
                               cudaStream_t s) {
  const int64_t total = lay.L * lay.ms;
  int nb = (int)((total + 255) / 256);
  if (nb > 4096) nb = 4096;
  k_layout_diag<<<nb, 256, 0, s>>>(diag, d, plane, lay.L, lay.m, lay.ms);
  return cudaGetLastError();
}

cudaError_t launch_check_paired(const double* tlo, const double* tup, const Layout& lay,
                                Header* hdr, cudaStream_t s) {
  k_check_paired<<<1024, 256, 0, s>>>(tlo, tup, lay.L, lay.m, lay.ms, hdr);
  return cudaGetLastError();
}

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
    const size_t bsm = sizeof(double) * (size_t)(kB * kLd + kLd * kLdU);
    cudaError_t e = cudaFuncSetAttribute(k_factor_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bsm);
    if (e != cudaSuccess) return e;
    int nbb = num_sms;
    if (nbb > lay.L) nbb = (int)lay.L;
    k_factor_big<<<nbb, kBigThreads, bsm, s>>>(planes + kPlaneTDD * pe, planes + kPlaneLU * pe,
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
