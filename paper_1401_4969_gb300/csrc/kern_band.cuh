// Banded LDL^T solves on one thread block for the coarse pencil S(mu) = K_H - mu M_H
// (symmetric band storage, row-major [r][d] = S(r, r-d), half bandwidth bw). Used by the
// Rayleigh-Ritz step of Algorithm 4.1 and by its adjoint.
#pragma once

#include "kern_common.cuh"

namespace mlev {

// Band LDL^T factorisation of S = K_H - mu M_H (row-major band [r][d] = S(r, r-d)) with
// the right-hand side eliminated alongside (forward substitution of L z = w), one block
// barrier per column. On return Lb holds the unscaled columns (L(i,j) = Lb[i][i-j] / D_j),
// invD[j] = 1 / D_j and y = z. Returns false (to all threads) if a pivot is not positive,
// i.e. mu is not below the smallest eigenvalue of (K_H, M_H).
__device__ inline bool band_ldlt(double* Lb, double* invD, double* y, const int* pairs, int npair, int N, int bw,
                          int* flag) {
  const int bw1 = bw + 1;
  if (threadIdx.x == 0) *flag = 1;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    const double Dj = Lb[(long long)j * bw1];
    if (!(Dj > 0.0)) {  // identical decision in every thread
      if (threadIdx.x == 0) *flag = 0;
      return false;
    }
    const double inv = 1.0 / Dj;
    const int last = min(N - 1, j + bw);
    const double yj = y[j];
    for (int q = threadIdx.x; q < npair + bw; q += blockDim.x) {
      if (q < npair) {
        const int aa = pairs[q] >> 16, bb = pairs[q] & 0xffff;
        const int i = j + 1 + aa, k = j + 1 + bb;
        if (i <= last)
          Lb[(long long)i * bw1 + (i - k)] -= Lb[(long long)i * bw1 + (i - j)] * Lb[(long long)k * bw1 + (k - j)] * inv;
      } else {
        const int i = j + 1 + (q - npair);
        if (i <= last) y[i] -= Lb[(long long)i * bw1 + (i - j)] * inv * yj;
      }
    }
    if (threadIdx.x == 0) invD[j] = inv;
    __syncthreads();
  }
  return true;
}

// Back substitution L^T x = D^{-1} z in place (x overwrites y), warp 0, column-oriented.
__device__ inline void band_back(const double* Lb, const double* invD, double* y, int N, int bw) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, bw1 = bw + 1;
    for (int i = N - 1; i >= 0; --i) {
      const double xi = y[i] * invD[i];
      __syncwarp();
      if (lane == 0) y[i] = xi;
      // remove x_i from the rows above it: z[i-d] -= L(i, i-d) D_{i-d} x_i = Lb[i][d] x_i
      for (int d = 1 + lane; d <= bw && i - d >= 0; d += 32) y[i - d] -= Lb[(long long)i * bw1 + d] * xi;
      __syncwarp();
    }
  }
  __syncthreads();
}

// Forward substitution L z = b in place (unit lower L with L(i, j) = Lb[i][i-j] / D_j),
// warp 0, column-oriented; pair with band_back to finish S x = b.
__device__ __forceinline__ void band_fwd(const double* Lb, const double* invD, double* y, int N, int bw) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, bw1 = bw + 1;
    for (int j = 0; j < N; ++j) {
      const double yj = y[j] * invD[j];
      __syncwarp();
      for (int d = 1 + lane; d <= bw && j + d < N; d += 32) y[j + d] -= Lb[(long long)(j + d) * bw1 + d] * yj;
      __syncwarp();
    }
  }
  __syncthreads();
}

}  // namespace mlev
