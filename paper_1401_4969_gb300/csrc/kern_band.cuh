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

// FP32 band LDL^T of S (no right-hand side), same storage and schedule as band_ldlt (one
// block barrier per column; a thread keeps its (i - j, k - j) pair for every column, which
// needs npair <= blockDim.x). The pivots' reciprocals are the fast approximate ones: the
// factors only precondition FP64 iterative refinement. Returns false (to all threads) on a
// non-positive pivot.
__device__ inline bool band_ldlt_f(float* Lb, float* invD, const int* pairs, int npair, int N, int bw) {
  const int bw1 = bw + 1;
  const bool mine = threadIdx.x < npair;
  const int aa = mine ? pairs[threadIdx.x] >> 16 : 0, bb = mine ? pairs[threadIdx.x] & 0xffff : 0;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    const float Dj = Lb[j * bw1];
    if (!(Dj > 0.f)) return false;  // identical decision in every thread
    const float inv = __fdividef(1.0f, Dj);
    const int i = j + 1 + aa, k = j + 1 + bb;
    if (mine && i <= min(N - 1, j + bw))
      Lb[i * bw1 + (i - k)] -= Lb[i * bw1 + (i - j)] * Lb[k * bw1 + (k - j)] * inv;
    if (threadIdx.x == 0) invD[j] = inv;
    __syncthreads();
  }
  return true;
}

// S x = b in place with FP32 factors whose off-diagonal band entries were pre-scaled to
// L(i, i-d) = Ls[i * ls + d], by warp 0 with the active part of the right-hand side in
// registers (needs bw <= 31). Entry e lives in lane e mod 32; at column j the head lane
// j mod 32 holds the final z_j, every lane holding an entry j + d (1 <= d <= bw) subtracts
// L(j + d, j) z_j, and the head lane then takes entry j + 32. One shuffle per step. Back
// substitution runs the same way from the bottom with t = D^{-1} z.
__device__ inline void band_solve_shfl(const float* Ls, int ls, const float* invD, float* y, int N, int bw) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned full = 0xffffffffu;
    float v = lane < N ? y[lane] : 0.f;
#pragma unroll 4
    for (int j = 0; j < N; ++j) {
      // loads independent of v first; the head lane's refill and the store of z_j are
      // done without branching (every lane stores the same value)
      const int h = j & 31, d = (lane - j) & 31;
      const float coef = (d >= 1 && d <= bw && j + d < N) ? Ls[(j + d) * ls + d] : 0.f;
      const float refill = (j + 32 < N) ? y[j + 32] : 0.f;
      const float dj = invD[j];
      const float zj = __shfl_sync(full, v, h);
      v = (lane == h) ? refill : v - coef * zj;
      y[j] = zj * dj;
    }
    __syncwarp();
    // entry i lives in lane (N - 1 - i) mod 32; x_i final at the head, entries i - d take
    // the update -L(i, i - d) x_i
    v = (N - 1 - lane >= 0) ? y[N - 1 - lane] : 0.f;
#pragma unroll 4
    for (int i = N - 1; i >= 0; --i) {
      const int h = (N - 1 - i) & 31, d = (lane - (N - 1 - i)) & 31;
      const float coef = (d >= 1 && d <= bw && i - d >= 0) ? Ls[i * ls + d] : 0.f;
      const float refill = (i - 32 >= 0) ? y[i - 32] : 0.f;
      const float xi = __shfl_sync(full, v, h);
      v = (lane == h) ? refill : v - coef * xi;
      y[i] = xi;
    }
  }
  __syncthreads();
}

// Row-blocked form of the FP32 factors for the T_H band (unknown r = (Y-1) b + (X-1),
// b = ncx - 1 per grid row, half bandwidth b + 1): with that ordering L is block
// lower-bidiagonal (the band profile of a first node in a row stops one grid row back, so
// no fill reaches two blocks back). For nb = ncy - 1 blocks this stores, per block I, the
// dense inverse of the unit lower triangular diagonal block (Dinv, rows r >= c) and the
// sub-diagonal block Loff(r, c) = L(I b + r, (I - 1) b + c), each as a BS x BS tile padded
// with zeros (BS >= b), so the solve can load whole rows without guards. Needs the scaled
// factors Ls (L(i, i - d) = Ls[i * ls + d]).
template <int BS>
__device__ inline void band_blocks_f(const float* Ls, int ls, int bw, int b, int nb, float* Dinv, float* Loff) {
  constexpr int T2 = BS * BS;
  for (int q = threadIdx.x; q < nb * T2; q += blockDim.x) {
    const int I = q / T2, rc = q - I * T2, r = rc / BS, c = rc - r * BS;
    const int i = I * b + r, j = (I - 1) * b + c, d = i - j;
    Loff[q] = (I > 0 && r < b && c < b && d >= 1 && d <= bw) ? Ls[i * ls + d] : 0.f;
  }
  // column c of the diagonal block's inverse: z_r = delta_rc - sum_{c <= k < r} L(r, k) z_k
  for (int q = threadIdx.x; q < nb * BS; q += blockDim.x) {
    const int I = q / BS, c = q - I * BS;
    float* Z = Dinv + (long long)I * T2;
    for (int r = 0; r < BS; ++r) {
      float z = (r == c && c < b) ? 1.f : 0.f;
      if (c < b && r < b && r > c)
        for (int k = c; k < r; ++k) z -= Ls[(I * b + r) * ls + (r - k)] * Z[k * BS + c];
      Z[r * BS + c] = (c < b && r < b && r >= c) ? z : 0.f;
    }
  }
  __syncthreads();
}

// S x = y in place with the row-blocked factors: 2 nb block steps, each a b x b product
// and a b x b triangular product, instead of 2 N dependent scalar steps. Run by warp 0
// alone (b <= BS <= 32 lanes, one row of the block per lane) with warp barriers between
// steps. y must be followed by BS readable finite floats and t (BS floats) zero beyond b;
// the zero padding of the tiles cancels every out-of-block term.
template <int BS>
__device__ inline void band_solve_blocked(const float* Dinv, const float* Loff, const float* invD, float* y, float* t,
                                          int b, int nb) {
  if (threadIdx.x < 32) {
    constexpr int T2 = BS * BS;
    const int r = threadIdx.x;
    for (int I = 0; I < nb; ++I) {
      if (r < b) {
        float s0 = y[I * b + r], s1 = 0.f;
        if (I > 0) {
          const float* Lo = Loff + (long long)I * T2 + r * BS;
          const float* yp = y + (I - 1) * b;
#pragma unroll
          for (int c = 0; c < BS; c += 2) {
            s0 -= Lo[c] * yp[c];
            s1 -= Lo[c + 1] * yp[c + 1];
          }
        }
        t[r] = s0 + s1;
      }
      __syncwarp();
      if (r < b) {
        const float* Z = Dinv + (long long)I * T2 + r * BS;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int c = 0; c < BS; c += 2) {
          s0 += Z[c] * t[c];
          s1 += Z[c + 1] * t[c + 1];
        }
        y[I * b + r] = s0 + s1;
      }
      __syncwarp();
    }
    for (int q = r; q < nb * b; q += 32) y[q] *= invD[q];
    __syncwarp();
    for (int I = nb - 1; I >= 0; --I) {
      if (r < b) {
        float s0 = y[I * b + r], s1 = 0.f;
        if (I + 1 < nb) {
          const float* Lo = Loff + (long long)(I + 1) * T2;  // transpose: column r of block I + 1
          const float* xn = y + (I + 1) * b;
#pragma unroll
          for (int c = 0; c < BS; c += 2) {
            s0 -= Lo[c * BS + r] * xn[c];
            s1 -= Lo[(c + 1) * BS + r] * xn[c + 1];
          }
        }
        t[r] = s0 + s1;
      }
      __syncwarp();
      if (r < b) {
        const float* Z = Dinv + (long long)I * T2;  // transpose of the lower inverse
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int c = 0; c < BS; c += 2) {
          s0 += Z[c * BS + r] * t[c];
          s1 += Z[(c + 1) * BS + r] * t[c + 1];
        }
        y[I * b + r] = s0 + s1;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

}  // namespace mlev
