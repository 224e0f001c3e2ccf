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
__device__ inline bool band_ldlt_f(float* Lb, float* invD, const int* pairs, int npair, int N, int bw, int ls = 0) {
  const int bw1 = ls > 0 ? ls : bw + 1;  // row stride (>= bw + 1)
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

// (A v)_q for a band of the T_H pencil (rows [q][d] = A(q, q - d), d = 0..bw, symmetric) in
// grid-row order with b unknowns per row: the 5-point stiffness and the 7-point mass have
// nonzeros only on the diagonals d = 0, 1, b, b + 1 (the W/E, S/N and SW/NE couplings), so
// the product takes 7 terms instead of 2 bw + 1. The terms are added in the order of the
// full band loop, so the result is the same bit for bit. b < 2 falls back to that loop.
__device__ __forceinline__ double coarse_band_mv(const double* A, int bw, int b, const double* v, int q, int N) {
  const long long bw1 = bw + 1;
  double s = A[q * bw1] * v[q];
  if (b < 2 || bw != b + 1) {
    for (int d = 1; d <= bw; ++d) {
      if (q - d >= 0) s += A[q * bw1 + d] * v[q - d];
      if (q + d < N) s += A[(q + d) * bw1 + d] * v[q + d];
    }
    return s;
  }
  if (q >= 1) s += A[q * bw1 + 1] * v[q - 1];
  if (q + 1 < N) s += A[(q + 1) * bw1 + 1] * v[q + 1];
  if (q >= b) s += A[q * bw1 + b] * v[q - b];
  if (q + b < N) s += A[(q + b) * bw1 + b] * v[q + b];
  if (q >= b + 1) s += A[q * bw1 + b + 1] * v[q - b - 1];
  if (q + b + 1 < N) s += A[(q + b + 1) * bw1 + b + 1] * v[q + b + 1];
  return s;
}

// Diagonal slot k = 0..3 of the nonzero diagonals d = 0, 1, b, b + 1 of the T_H pencil band.
__device__ __forceinline__ int coarse_band_diag(int k, int b) { return k < 2 ? k : b + (k - 2); }

// Asynchronous global -> shared copies (no registers held while in flight): 16 bytes (both
// addresses 16-byte aligned, cached in L2 only) or 8 bytes (8-byte aligned); wait_all
// returns once every copy this thread issued has landed (a barrier then publishes them).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Block LDL^T of the T_H pencil S = K_H - mu M_H by grid rows (FP32), for unknowns ordered
// r = (Y-1) b + (X-1): S is block tridiagonal with b x b diagonal blocks S_II (couplings
// W/E) and sub-diagonal blocks S_{I,I-1} holding only the S and SW couplings (row r: columns
// r and r - 1). With W_I = S_{I,I-1} P_{I-1}^{-1} and P_I = S_II - W_I S_{I,I-1}^T
// (P_0 = S_00), S = L P L^T with L unit block lower bidiagonal (L_{I,I-1} = W_I) and P block
// diagonal; the blocks are stored as BS x BS tiles (zero padded) with row stride BS + 4
// (blk_ld): rows start on 16-byte boundaries, so the solve reads a row as float4 vectors,
// and a quarter-warp reading 8 rows as float4 (or a warp reading one column per lane) hits
// distinct shared-memory banks. Pinv[I] = P_I^{-1}, W[I] and its transpose WT[I] (the
// backward sweep reads W_{I+1}^T by rows). Sparse S_{I,I-1} makes W_I and P_I O(b^2) each;
// P_I is inverted by warp 0 alone (Gauss-Jordan with warp shuffles; for BS = 16 lanes 0-15
// reduce the rows of P_I and lanes 16-31 carry the rows of the inverse). The band S(mu)
// (FP64, [r][d] = S(r, r-d)) is read from shared memory. `work` holds 2 tiles. Returns false
// (to all threads) if a pivot is not positive (S(mu) not positive definite); `flag` is a
// shared int. All tile pointers 16-byte aligned.
template <int BS>
__host__ __device__ constexpr int blk_ld() { return BS + 4; }
template <int BS>
__host__ __device__ constexpr int blk_tile() { return BS * (BS + 4); }

template <int BS>
__device__ bool block_ldlt_f(const double* Sb, int bw1, int b, int nb, float* Pinv, float* W, float* WT, float* work,
                             int* flag) {
  constexpr int T2 = BS * BS, LD = blk_ld<BS>(), TS = blk_tile<BS>();
  const int tid = threadIdx.x, nt = blockDim.x;
  float* A = work;        // P_I before inversion
  float* Sub = work + TS; // dense copy of S_{I,I-1} (rows r: cols r, r-1)
  auto s_at = [&](int i, int j) -> float {  // S(i, j) for |i - j| <= bw from the band
    return i >= j ? (float)Sb[(long long)i * bw1 + (i - j)] : (float)Sb[(long long)j * bw1 + (j - i)];
  };
  if (tid == 0) *flag = 1;
  for (int I = 0; I < nb; ++I) {
    const float* Pp = Pinv + (long long)(I - 1) * TS;
    float* Wi = W + (long long)I * TS;
    float* WTi = WT + (long long)I * TS;
    // S_{I,I-1} (two nonzeros per row) and W_I = S_{I,I-1} P_{I-1}^{-1}
    if (I > 0) {
      for (int q = tid; q < T2; q += nt) {
        const int r = q / BS, c = q % BS;
        float v = 0.f;
        if (r < b && c < b) {
          const int i = I * b + r, j = (I - 1) * b + c;
          if (c == r || c == r - 1) v = s_at(i, j);
        }
        Sub[r * LD + c] = v;
      }
      __syncthreads();
      for (int q = tid; q < T2; q += nt) {
        const int r = q / BS, c = q % BS;
        float v = Sub[r * LD + r] * Pp[r * LD + c];
        if (r > 0) v += Sub[r * LD + r - 1] * Pp[(r - 1) * LD + c];
        v = (r < b && c < b) ? v : 0.f;
        Wi[r * LD + c] = v;
        WTi[c * LD + r] = v;
      }
      __syncthreads();
    } else {
      for (int q = tid; q < T2; q += nt) Wi[(q / BS) * LD + q % BS] = WTi[(q / BS) * LD + q % BS] = 0.f;
    }
    // P_I = S_II - W_I S_{I,I-1}^T  ((S^T)_{kc} nonzero for k = c, c - 1... i.e. Sub[c][k], k in {c, c-1})
    for (int q = tid; q < T2; q += nt) {
      const int r = q / BS, c = q % BS;
      float v = 0.f;
      if (r < b && c < b) {
        const int i = I * b + r, j = I * b + c;
        if (r - c <= 1 && c - r <= 1) v = s_at(i, j);
        if (I > 0) {
          v -= Wi[r * LD + c] * Sub[c * LD + c];
          if (c > 0) v -= Wi[r * LD + c - 1] * Sub[c * LD + c - 1];
        }
      } else if (r == c) {
        v = 1.f;  // padding: identity keeps the inverse's padding at zero off the diagonal
      }
      A[r * LD + c] = v;
    }
    __syncthreads();
    if (tid < 32) {
      float* Pi = Pinv + (long long)I * TS;
      const int lane = tid;
      int ok = 1;
      if constexpr (BS == 16) {
        // lane r < 16 holds row r of A, lane 16 + r row r of the inverse (starts as I)
        const int r = lane & 15, hi = lane >> 4;
        float v[BS];
#pragma unroll
        for (int c = 0; c < BS; ++c) v[c] = hi ? (r == c ? 1.f : 0.f) : A[r * LD + c];
#pragma unroll
        for (int k = 0; k < BS; ++k) {
          const float pv = __shfl_sync(0xffffffffu, v[k], k);
          const float f = __shfl_sync(0xffffffffu, v[k], r);  // A(r, k) of the current step
          if (!(pv > 0.f)) ok = 0;
          // one update for every row: row r -= g (pivot row) with g = A(r, k) / p, and for the
          // pivot row itself g = (p - 1) / p, which leaves it divided by p; one FMA per entry.
          // The approximate reciprocal (a few ulp) suffices for a preconditioner's factors and
          // takes the rounding fix-up off the step's dependency chain.
          const float g = (r == k ? f - 1.f : f) * __fdividef(1.0f, pv);
#pragma unroll
          for (int c = 0; c < BS; ++c) v[c] = fmaf(-g, __shfl_sync(0xffffffffu, v[c], k + 16 * hi), v[c]);
        }
        if (hi)
#pragma unroll
          for (int c = 0; c < BS; ++c) Pi[r * LD + c] = (r < b && c < b) ? v[c] : 0.f;
      } else {
        // one row per lane: row r of A and of its inverse
        const int r = lane;
        float row[BS], inv_row[BS];
#pragma unroll
        for (int c = 0; c < BS; ++c) {
          row[c] = r < BS ? A[r * LD + c] : 0.f;
          inv_row[c] = (r == c) ? 1.f : 0.f;
        }
#pragma unroll
        for (int k = 0; k < BS; ++k) {
          const float pv = __shfl_sync(0xffffffffu, row[k], k);
          if (!(pv > 0.f)) ok = 0;
          const float ip = __fdividef(1.0f, pv);
          const float f = row[k];
#pragma unroll
          for (int c = 0; c < BS; ++c) {
            const float pr = __shfl_sync(0xffffffffu, row[c], k) * ip;
            const float pi = __shfl_sync(0xffffffffu, inv_row[c], k) * ip;
            row[c] = (r == k) ? pr : row[c] - f * pr;
            inv_row[c] = (r == k) ? pi : inv_row[c] - f * pi;
          }
        }
        if (r < BS)
#pragma unroll
          for (int c = 0; c < BS; ++c) Pi[r * LD + c] = (r < b && c < b) ? inv_row[c] : 0.f;
      }
      if (lane == 0 && !ok) *flag = 0;
    }
    __syncthreads();
    if (!*flag) return false;
  }
  return true;
}

// S x = y with the block factors (L_{I,I-1} = W_I, P_I^{-1}): forward
// u_I = y_I - W_I u_{I-1} in place in yp, backward x_I = P_I^{-1} u_I - W_{I+1}^T x_{I+1} into
// xp, by warp 0 (lane = row). yp and xp hold block I at [I * BS, I * BS + b) with the BS - b
// padding entries zero, 16-byte aligned; every row product is BS / 4 float4 loads of the
// tile row and BS / 4 broadcast float4 loads of the vector.
template <int BS>
__device__ __forceinline__ float blk_dot(const float* row, const float* v) {
  const float4* a4 = reinterpret_cast<const float4*>(row);
  const float4* v4 = reinterpret_cast<const float4*>(v);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int k = 0; k < BS / 4; ++k) {
    const float4 x = a4[k], y = v4[k];
    s0 = fmaf(x.x, y.x, s0);
    s1 = fmaf(x.y, y.y, s1);
    s2 = fmaf(x.z, y.z, s2);
    s3 = fmaf(x.w, y.w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// Half of a 16-wide tile row times a vector held one entry per lane (lane k and k + 16 hold
// entry k): lanes 0-15 take columns 0-7, lanes 16-31 columns 8-15 (row part a0, a1), the
// entries come by shuffles; the caller adds the two halves.
__device__ __forceinline__ float blk_hdot16(const float4 a0, const float4 a1, float v, int k0) {
  float s0 = a0.x * __shfl_sync(0xffffffffu, v, k0 + 0);
  float s1 = a0.y * __shfl_sync(0xffffffffu, v, k0 + 1);
  s0 = fmaf(a0.z, __shfl_sync(0xffffffffu, v, k0 + 2), s0);
  s1 = fmaf(a0.w, __shfl_sync(0xffffffffu, v, k0 + 3), s1);
  s0 = fmaf(a1.x, __shfl_sync(0xffffffffu, v, k0 + 4), s0);
  s1 = fmaf(a1.y, __shfl_sync(0xffffffffu, v, k0 + 5), s1);
  s0 = fmaf(a1.z, __shfl_sync(0xffffffffu, v, k0 + 6), s0);
  s1 = fmaf(a1.w, __shfl_sync(0xffffffffu, v, k0 + 7), s1);
  return s0 + s1;
}

template <int BS>
__device__ inline void block_solve_f(const float* Pinv, const float* W, const float* WT, float* yp, float* xp, int b,
                                     int nb) {
  if constexpr (BS == 16) {
    // 16-wide rows: the recurrence's vector stays in registers (lane r and r + 16 hold row r)
    // and moves by shuffles; each half-warp forms half of every row product, and the tile
    // rows of the next block are loaded one step ahead, so a step's critical path is the
    // shuffles, 4 FMAs and one exchange of the halves. Padding rows of every tile are zero,
    // so rows r >= b carry zeros without a test.
    if (threadIdx.x < 32) {
      constexpr int LD = blk_ld<16>(), TS = blk_tile<16>();
      const int lane = threadIdx.x, r = lane & 15, k0 = (lane >> 4) * 8;
      const bool wr = lane < 16 && r < b;
      auto row2 = [&](const float* tile, float4& a0, float4& a1) {
        const float4* p4 = reinterpret_cast<const float4*>(tile + r * LD + k0);
        a0 = p4[0];
        a1 = p4[1];
      };
      // forward: u_I = y_I - W_I u_{I-1}, u_I back into yp for the backward sweep
      float u = yp[r];
      float4 a0, a1;
      float yn = 0.f;
      if (nb > 1) {
        row2(W + TS, a0, a1);
        yn = yp[BS + r];
      }
      for (int I = 1; I < nb; ++I) {
        const float4 c0 = a0, c1 = a1;
        const float yc = yn;
        if (I + 1 < nb) {
          row2(W + (long long)(I + 1) * TS, a0, a1);
          yn = yp[(I + 1) * BS + r];
        }
        float s = blk_hdot16(c0, c1, u, k0);
        s += __shfl_xor_sync(0xffffffffu, s, 16);
        u = yc - s;
        if (wr) yp[I * BS + r] = u;
      }
      __syncwarp();
      // backward: x_I = P_I^{-1} u_I - W_{I+1}^T x_{I+1}; the P_I^{-1} u_I half products are
      // off the recurrence and formed one step ahead
      auto pu_half = [&](int I) {
        float4 p0, p1;
        row2(Pinv + (long long)I * TS, p0, p1);
        const float4* v4 = reinterpret_cast<const float4*>(yp + I * BS + k0);
        const float4 v0 = v4[0], v1 = v4[1];
        float s0 = p0.x * v0.x, s1 = p0.y * v0.y;
        s0 = fmaf(p0.z, v0.z, s0);
        s1 = fmaf(p0.w, v0.w, s1);
        s0 = fmaf(p1.x, v1.x, s0);
        s1 = fmaf(p1.y, v1.y, s1);
        s0 = fmaf(p1.z, v1.z, s0);
        s1 = fmaf(p1.w, v1.w, s1);
        return s0 + s1;
      };
      float x = 0.f;
      float pn = pu_half(nb - 1);
      for (int I = nb - 1; I >= 0; --I) {
        float s = pn;
        float4 t0, t1;
        if (I + 1 < nb) row2(WT + (long long)(I + 1) * TS, t0, t1);
        if (I > 0) pn = pu_half(I - 1);
        if (I + 1 < nb) s -= blk_hdot16(t0, t1, x, k0);
        s += __shfl_xor_sync(0xffffffffu, s, 16);
        x = s;
        if (wr) xp[I * BS + r] = x;
      }
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x < 32) {
    constexpr int LD = blk_ld<BS>(), TS = blk_tile<BS>();
    const int r = threadIdx.x;
    for (int I = 1; I < nb; ++I) {
      if (r < b) yp[I * BS + r] -= blk_dot<BS>(W + (long long)I * TS + r * LD, yp + (I - 1) * BS);
      __syncwarp();
    }
    for (int I = nb - 1; I >= 0; --I) {
      if (r < b) {
        float v = blk_dot<BS>(Pinv + (long long)I * TS + r * LD, yp + I * BS);
        if (I + 1 < nb) v -= blk_dot<BS>(WT + (long long)(I + 1) * TS + r * LD, xp + (I + 1) * BS);
        xp[I * BS + r] = v;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// Factors of S(sigma) = K_H - sigma M_H for the Rayleigh-Ritz step of level L, prepared by
// one block of the inner-product kernel of the same level (which runs just before the
// Rayleigh-Ritz kernel and reads neither input nor output of this). sigma extrapolates the
// eigenvalues of the earlier levels: with d1 = lambda_{L-2} - lambda_{L-1} and
// d2 = lambda_{L-3} - lambda_{L-2} the differences shrink by r = d2 / d1 per level, so
// lambda_L ~ lambda_{L-1} - d1 / r. Only a regular sequence (2 <= r <= 8, as for the O(h^2)
// and corner-limited rates) is used. Level 3 has only d1 and takes r = 4, the O(h^2) rate of
// a smooth eigenfunction (on a re-entrant corner the rate is lower and sigma lands a little
// above lambda_3, which slows the refinement but keeps S(sigma) positive definite while
// sigma stays below the coarse eigenvalue). The Rayleigh-Ritz kernel refines against these
// factors and refactors at its own mu if the refinement stalls. `out` holds the layout of
// mlev_rr_prefactor_stride; `sm` is dynamic shared memory of rr_prefactor_smem bytes.
// Called by all threads of the block. Only for 16-wide row blocks (b <= 16): the 32-wide
// Gauss-Jordan would raise the register count of every block of the host kernel.
__device__ inline void rr_prefactor_block(const double* KH, const double* MH, const double* lamp, int L, int nhb,
                                          int bw, unsigned char* out, double* sm, int* flag) {
  constexpr int BS = 16, TS = BS * (BS + 4);
  const int N = nhb, bw1 = bw + 1, bsz = bw - 1, nbk = N / bsz;
  double sigma = NAN;
  bool use = L >= 3 && bsz <= BS;
  if (use) {
    const double l1 = lamp[L - 1], l2 = lamp[L - 2];
    const double d1 = l2 - l1;
    double r = 4.0;
    bool regular = true;
    if (L >= 4) {
      const double d2 = lamp[L - 3] - l2;
      r = d2 / d1;
      regular = d2 > 0.0 && r >= 2.0 && r <= 8.0;
    }
    use = d1 > 0.0 && regular;
    sigma = l1 - d1 / r;
  }
  if (!use) {
    if (threadIdx.x == 0) *reinterpret_cast<int*>(out + 8) = 0;
    return;
  }
  double* sb = sm;  // S(sigma), FP64 band; then P_I^{-1}, W_I and W_I^T tiles (16-byte aligned)
  float* tiles = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sb + (long long)N * bw1) + 15) & ~uintptr_t(15));
  float* work = tiles + 3LL * nbk * TS;
  for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) sb[q] = KH[q] - sigma * MH[q];
  __syncthreads();
  float* W = tiles + (long long)nbk * TS;
  const bool ok = block_ldlt_f<BS>(sb, bw1, bsz, nbk, tiles, W, W + (long long)nbk * TS, work, flag);
  float* dst = reinterpret_cast<float*>(out + 16);
  if (ok)
    for (long long q = threadIdx.x; q < 3LL * nbk * TS; q += blockDim.x) dst[q] = tiles[q];
  if (threadIdx.x == 0) {
    *reinterpret_cast<double*>(out) = sigma;
    *reinterpret_cast<int*>(out + 8) = ok ? 1 : 0;
  }
}

}  // namespace mlev
