// Several eigenpairs: the subspace form of Algorithms 4.1 / 4.2 (Section 4 states the
// correction for one simple eigenvalue and says the multiple-eigenvalue version follows in
// the same way; Section 6, Table 1, runs the first five). The q smallest eigenpairs of each
// problem are carried as q "virtual" batch members b q + i, so steps 1 and 2 of the
// correction (the local problems with lambda_i, the gluing and the G_{m+1} problem) and the
// per-member inner products run in the one-eigenpair kernels unchanged. This file adds:
//
// * k_band_level: the pencil (K_l, M_l) of level l in symmetric band storage (rows by grid
//   row, identity rows of K and zero rows of M for nodes on dOmega);
// * k_cross_gram: the Gram matrices a(u~_i, u~_j), b(u~_i, u~_j) of the q glued functions of
//   a problem, per T_H cell (deterministic partial sums);
// * k_border_prep: the bordered pencil of step 3 on V_{0H} + span{u~_1..u~_q}:
//   A = [[K_H, G_a], [G_a^T, A_q]], B = [[M_H, G_b], [G_b^T, B_q]];
// * k_sub_eig: the q smallest eigenpairs of a banded (optionally bordered) SPD pencil by block
//   subspace iteration with A^{-1} (FP32 band LDL^T plus iterative refinement) and
//   Rayleigh-Ritz on the block: the level-1 eigenproblem (Algorithm 4.2 step 1) and the
//   Rayleigh-Ritz step of Algorithm 4.1;
// * k_combine: u_i = sum_j D_ij u~_j, the eigenvector fields handed to the next level.
#include "kern_band.cuh"
#include "kern_coarse.cuh"
#include "kern_launch.h"

namespace mlev {

namespace {
__host__ __device__ __forceinline__ int mlidx(int l) { return l - MLEV_LMIN; }
}  // namespace

// Band pencil of level l (l >= 0) for real problem b (its coefficient is that of virtual
// member b q): row r = (Y - 1)(nx - 1) + (X - 1) for the interior lattice node (X, Y),
// entry [r][d] = A(r, r - d), d = 0..bw with bw = nx = ncx 2^l; the stiffness is the 5-point
// stencil of edge_weights, the mass (h^2 / 12)(6 on the diagonal, 1 to W, S, SW).
template <int KK>
__global__ void k_band_level(DevGeom G, int Breal, int q, int l, double* K, double* M) {
  const int nx = G.ncx << l, ny = G.ncy << l, nb = (nx - 1) * (ny - 1), bw = nx;
  const long long tot = (long long)Breal * nb;
  const double h = G.H * pow2(-l), h2 = h * h;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / nb), r = (int)(t % nb);
    const int X = r % (nx - 1) + 1, Y = r / (nx - 1) + 1;
    double* kr = K + ((long long)b * nb + r) * (bw + 1);
    double* mr = M + ((long long)b * nb + r) * (bw + 1);
    for (int d = 0; d <= bw; ++d) kr[d] = mr[d] = 0.0;
    if (!is_free(G, l, nx, ny, X, Y)) {
      kr[0] = 1.0;
      continue;
    }
    const W4 w = edge_weights<KK>(G.kap, b * q, l, X, Y);
    kr[0] = w.e + w.w + w.n + w.s;
    mr[0] = h2 / 2.0;
    if (X > 1 && is_free(G, l, nx, ny, X - 1, Y)) {
      kr[1] = -w.w;
      mr[1] = h2 / 12.0;
    }
    if (Y > 1 && is_free(G, l, nx, ny, X, Y - 1)) {
      kr[nx - 1] = -w.s;
      mr[nx - 1] = h2 / 12.0;
    }
    if (X > 1 && Y > 1 && is_free(G, l, nx, ny, X - 1, Y - 1)) mr[nx] = h2 / 12.0;
  }
}

// Gram matrices of the q glued functions u~_i of real problem b on level L, summed per T_H
// cell: one block of 256 threads per (problem, cell, pair a <= k) writes
// out[b][cell][pair][0] = sum over the cell's nodes of u~_a (K u~_k) (= a(u~_a, u~_k) after the
// cell sum) and [1] = sum of u~_a (M u~_k) (= b(u~_a, u~_k)); pairs in the order
// (0,0), (0,1), .., (0,q-1), (1,1), ...
template <int KK>
__global__ void __launch_bounds__(256) k_cross_gram(DevGeom G, GlobalLayout gl, int L, int q, const double* ut,
                                                    double* out) {
  __shared__ double scratch[8 * 2];
  __shared__ double sums[2];
  const int ncell = G.ncx * G.ncy, npair = q * (q + 1) / 2;
  const int pair = blockIdx.x % npair, cell = (blockIdx.x / npair) % ncell, b = blockIdx.x / (npair * ncell);
  int a = 0, rem = pair;
  while (rem >= q - a) {
    rem -= q - a;
    ++a;
  }
  const int k = a + rem;
  const int ci = cell % G.ncx, cj = cell / G.ncx;
  const int nx = gl.nx[mlidx(L)], ny = gl.ny[mlidx(L)], pitch = gl.pitch[mlidx(L)];
  const int S = 1 << L;
  const double h = G.H * pow2(-L), m12 = h * h / 12.0;
  const double* ua = ut + (long long)(b * q + a) * gl.bstride;
  const double* uk = ut + (long long)(b * q + k) * gl.bstride;
  double v[2] = {0.0, 0.0};
  if (G.cell_in[cj * G.ncx + ci]) {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
      const int i = (ci << L) + e % S, j = (cj << L) + e / S;
      if (!is_free(G, L, nx, ny, i, j)) continue;
      const long long c = (long long)j * pitch + i;
      const W4 w = edge_weights<KK>(G.kap, b * q, L, i, j);
      v[0] += ua[c] * apply_k<double, double>(uk, c, pitch, w);
      v[1] += ua[c] * (m12 * apply_m12<double, double>(uk, c, pitch));
    }
  }
  block_sum<2>(v, scratch, sums);
  if (threadIdx.x < 2) out[(((long long)b * ncell + cell) * npair + pair) * 2 + threadIdx.x] = sums[threadIdx.x];
}

// u_i = sum_j D[b][i][j] u~_j on level L for every real problem (fields of virtual members
// b q + j in `src`, results into the same members of `dst`; both global layouts).
__global__ void k_combine(GlobalLayout gl, int L, int Breal, int q, const double* D, const double* src, double* dst) {
  const int nx = gl.nx[mlidx(L)], ny = gl.ny[mlidx(L)], pitch = gl.pitch[mlidx(L)];
  const long long per = (long long)(ny + 1) * pitch;
  const long long tot = per * Breal;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    const long long c = t % per;
    if ((int)(c % pitch) > nx) continue;
    double v[MLEV_MAX_EIGENPAIRS];
    for (int j = 0; j < q; ++j) v[j] = src[(long long)(b * q + j) * gl.bstride + c];
    const double* Db = D + (long long)b * q * q;
    for (int i = 0; i < q; ++i) {
      double s = 0.0;
      for (int j = 0; j < q; ++j) s += Db[i * q + j] * v[j];
      dst[(long long)(b * q + i) * gl.bstride + c] = s;
    }
  }
}

namespace {

// Blocked form of the FP32 band factor K = L D L^T (half bandwidth < 32): rows in blocks of
// 32. Tile k (32 x 33 floats, row stride 33 so that a lane reading a row or a column of the
// tile hits its own bank) holds T_k = L_kk^{-1} below the diagonal (unit diagonal implicit)
// and the coupling C_k[i][m] = L(32 k + i, 32 (k - 1) + m) above it (nonzero only for m > i).
constexpr int kTB = 32;
constexpr int kTP = kTB + 1;
constexpr int kTT = kTB * kTP;
__host__ __device__ inline int sub_eig_nbk(int nb) { return (nb + kTB - 1) / kTB; }

// K~^{-1} y in place by one warp: z_k = T_k (y_k - C_k z_{k-1}) block by block, then
// x_k = T_k^T (D^{-1} z_k - C_{k+1}^T x_{k+1}) from the last block. Each block is two 32-term
// products (shuffles and FMAs) instead of 32 dependent substitution steps. y has 32 nbk
// entries, those past the last row zero.
__device__ void warp_block_solve(const float* tiles, const float* invD, float* y, int nbk) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  float zp = 0.f;
  for (int k = 0; k < nbk; ++k) {
    const float* Tr = tiles + (size_t)k * kTT + lane * kTP;  // row `lane` of tile k
    float t = y[k * kTB + lane];
    if (k > 0) {
      float t1 = 0.f;
#pragma unroll
      for (int m = 0; m < kTB; m += 2) {
        const float z0 = __shfl_sync(full, zp, m), z1 = __shfl_sync(full, zp, m + 1);
        t -= (m > lane ? Tr[m] : 0.f) * z0;
        t1 -= (m + 1 > lane ? Tr[m + 1] : 0.f) * z1;
      }
      t += t1;
    }
    float z = t, z1 = 0.f;
#pragma unroll
    for (int m = 0; m < kTB; m += 2) {
      const float t0 = __shfl_sync(full, t, m), tt = __shfl_sync(full, t, m + 1);
      z += (m < lane ? Tr[m] : 0.f) * t0;
      z1 += (m + 1 < lane ? Tr[m + 1] : 0.f) * tt;
    }
    z += z1;
    y[k * kTB + lane] = z * invD[k * kTB + lane];
    zp = z;
  }
  __syncwarp();
  float xn = 0.f;
  for (int k = nbk - 1; k >= 0; --k) {
    float sv = y[k * kTB + lane];
    if (k + 1 < nbk) {
      const float* Tn = tiles + (size_t)(k + 1) * kTT + lane;  // column `lane` of tile k + 1
      float s1 = 0.f;
#pragma unroll
      for (int m = 0; m < kTB; m += 2) {
        const float x0 = __shfl_sync(full, xn, m), x1 = __shfl_sync(full, xn, m + 1);
        sv -= (lane > m ? Tn[m * kTP] : 0.f) * x0;
        s1 -= (lane > m + 1 ? Tn[(m + 1) * kTP] : 0.f) * x1;
      }
      sv += s1;
    }
    const float* Tc = tiles + (size_t)k * kTT + lane;  // column `lane` of tile k
    float x = sv, x1 = 0.f;
#pragma unroll
    for (int m = 0; m < kTB; m += 2) {
      const float s0 = __shfl_sync(full, sv, m), s1 = __shfl_sync(full, sv, m + 1);
      x += (m > lane ? Tc[m * kTP] : 0.f) * s0;
      x1 += (m + 1 > lane ? Tc[(m + 1) * kTP] : 0.f) * s1;
    }
    x += x1;
    y[k * kTB + lane] = x;
    xn = x;
  }
  __syncwarp();
}

constexpr int kSMax = 16;  // largest block of the subspace iteration
constexpr int kCheck = 4;  // Rayleigh-Ritz (FP64 and the residual test in the FP64 phase) every kCheck-th step

// row stride of the FP32 band factor: bw + 1 rounded up to even (conflict-free coefficient loads)
__host__ __device__ inline int sub_eig_ls(int bwk) { return (bwk + 2) & ~1; }

// The s smallest eigenpairs of the s x s pencil (A, B) (FP64, row-major, symmetric, B SPD), by
// warp 0: B = L L^T, C = L^{-1} A L^{-T}, cyclic Jacobi on C in the round-robin order (s / 2
// disjoint rotations per round, lanes = rows / columns), W = L^{-T} V, all in precision R;
// then, in FP64, theta_c = w_c^T A w_c / w_c^T B w_c and w_c scaled to w_c^T B w_c = 1.
// Columns of W (row-major s x s, W[k * s + c]) in ascending order of theta. wk: 4 * 16 * 16 R.
template <typename R>
__device__ void small_eig_warp(int s, const double* A, const double* B, double* W, double* th, R* wk) {
  const int lane = threadIdx.x & 31;
  R* L = wk;
  R* C = wk + kSMax * kSMax;
  R* V = C + kSMax * kSMax;
  R* rot = V + kSMax * kSMax;  // per pair: c, s, p, q
  const int n2 = (s + 1) & ~1;
  // Cholesky, column by column
  for (int j = 0; j < s; ++j) {
    if (lane == 0) {
      R d = (R)B[j * s + j];
      for (int k = 0; k < j; ++k) d -= L[j * kSMax + k] * L[j * kSMax + k];
      L[j * kSMax + j] = sqrt(d > (R)0 ? d : (R)(sizeof(R) == 4 ? 1e-30 : 1e-300));
    }
    __syncwarp();
    if (lane > j && lane < s) {
      R v = (R)B[lane * s + j];
      for (int k = 0; k < j; ++k) v -= L[lane * kSMax + k] * L[j * kSMax + k];
      L[lane * kSMax + j] = v / L[j * kSMax + j];
    }
    __syncwarp();
  }
  // T = L^{-1} A (lane = column), then C = L^{-1} T^T (C symmetric)
  if (lane < s) {
    for (int i = 0; i < s; ++i) {
      R v = (R)A[i * s + lane];
      for (int k = 0; k < i; ++k) v -= L[i * kSMax + k] * C[k * kSMax + lane];
      C[i * kSMax + lane] = v / L[i * kSMax + i];
    }
  }
  __syncwarp();
  if (lane < s) {  // transpose of T into V (scratch), then the second solve into C
    for (int i = 0; i < s; ++i) V[lane * kSMax + i] = C[i * kSMax + lane];
  }
  __syncwarp();
  if (lane < s) {
    for (int i = 0; i < s; ++i) {
      R v = V[i * kSMax + lane];
      for (int k = 0; k < i; ++k) v -= L[i * kSMax + k] * C[k * kSMax + lane];
      C[i * kSMax + lane] = v / L[i * kSMax + i];
    }
  }
  __syncwarp();
  if (lane < s)
    for (int k = 0; k < s; ++k) V[lane * kSMax + k] = lane == k ? (R)1 : (R)0;
  __syncwarp();
  // Jacobi sweeps
  // stop when the off-diagonal part is below eps times the diagonal: above the rounding noise
  // the rotations leave behind (about sqrt(s (s - 1)) u |C|), which a tighter eps never gets
  // under, so that every call would run all 16 sweeps; Jacobi converges quadratically, so the
  // sweep that crosses eps usually lands far below it
  const R eps = sizeof(R) == 4 ? (R)1e-5 : (R)1e-12;
  for (int sweep = 0; sweep < 16; ++sweep) {
    R off = 0, dia = 0;
    if (lane < s)
      for (int k = 0; k < s; ++k) {
        const R v = C[lane * kSMax + k];
        if (k == lane) dia += v * v;
        else off += v * v;
      }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (!(off > eps * eps * dia)) break;
    for (int r = 0; r < n2 - 1; ++r) {
      if (lane < n2 / 2) {  // pair `lane` of round r (circle method; player n2 - 1 fixed)
        const int a = (r + lane) % (n2 - 1);
        const int b = lane == 0 ? n2 - 1 : (r - lane + n2 - 1) % (n2 - 1);
        const int p = a < b ? a : b, q = a < b ? b : a;
        R c = 1, sn = 0;
        if (q < s) {
          const R apq = C[p * kSMax + q];
          if (apq != (R)0) {
            const R theta = (C[q * kSMax + q] - C[p * kSMax + p]) / (2 * apq);
            const R t = (theta >= 0 ? (R)1 : (R)-1) / (fabs(theta) + sqrt(theta * theta + 1));
            c = 1 / sqrt(t * t + 1);
            sn = t * c;
          }
        }
        rot[lane * 4 + 0] = c;
        rot[lane * 4 + 1] = sn;
        rot[lane * 4 + 2] = (R)p;
        rot[lane * 4 + 3] = (R)q;
      }
      __syncwarp();
      if (lane < s)  // columns p, q of C and of V (lane = row)
        for (int k = 0; k < n2 / 2; ++k) {
          const int p = (int)rot[k * 4 + 2], q = (int)rot[k * 4 + 3];
          if (q >= s) continue;
          const R c = rot[k * 4 + 0], sn = rot[k * 4 + 1];
          const R cp = C[lane * kSMax + p], cq = C[lane * kSMax + q];
          C[lane * kSMax + p] = c * cp - sn * cq;
          C[lane * kSMax + q] = sn * cp + c * cq;
          const R vp = V[lane * kSMax + p], vq = V[lane * kSMax + q];
          V[lane * kSMax + p] = c * vp - sn * vq;
          V[lane * kSMax + q] = sn * vp + c * vq;
        }
      __syncwarp();
      if (lane < s)  // rows p, q of C (lane = column)
        for (int k = 0; k < n2 / 2; ++k) {
          const int p = (int)rot[k * 4 + 2], q = (int)rot[k * 4 + 3];
          if (q >= s) continue;
          const R c = rot[k * 4 + 0], sn = rot[k * 4 + 1];
          const R rp = C[p * kSMax + lane], rq = C[q * kSMax + lane];
          C[p * kSMax + lane] = c * rp - sn * rq;
          C[q * kSMax + lane] = sn * rp + c * rq;
        }
      __syncwarp();
    }
  }
  // W = L^{-T} V (lane = column), unsorted, in FP64
  if (lane < s) {
    for (int i = s - 1; i >= 0; --i) {
      R v = V[i * kSMax + lane];
      for (int k = i + 1; k < s; ++k) v -= L[k * kSMax + i] * (R)W[k * s + lane];
      W[i * s + lane] = (double)(v / L[i * kSMax + i]);
    }
  }
  __syncwarp();
  // FP64 Rayleigh quotients and B-normalisation (lane = column)
  double num = 0.0, den = 1.0;
  if (lane < s) {
    num = 0.0;
    den = 0.0;
    for (int i = 0; i < s; ++i)
      for (int k = 0; k < s; ++k) {
        num += W[i * s + lane] * A[i * s + k] * W[k * s + lane];
        den += W[i * s + lane] * B[i * s + k] * W[k * s + lane];
      }
  }
  const double scale = lane < s ? 1.0 / sqrt(den > 0.0 ? den : 1e-300) : 0.0;
  const double myth = lane < s ? num / den : 0.0;
  __syncwarp();
  if (lane < s)
    for (int i = 0; i < s; ++i) W[i * s + lane] *= scale;
  __syncwarp();
  // ascending order: rank of each column by theta (ties by index), then permute
  int rank = 0;
  for (int k = 0; k < s; ++k) {
    const double tk = __shfl_sync(0xffffffffu, myth, k);
    if (lane < s && (tk < myth || (tk == myth && k < lane))) ++rank;
  }
  double col[kSMax];
  if (lane < s)
    for (int i = 0; i < s; ++i) col[i] = W[i * s + lane];
  __syncwarp();
  if (lane < s) {
    for (int i = 0; i < s; ++i) W[i * s + rank] = col[i];
    th[rank] = myth;
  }
  __syncwarp();
}

}  // namespace

// Step 3's bordered pencil for real problem b on one level: from the per-cell inner products
// of the virtual members b q + i (k_aug: corner shares of g_a = P_H^T K u~, g_b = P_H^T M u~)
// and the cross Gram partials: Ga[b][i][r], Gb[b][i][r] for the T_H band rows r (0 on nodes of
// dOmega, whose rows are identity rows of K_H), Aq[b][i][j] = a(u~_i, u~_j), Bq = b(u~_i, u~_j).
// One block per real problem.
__global__ void k_border_prep(DevGeom G, int q, const double* partials, const double* cross, double* Ga, double* Gb,
                              double* Aq, double* Bq) {
  const int b = blockIdx.x, ncx = G.ncx, ncy = G.ncy, ncell = ncx * ncy, nb = (ncx - 1) * (ncy - 1);
  const int npair = q * (q + 1) / 2;
  for (int e = threadIdx.x; e < q * nb; e += blockDim.x) {
    const int i = e / nb, r = e % nb;
    const int X = r % (ncx - 1) + 1, Y = r / (ncx - 1) + 1;
    double sa = 0.0, sb = 0.0;
    if (is_free(G, 0, ncx, ncy, X, Y)) {
      const double* part = partials + (long long)(b * q + i) * ncell * 12;
      // node (X, Y) is corner 11 of cell (X-1, Y-1), 01 of (X, Y-1), 10 of (X-1, Y), 00 of (X, Y)
      const double* c11 = part + ((Y - 1) * ncx + (X - 1)) * 12;
      const double* c01 = part + ((Y - 1) * ncx + X) * 12;
      const double* c10 = part + (Y * ncx + (X - 1)) * 12;
      const double* c00 = part + (Y * ncx + X) * 12;
      sa = c00[3] + c10[4] + c01[5] + c11[6];
      sb = c00[7] + c10[8] + c01[9] + c11[10];
    }
    Ga[((long long)b * q + i) * nb + r] = sa;
    Gb[((long long)b * q + i) * nb + r] = sb;
  }
  for (int e = threadIdx.x; e < npair; e += blockDim.x) {
    int a = 0, rem = e;
    while (rem >= q - a) {
      rem -= q - a;
      ++a;
    }
    const int k = a + rem;
    double sa = 0.0, sb = 0.0;
    for (int c = 0; c < ncell; ++c) {  // fixed order: deterministic
      sa += cross[(((long long)b * ncell + c) * npair + e) * 2 + 0];
      sb += cross[(((long long)b * ncell + c) * npair + e) * 2 + 1];
    }
    Aq[((long long)b * q + a) * q + k] = Aq[((long long)b * q + k) * q + a] = sa;
    Bq[((long long)b * q + a) * q + k] = Bq[((long long)b * q + k) * q + a] = sb;
  }
}

// W = L^{-T} for B = L L^T (FP32, warp 0; W row-major s x s, W[k * s + c]): X = Y W has
// B-orthonormal columns to FP32 accuracy. Used between the Rayleigh-Ritz steps, where the
// block only has to stay well conditioned (span(X) = span(Y)). wk: 2 * 16 * 16 floats.
__device__ void chol_orth_warp(int s, const double* B, double* W, float* wk) {
  const int lane = threadIdx.x & 31;
  float* L = wk;
  float* Wt = wk + kSMax * kSMax;
  for (int j = 0; j < s; ++j) {
    if (lane == 0) {
      float d = (float)B[j * s + j];
      for (int k = 0; k < j; ++k) d -= L[j * kSMax + k] * L[j * kSMax + k];
      L[j * kSMax + j] = sqrtf(d > 0.f ? d : 1e-30f);
    }
    __syncwarp();
    if (lane > j && lane < s) {
      float v = (float)B[lane * s + j];
      for (int k = 0; k < j; ++k) v -= L[lane * kSMax + k] * L[j * kSMax + k];
      L[lane * kSMax + j] = v / L[j * kSMax + j];
    }
    __syncwarp();
  }
  if (lane < s) {  // column `lane` of L^{-T}: L^T w = e_lane, from the last row up
    for (int i = s - 1; i >= 0; --i) {
      float v = i == lane ? 1.f : 0.f;
      for (int k = i + 1; k < s; ++k) v -= L[k * kSMax + i] * Wt[k * kSMax + lane];
      Wt[i * kSMax + lane] = v / L[i * kSMax + i];
    }
  }
  __syncwarp();
  if (lane < s)
    for (int i = 0; i < s; ++i) W[i * s + lane] = (double)Wt[i * kSMax + lane];
  __syncwarp();
}

// A v and / or B v of the (bordered) pencil, all N = nb + nbord rows, by one warp (every lane
// calls it: the border rows are warp sums). Band rows: the band has nonzeros only on the
// diagonals 0, 1, nx - 1, nx (b = nx - 1 unknowns per grid row), plus the border columns.
// Only the requested products are formed (FP64 runs at a small fraction of the FP32 rate).
template <bool WA, bool WB>
__device__ void warp_pencil_apply(const SubEigArgs& a, int b, const double* K, const double* M, const double* Ga,
                                  const double* Gb, const double* v, double* av_out, double* bv_out) {
  const int lane = threadIdx.x & 31, nb = a.nb, nbd = a.nbord;
  double ga[MLEV_MAX_EIGENPAIRS], gb[MLEV_MAX_EIGENPAIRS];
  for (int i = 0; i < nbd; ++i) ga[i] = gb[i] = 0.0;
  for (int r = lane; r < nb; r += 32) {
    double av = WA ? coarse_band_mv(K, a.bwm, a.bwm - 1, v, r, nb) : 0.0;
    double bv = WB ? coarse_band_mv(M, a.bwm, a.bwm - 1, v, r, nb) : 0.0;
    for (int i = 0; i < nbd; ++i) {
      const double vb = v[nb + i], vr = v[r];
      if (WA) {
        av += Ga[(long long)i * nb + r] * vb;
        ga[i] += Ga[(long long)i * nb + r] * vr;
      }
      if (WB) {
        bv += Gb[(long long)i * nb + r] * vb;
        gb[i] += Gb[(long long)i * nb + r] * vr;
      }
    }
    if (WA) av_out[r] = av;
    if (WB) bv_out[r] = bv;
  }
  for (int i = 0; i < nbd; ++i)
    for (int o = 16; o > 0; o >>= 1) {
      if (WA) ga[i] += __shfl_xor_sync(0xffffffffu, ga[i], o);
      if (WB) gb[i] += __shfl_xor_sync(0xffffffffu, gb[i], o);
    }
  if (lane < nbd) {
    double av = 0.0, bv = 0.0;
    for (int i = 0; i < nbd; ++i)
      if (i == lane) {
        av = ga[i];
        bv = gb[i];
      }
    for (int j = 0; j < nbd; ++j) {
      if (WA) av += a.Aq[((long long)b * nbd + lane) * nbd + j] * v[nb + j];
      if (WB) bv += a.Bq[((long long)b * nbd + lane) * nbd + j] * v[nb + j];
    }
    if (WA) av_out[nb + lane] = av;
    if (WB) bv_out[nb + lane] = bv;
  }
  __syncwarp();
}

// y = A~^{-1} rhs (add: y += A~^{-1} rhs) by one warp, all N rows. A~ is A with the FP32
// factor of K (blocked form): t = K~^{-1} rhs_band, y_border = S^{-1} (rhs_border - G_a^T t) with the FP64
// Cholesky factor of the Schur complement S = A_q - G_a^T Z, y_band = t - Z y_border.
// yb: the warp's 32 nbk floats of shared scratch; w2: its nbord doubles.
__device__ void warp_bordered_solve(const SubEigArgs& a, const float* tiles, const float* invDf,
                                    const double* Ga, const double* Z, const double* Sq, double* w2, float* yb,
                                    const double* rhs, double* y, bool add) {
  const int lane = threadIdx.x & 31, nb = a.nb, nbd = a.nbord, nbk = sub_eig_nbk(nb);
  for (int r = lane; r < nbk * kTB; r += 32) yb[r] = r < nb ? (float)rhs[r] : 0.f;
  __syncwarp();
  warp_block_solve(tiles, invDf, yb, nbk);
  if (nbd) {
    double gt[MLEV_MAX_EIGENPAIRS];
    for (int i = 0; i < nbd; ++i) {
      double v = 0.0;
      for (int r = lane; r < nb; r += 32) v += Ga[(long long)i * nb + r] * (double)yb[r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      gt[i] = v;
    }
    if (lane == 0) {
      for (int i = 0; i < nbd; ++i) w2[i] = rhs[nb + i] - gt[i];
      for (int i = 0; i < nbd; ++i) {  // forward, then backward with the Cholesky factor
        double v = w2[i];
        for (int k = 0; k < i; ++k) v -= Sq[i * MLEV_MAX_EIGENPAIRS + k] * w2[k];
        w2[i] = v / Sq[i * MLEV_MAX_EIGENPAIRS + i];
      }
      for (int i = nbd - 1; i >= 0; --i) {
        double v = w2[i];
        for (int k = i + 1; k < nbd; ++k) v -= Sq[k * MLEV_MAX_EIGENPAIRS + i] * w2[k];
        w2[i] = v / Sq[i * MLEV_MAX_EIGENPAIRS + i];
      }
    }
    __syncwarp();
  }
  for (int r = lane; r < nb; r += 32) {
    double v = (double)yb[r];
    for (int i = 0; i < nbd; ++i) v -= Z[(long long)i * nb + r] * w2[i];
    y[r] = add ? y[r] + v : v;
  }
  if (lane < nbd) y[nb + lane] = add ? y[nb + lane] + w2[lane] : w2[lane];
  __syncwarp();
}

// The q smallest eigenpairs of a banded (bordered when nbord = q) SPD pencil (A, B), one block
// of 1024 threads per real problem: block subspace iteration X <- A^{-1} B X with the
// Rayleigh-Ritz step on the block (Algorithm 4.2 step 1 on V_{0h_1}, and Algorithm 4.1
// step 3 on V_{0H} + span{u~_1..u~_q}). A^{-1} uses the FP32 band LDL^T of K in shared memory
// (warp-parallel solves, one column per warp) and, with a border, the q x q Schur complement
// S = A_q - G_a^T K^{-1} G_a; the products A Y, B Y, the Gram matrices and the Ritz values are
// FP64. Columns of X live in global memory. The Rayleigh-Ritz step on the block runs every
// kCheck-th step; the steps between only B-orthonormalise it (Cholesky of Y^T B Y in FP32:
// the iteration's subspace is span(Y) either way). Two phases:
// * while the q wanted Ritz values change by more than tol (relative) between Rayleigh-Ritz
//   steps: one FP32-factor solve per column and FP32 Jacobi on the small pencil;
// * then two steps of iterative refinement against the FP64 pencil per solve, and at each
//   Rayleigh-Ritz step FP64 Jacobi and the residual test: stop when every wanted Ritz pair has
//   ||A x - theta B x||_2 <= rtol ||theta B x||_2. A stop on the Ritz values alone would leave
//   the vectors accurate only to about the square root of tol, and the correction steps carry
//   the level-1 vectors' error into lambda_{h_n}.
__global__ void __launch_bounds__(1024) k_sub_eig(DevGeom G, SubEigArgs a) {
  extern __shared__ __align__(16) unsigned char se_raw[];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int nb = a.nb, N = nb + a.nbord, s = a.s, ls = sub_eig_ls(a.bwk);
  const int npair = a.bwk * (a.bwk + 1) / 2;
  // shared layout: doubles first (8-byte aligned), then floats, then ints
  double* Ah = reinterpret_cast<double*>(se_raw);
  double* Bh = Ah + kSMax * kSMax;
  double* Wm = Bh + kSMax * kSMax;
  double* th = Wm + kSMax * kSMax;
  double* thp = th + kSMax;
  double* Sq = thp + kSMax;           // nbord x nbord Cholesky factor of the Schur complement
  double* y2 = Sq + MLEV_MAX_EIGENPAIRS * MLEV_MAX_EIGENPAIRS;  // per warp: nbord values
  double* wkd = y2 + 32 * MLEV_MAX_EIGENPAIRS;                    // small_eig workspace (4 * 256)
  // FP32 factor: the band (nb rows of ls floats) is factored at the end of the tile region and
  // converted block by block into the tiles, which never overwrite a band row not yet read
  const int nbk = sub_eig_nbk(nb), nb32 = nbk * kTB;
  float* tiles = reinterpret_cast<float*>(wkd + 4 * kSMax * kSMax);
  float* Lf = tiles + ((size_t)nbk * kTT - (size_t)nb * ls);
  float* invDf = tiles + (size_t)nbk * kTT;  // nb32 entries, 1 on the padding rows
  float* ybuf = invDf + nb32;                // s columns of nb32 floats
  int* pairs = reinterpret_cast<int*>(ybuf + (size_t)s * nb32);
  __shared__ int done, conv, phase2, hi_now, p2it;
  __shared__ double rpart[32], dpart[32], res_final;
  const double* K = a.K + (long long)b * a.kstride;
  const double* M = a.M + (long long)b * a.mstride;
  const double* Ga = a.Ga ? a.Ga + (long long)b * a.nbord * nb : nullptr;
  const double* Gb = a.Gb ? a.Gb + (long long)b * a.nbord * nb : nullptr;
  double* X = a.X + (long long)b * s * N;
  double* Y = a.Y + (long long)b * s * N;
  double* AY = a.AY + (long long)b * s * N;
  double* BY = a.BY + (long long)b * s * N;
  double* Z = a.Z ? a.Z + (long long)b * a.nbord * nb : nullptr;
  // ---- FP32 band LDL^T of K (half bandwidth bwk), pre-scaled to L(i, i - d)
  for (int e = tid; e < nb * ls; e += blockDim.x) {
    const int r = e / ls, d = e % ls;
    Lf[e] = d <= a.bwk ? (float)K[(long long)r * (a.bwm + 1) + d] : 0.f;
  }
  for (int e = tid; e < npair; e += blockDim.x) {
    int aa = 0;
    while ((aa + 1) * (aa + 2) / 2 <= e) ++aa;
    pairs[e] = (aa << 16) | (e - aa * (aa + 1) / 2);
  }
  __syncthreads();
  if (!band_ldlt_f(Lf, invDf, pairs, npair, nb, a.bwk, ls)) {
    if (tid == 0) atomicOr((unsigned long long*)&a.stat[(long long)b * a.q * a.stat_stride + MLEV_STAT_FLAGS],
                           (unsigned long long)MLEV_ST_RR_BREAKDOWN);
    return;
  }
  for (int e = tid; e < nb * ls; e += blockDim.x) {
    const int r = e / ls, d = e % ls;
    if (d >= 1 && r - d >= 0) Lf[e] *= invDf[r - d];
  }
  for (int r = nb + tid; r < nb32; r += blockDim.x) invDf[r] = 1.f;
  __syncthreads();
  // ---- blocked form (32 warps x 32 lanes: one thread per tile entry). Tile k is written at
  // [k kTT, (k + 1) kTT), below the band rows of the blocks after k (the band region starts
  // nbk kTT - nb ls floats in, and ls <= 32 < kTP), so only block k's own rows can overlap:
  // they are read before the barrier, the tile written after it
  for (int k = 0; k < nbk; ++k) {
    auto Lkk = [&](int i, int j) {  // L(32 k + i, 32 k + j), j < i
      const int r = k * kTB + i, d = i - j;
      return (d <= a.bwk && r < nb) ? Lf[(size_t)r * ls + d] : 0.f;
    };
    // warp c: column c of T_k = L_kk^{-1} (lane i holds entry i): L_kk x = e_c
    float x = lane == warp ? 1.f : 0.f;
    for (int j = warp; j < kTB; ++j) {
      const float xj = __shfl_sync(0xffffffffu, x, j);
      if (lane > j) x -= Lkk(lane, j) * xj;
    }
    // thread (row warp, column lane): C_k[warp][lane] = L(32 k + warp, 32 (k - 1) + lane)
    float cpl = 0.f;
    {
      const int r = k * kTB + warp, d = kTB + warp - lane;
      if (k > 0 && lane > warp && d <= a.bwk && r < nb) cpl = Lf[(size_t)r * ls + d];
    }
    __syncthreads();
    float* T = tiles + (size_t)k * kTT;
    if (lane > warp) {
      T[lane * kTP + warp] = x;    // T_k[lane][warp], below the diagonal
      T[warp * kTP + lane] = cpl;  // C_k[warp][lane], above it
    } else if (lane == warp) {
      T[lane * kTP + lane] = 0.f;
    }
  }
  __syncthreads();
  // ---- border: Z_i = K^{-1} G_a,i (warp i), S = A_q - G_a^T Z, Cholesky (thread 0)
  const int nbd = a.nbord;
  if (nbd) {
    for (int i = warp; i < nbd; i += nwarp) {
      float* yb = ybuf + (size_t)i * nb32;
      for (int r = lane; r < nb32; r += 32) yb[r] = r < nb ? (float)Ga[(long long)i * nb + r] : 0.f;
      __syncwarp();
      warp_block_solve(tiles, invDf, yb, nbk);
      for (int r = lane; r < nb; r += 32) Z[(long long)i * nb + r] = (double)yb[r];
    }
    __syncthreads();
    for (int e = warp; e < nbd * nbd; e += nwarp) {
      const int i = e / nbd, j = e % nbd;
      double v = 0.0;
      for (int r = lane; r < nb; r += 32) v += Ga[(long long)i * nb + r] * Z[(long long)j * nb + r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) Sq[i * MLEV_MAX_EIGENPAIRS + j] = a.Aq[((long long)b * nbd + i) * nbd + j] - v;
    }
    __syncthreads();
    if (tid == 0) {  // in-place Cholesky of the symmetric part (lower triangle)
      for (int j = 0; j < nbd; ++j) {
        double d = 0.5 * (Sq[j * MLEV_MAX_EIGENPAIRS + j] + Sq[j * MLEV_MAX_EIGENPAIRS + j]);
        for (int k = 0; k < j; ++k) d -= Sq[j * MLEV_MAX_EIGENPAIRS + k] * Sq[j * MLEV_MAX_EIGENPAIRS + k];
        d = sqrt(d > 0.0 ? d : 1e-300);
        Sq[j * MLEV_MAX_EIGENPAIRS + j] = d;
        for (int i = j + 1; i < nbd; ++i) {
          double v = 0.5 * (Sq[i * MLEV_MAX_EIGENPAIRS + j] + Sq[j * MLEV_MAX_EIGENPAIRS + i]);
          for (int k = 0; k < j; ++k) v -= Sq[i * MLEV_MAX_EIGENPAIRS + k] * Sq[j * MLEV_MAX_EIGENPAIRS + k];
          Sq[i * MLEV_MAX_EIGENPAIRS + j] = v / d;
        }
      }
    }
    __syncthreads();
  }
  // ---- start block: the border unit vectors (the u~_i themselves) then deterministic
  // pseudo-random columns, or pseudo-random columns only (level 1)
  for (long long e = tid; e < (long long)s * N; e += blockDim.x) {
    const int c = (int)(e / N), r = (int)(e % N);
    double v;
    if (a.init_border && c < a.q) v = (r == nb + c) ? 1.0 : 0.0;
    else if (r >= nb) v = 0.0;
    else {
      unsigned h = (unsigned)(r * 2654435761u) ^ (unsigned)((c + 1) * 40503u);
      h ^= h >> 13;
      h *= 0x5bd1e995u;
      h ^= h >> 15;
      v = (double)(h & 0xffffff) / 16777216.0 - 0.5;
    }
    X[e] = v;
  }
  if (tid < kSMax) thp[tid] = 0.0;
  if (tid == 0) {
    done = conv = phase2 = hi_now = p2it = 0;
    res_final = 0.0;
  }
  __syncthreads();
  int it = 0;
  for (; it < a.max_iter; ++it) {
    // Y = A^{-1} B X, column c by warp c (s <= 16 <= 32 warps): the FP32-factor solve, and in
    // the FP64 phase two steps of iterative refinement against the FP64 pencil,
    // y += A~^{-1} (B x - A y), so that the iteration converges to the invariant subspace of
    // A^{-1} B and not of A~^{-1} B (the factor's error is about u_32 cond(K) ~ 1e-5 on a
    // 32 x 32 level-1 grid, each step multiplies the solve error by it); BY and AY of the
    // column serve as scratch; then A Y and B Y in FP64
    const int nref = phase2 ? 2 : 0;
    // Rayleigh-Ritz (and A Y) only every kCheck-th step of either phase and at the cap; the
    // steps between only B-orthonormalise the block
    const bool rr_it = (phase2 ? (it - p2it) % kCheck == kCheck - 1 : it % kCheck == kCheck - 1) ||
                       it + 1 == a.max_iter;
    if (warp < s) {
      const double* x = X + (long long)warp * N;
      double* y = Y + (long long)warp * N;
      double* t1 = BY + (long long)warp * N;
      double* t2 = AY + (long long)warp * N;
      float* yb = ybuf + (size_t)warp * nb32;
      double* w2 = y2 + warp * MLEV_MAX_EIGENPAIRS;
      warp_pencil_apply<false, true>(a, b, K, M, Ga, Gb, x, nullptr, t1);
      warp_bordered_solve(a, tiles, invDf, Ga, Z, Sq, w2, yb, t1, y, false);
      for (int k = 0; k < nref; ++k) {
        warp_pencil_apply<true, false>(a, b, K, M, Ga, Gb, y, t2, nullptr);
        for (int r = lane; r < N; r += 32) t2[r] = t1[r] - t2[r];
        __syncwarp();
        warp_bordered_solve(a, tiles, invDf, Ga, Z, Sq, w2, yb, t2, y, true);
      }
      if (rr_it) warp_pencil_apply<true, true>(a, b, K, M, Ga, Gb, y, t2, t1);
      else warp_pencil_apply<false, true>(a, b, K, M, Ga, Gb, y, nullptr, t1);
    }
    __syncthreads();
    // Gram matrices Y^T A Y, Y^T B Y (FP64), entry pairs by warps
    for (int e = warp; e < s * s; e += nwarp) {
      const int i = e / s, j = e % s;
      if (j < i) continue;
      const double* yi = Y + (long long)i * N;
      const double* ayj = AY + (long long)j * N;
      const double* byj = BY + (long long)j * N;
      double va = 0.0, vb = 0.0;
      if (rr_it) {
        for (int r = lane; r < N; r += 32) {
          va += yi[r] * ayj[r];
          vb += yi[r] * byj[r];
        }
      } else {
        for (int r = lane; r < N; r += 32) vb += yi[r] * byj[r];
      }
      for (int o = 16; o > 0; o >>= 1) {
        va += __shfl_down_sync(0xffffffffu, va, o);
        vb += __shfl_down_sync(0xffffffffu, vb, o);
      }
      if (lane == 0) {
        Ah[i * s + j] = Ah[j * s + i] = va;
        Bh[i * s + j] = Bh[j * s + i] = vb;
      }
    }
    __syncthreads();
    // between Rayleigh-Ritz steps: B-orthonormalise the block; at them, FP32 Jacobi (it only
    // steers: X = Y W spans span(Y) for any invertible W) or, in the FP64 phase, FP64 Jacobi,
    // whose Ritz pairs the residual test then checks (FP64 arithmetic runs at a small fraction
    // of the FP32 rate: a Jacobi call costs more than a step's solves)
    if (warp == 0 && !rr_it) {
      chol_orth_warp(s, Bh, Wm, reinterpret_cast<float*>(wkd));
      if (lane == 0) hi_now = 0;
    } else if (warp == 0) {
      const bool hi = (phase2 && (it - p2it) % kCheck == kCheck - 1) || it + 1 == a.max_iter;
      if (hi) small_eig_warp<double>(s, Ah, Bh, Wm, th, wkd);
      else small_eig_warp<float>(s, Ah, Bh, Wm, th, reinterpret_cast<float*>(wkd));
      if (lane == 0) {
        double ch = 0.0;
        for (int i = 0; i < a.q; ++i) ch = fmax(ch, fabs(th[i] - thp[i]) / fabs(th[i]));
        for (int i = 0; i < s; ++i) thp[i] = th[i];
        hi_now = hi;
        if (!phase2 && it > 0 && ch <= a.tol) {
          phase2 = 1;
          p2it = it + 1;
        }
      }
    }
    __syncthreads();
    // X = Y W
    for (long long e = tid; e < (long long)s * N; e += blockDim.x) {
      const int c = (int)(e / N), r = (int)(e % N);
      double v = 0.0;
      for (int k = 0; k < s; ++k) v += Y[(long long)k * N + r] * Wm[k * s + c];
      X[e] = v;
    }
    // with FP64 Ritz vectors: the residuals ||A x_c - theta_c B x_c|| of the wanted pairs
    // (x_c = Y w_c, so A x_c = AY w_c), warp (chunk, c) over every nch-th row block of 32
    const int nch = nwarp / a.q;
    if (hi_now && warp < nch * a.q) {
      const int c = warp % a.q, chn = warp / a.q;
      double rr2 = 0.0, dd2 = 0.0;
      for (int r = chn * 32 + lane; r < N; r += nch * 32) {
        double ax = 0.0, bx = 0.0;
        for (int k = 0; k < s; ++k) {
          ax += AY[(long long)k * N + r] * Wm[k * s + c];
          bx += BY[(long long)k * N + r] * Wm[k * s + c];
        }
        const double t = ax - th[c] * bx;
        rr2 += t * t;
        dd2 += th[c] * th[c] * bx * bx;
      }
      for (int o = 16; o > 0; o >>= 1) {
        rr2 += __shfl_xor_sync(0xffffffffu, rr2, o);
        dd2 += __shfl_xor_sync(0xffffffffu, dd2, o);
      }
      if (lane == 0) {
        rpart[warp] = rr2;
        dpart[warp] = dd2;
      }
    }
    __syncthreads();
    if (tid == 0 && hi_now) {
      double worst = 0.0;
      for (int c = 0; c < a.q; ++c) {
        double rr2 = 0.0, dd2 = 0.0;
        for (int k = 0; k < nch; ++k) {  // fixed order: deterministic
          rr2 += rpart[k * a.q + c];
          dd2 += dpart[k * a.q + c];
        }
        worst = fmax(worst, sqrt(rr2 / (dd2 > 0.0 ? dd2 : 1e-300)));
      }
      res_final = worst;
      conv = worst <= a.rtol;
      done = conv || it + 1 == a.max_iter;
    }
    __syncthreads();
    if (done) break;
  }
  if (tid < s) a.theta[(long long)b * s + tid] = th[tid];
  if (tid == 0) {
    for (int i = 0; i < a.q; ++i) {
      long long* st = a.stat + (long long)(b * a.q + i) * a.stat_stride;
      st[a.it_slot] = it + 1;
      if (a.res_slot >= 0) st[a.res_slot] = (long long)__double_as_longlong(res_final);
      if (!conv) atomicOr((unsigned long long*)&st[MLEV_STAT_FLAGS], (unsigned long long)a.noconv_flag);
    }
  }
}

// Level-1 results of the q-eigenpair solve: virtual member b q + i gets u_{i,h_1} (column i of
// X, B-normalised) as its level-1 field, lambda_{i,h_1}, and the representation
// u = c0 u~ + P_H c with c0 = 1, c = 0.
__global__ void k_level1_multi_out(DevGeom G, GlobalLayout gl, int q, int s, const double* X, const double* theta,
                                   double* ut1, double* lam, int lam_stride, double* c, double* c0) {
  const int p = blockIdx.x, b = p / q, i = p % q;
  const int nx = gl.nx[mlidx(1)], ny = gl.ny[mlidx(1)], pitch = gl.pitch[mlidx(1)], nb = (nx - 1) * (ny - 1);
  const double* x = X + ((long long)b * s + i) * nb;
  double* u = ut1 + (long long)p * gl.bstride;
  for (int e = threadIdx.x; e < (ny + 1) * (nx + 1); e += blockDim.x) {
    const int X_ = e % (nx + 1), Y_ = e / (nx + 1);
    u[(long long)Y_ * pitch + X_] =
        is_free(G, 1, nx, ny, X_, Y_) ? x[(Y_ - 1) * (nx - 1) + (X_ - 1)] : 0.0;
  }
  const int ncoef = (G.ncx + 1) * (G.ncy + 1);
  for (int e = threadIdx.x; e < ncoef; e += blockDim.x) c[(long long)p * ncoef + e] = 0.0;
  if (threadIdx.x == 0) {
    c0[p] = 1.0;
    lam[(long long)p * lam_stride + 1] = theta[(long long)b * s + i];
  }
}

// Rayleigh-Ritz results on level L for real problem b: eigenvector i = [c_H; d] (column i of X)
// gives u_i = P_H c_H + sum_j d_j u~_j; its sign makes b(u_i, W) > 0 for the coarse function
// W = sum_k omega_k phi_k with omega = 1 + frac(0.6180339887498949 k) at the coarse node (X, Y),
// k = Y (ncx + 1) + X (b(u_i, W) = omega^T (M_H c_H + G_b d)). Writes c and c0 = 1 for virtual member
// b q + i, D[b][i][j] = d_j, lambda_{i,h_L}. One block per real problem, warp i per eigenvector.
__global__ void k_rr_multi_out(DevGeom G, int q, int s, int nb, int bw, int L, int lam_stride, const double* X,
                               const double* theta, const double* MH, long long mstride, const double* Gb, double* c,
                               double* c0, double* D, double* lam) {
  const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncx = G.ncx, ncy = G.ncy, N = nb + q, ncoef = (ncx + 1) * (ncy + 1);
  const double* M = MH + (long long)b * mstride;
  __shared__ double sgn[MLEV_MAX_EIGENPAIRS];
  if (warp < q) {
    const double* x = X + ((long long)b * s + warp) * N;
    double t = 0.0;
    for (int r = lane; r < nb; r += 32) {
      const int Xn = r % (ncx - 1) + 1, Yn = r / (ncx - 1) + 1;
      double bx = coarse_band_mv(M, bw, bw - 1, x, r, nb);
      for (int j = 0; j < q; ++j) bx += Gb[((long long)b * q + j) * nb + r] * x[nb + j];
      const double xk = (double)(Yn * (ncx + 1) + Xn) * 0.6180339887498949;
      if (is_free(G, 0, ncx, ncy, Xn, Yn)) t += (1.0 + (xk - floor(xk))) * bx;
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sgn[warp] = t >= 0.0 ? 1.0 : -1.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < q * ncoef; e += blockDim.x) {
    const int i = e / ncoef, k = e % ncoef, Xn = k % (ncx + 1), Yn = k / (ncx + 1);
    double v = 0.0;
    if (Xn >= 1 && Yn >= 1 && Xn < ncx && Yn < ncy && is_free(G, 0, ncx, ncy, Xn, Yn))
      v = sgn[i] * X[((long long)b * s + i) * N + (Yn - 1) * (ncx - 1) + (Xn - 1)];
    c[(long long)(b * q + i) * ncoef + k] = v;
  }
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int i = e / q, j = e % q;
    D[((long long)b * q + i) * q + j] = sgn[i] * X[((long long)b * s + i) * N + nb + j];
  }
  if (threadIdx.x < q) {
    c0[b * q + threadIdx.x] = 1.0;
    lam[(long long)(b * q + threadIdx.x) * lam_stride + L] = theta[(long long)b * s + threadIdx.x];
  }
}

// ------------------------------------------------------------------ launchers
#define MLEV_DISPATCH_KK3(kk, ...)                   \
  switch (kk) {                                      \
    case MLEV_KAPPA_ONE: {                           \
      constexpr int KK = MLEV_KAPPA_ONE;             \
      __VA_ARGS__;                                   \
    } break;                                         \
    case MLEV_KAPPA_PER_COARSE_CELL: {               \
      constexpr int KK = MLEV_KAPPA_PER_COARSE_CELL; \
      __VA_ARGS__;                                   \
    } break;                                         \
    default: {                                       \
      constexpr int KK = MLEV_KAPPA_PER_FINE_ELEM;   \
      __VA_ARGS__;                                   \
    } break;                                         \
  }

void launch_band_level(const DevGeom& G, int Breal, int q, int l, double* K, double* M, cudaStream_t s) {
  MLEV_DISPATCH_KK3(G.kap.kind, (k_band_level<KK><<<512, 256, 0, s>>>(G, Breal, q, l, K, M)));
}
void launch_cross_gram(const DevGeom& G, const GlobalLayout& gl, int L, int Breal, int q, const double* ut, double* out,
                       cudaStream_t s) {
  const long long nblk = (long long)Breal * G.ncx * G.ncy * (q * (q + 1) / 2);
  MLEV_DISPATCH_KK3(G.kap.kind, (k_cross_gram<KK><<<(unsigned)nblk, 256, 0, s>>>(G, gl, L, q, ut, out)));
}
void launch_border_prep(const DevGeom& G, int Breal, int q, const double* partials, const double* cross, double* Ga,
                        double* Gb, double* Aq, double* Bq, cudaStream_t s) {
  k_border_prep<<<Breal, 256, 0, s>>>(G, q, partials, cross, Ga, Gb, Aq, Bq);
}
size_t sub_eig_smem_bytes(int nb, int bwk, int s) {
  const size_t dbl = (size_t)(3 * kSMax * kSMax + 2 * kSMax + MLEV_MAX_EIGENPAIRS * MLEV_MAX_EIGENPAIRS +
                              32 * MLEV_MAX_EIGENPAIRS + 4 * kSMax * kSMax) * 8;
  const size_t nb32 = (size_t)sub_eig_nbk(nb) * kTB;
  const size_t flt = ((size_t)sub_eig_nbk(nb) * kTT + nb32 + (size_t)s * nb32) * 4;
  return dbl + flt + (size_t)bwk * (bwk + 1) / 2 * 4 + 64;
}
void launch_sub_eig(const DevGeom& G, const SubEigArgs& a, int Breal, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sub_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, kSubEigSmemMax);
    attr = true;
  }
  k_sub_eig<<<Breal, 1024, sub_eig_smem_bytes(a.nb, a.bwk, a.s), s>>>(G, a);
}
void launch_level1_multi_out(const DevGeom& G, const GlobalLayout& gl, int Breal, int q, int s_, const double* X,
                             const double* theta, double* ut1, double* lam, int lam_stride, double* c, double* c0,
                             cudaStream_t s) {
  k_level1_multi_out<<<Breal * q, 256, 0, s>>>(G, gl, q, s_, X, theta, ut1, lam, lam_stride, c, c0);
}
void launch_rr_multi_out(const DevGeom& G, int Breal, int q, int s_, int nb, int bw, int L, int lam_stride,
                         const double* X, const double* theta, const double* MH, long long mstride, const double* Gb,
                         double* c, double* c0, double* D, double* lam, cudaStream_t s) {
  k_rr_multi_out<<<Breal, 256, 0, s>>>(G, q, s_, nb, bw, L, lam_stride, X, theta, MH, mstride, Gb, c, c0, D, lam);
}
void launch_combine(const GlobalLayout& gl, int L, int Breal, int q, const double* D, const double* src, double* dst,
                    cudaStream_t s) {
  k_combine<<<1024, 256, 0, s>>>(gl, L, Breal, q, D, src, dst);
}

}  // namespace mlev
