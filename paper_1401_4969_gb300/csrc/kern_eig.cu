// The two small eigen solves of Algorithm 4.2:
//
// * k_level1: step 1, the smallest eigenpair of K_1 x = lambda M_1 x on V_{0h_1}
//   (Eq. Discrete_Weak_Eigen_Problem on T_{h_1}). One block per batch member runs a
//   block-size-1 LOBPCG (locally optimal preconditioned iteration) whose
//   preconditioner is one multigrid V-cycle on the level-1 hierarchy; Gram matrices
//   and Ritz values are FP64.
//
// * k_rr: step 3 of Algorithm 4.1 (Eq. Eigen_Augment_Problem), the smallest eigenpair
//   of the (N_H+1) pencil A c = mu B c with A = [[K_H, g_a], [g_a^T, alpha]],
//   B = [[M_H, g_b], [g_b^T, beta]] in the basis {coarse hats, u~}. For mu below the
//   smallest eigenvalue of (K_H, M_H), S(mu) = K_H - mu M_H is SPD and
//   det(A - mu B) = det S(mu) * f(mu) with the Schur complement
//   f(mu) = alpha - mu beta - w^T S(mu)^{-1} w,  w = g_a - mu g_b.
//   f is strictly decreasing and concave there, so the smallest eigenvalue is its
//   unique root; it is found by Newton's method safeguarded by bisection, with a
//   banded Cholesky factorisation of S(mu) per step. The eigenvector is
//   c = [-S(mu)^{-1} w ; 1], scaled to b(u,u) = 1 and int u > 0.
#include "kern_band.cuh"
#include "kern_blk.cuh"
#include "kern_tail.cuh"
#include "kern_launch.h"

namespace mlev {

// ---------------------------------------------------------------- small dense helpers
// Smallest eigenpair of the symmetric-definite pencil (A, B) of order n <= 3 with
// symmetric diagonal scaling, Cholesky of B and cyclic Jacobi rotations. Returns false
// if B is numerically singular.
__device__ bool small_geneig(int n, const double A[3][3], const double B[3][3], double& theta, double coef[3]) {
  double d[3], As[3][3], Bs[3][3], Lc[3][3] = {{0}}, C[3][3], V[3][3];
  for (int i = 0; i < n; ++i) d[i] = 1.0 / sqrt(B[i][i]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      As[i][j] = A[i][j] * d[i] * d[j];
      Bs[i][j] = B[i][j] * d[i] * d[j];
    }
  for (int j = 0; j < n; ++j) {
    double s = Bs[j][j];
    for (int k = 0; k < j; ++k) s -= Lc[j][k] * Lc[j][k];
    if (!(s > 1e-10)) return false;
    Lc[j][j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = Bs[i][j];
      for (int k = 0; k < j; ++k) t -= Lc[i][k] * Lc[j][k];
      Lc[i][j] = t / Lc[j][j];
    }
  }
  // C = L^{-1} As L^{-T}: Y = L^{-1} As, then C = (L^{-1} Y^T)^T
  double Y[3][3];
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double t = As[i][c];
      for (int k = 0; k < i; ++k) t -= Lc[i][k] * Y[k][c];
      Y[i][c] = t / Lc[i][i];
    }
  for (int r = 0; r < n; ++r)
    for (int i = 0; i < n; ++i) {
      double t = Y[r][i];
      for (int k = 0; k < i; ++k) t -= Lc[i][k] * C[r][k];
      C[r][i] = t / Lc[i][i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i][j] = (i == j);
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += C[p][q] * C[p][q];
    if (off < 1e-32 * (C[0][0] * C[0][0] + 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (C[p][q] == 0.0) continue;
        const double tau = (C[q][q] - C[p][p]) / (2.0 * C[p][q]);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          const double a = C[k][p], b = C[k][q];
          C[k][p] = cs * a - sn * b;
          C[k][q] = sn * a + cs * b;
        }
        for (int k = 0; k < n; ++k) {
          const double a = C[p][k], b = C[q][k];
          C[p][k] = cs * a - sn * b;
          C[q][k] = sn * a + cs * b;
        }
        for (int k = 0; k < n; ++k) {
          const double a = V[k][p], b = V[k][q];
          V[k][p] = cs * a - sn * b;
          V[k][q] = sn * a + cs * b;
        }
      }
  }
  int im = 0;
  for (int i = 1; i < n; ++i)
    if (C[i][i] < C[im][im]) im = i;
  theta = C[im][im];
  // coef = D L^{-T} v
  double y[3];
  for (int i = n - 1; i >= 0; --i) {
    double t = V[i][im];
    for (int k = i + 1; k < n; ++k) t -= Lc[k][i] * y[k];
    y[i] = t / Lc[i][i];
  }
  for (int i = 0; i < n; ++i) coef[i] = d[i] * y[i];
  for (int i = n; i < 3; ++i) coef[i] = 0.0;
  return true;
}

// Reciprocal and reciprocal square root: the fast rounded FP32 forms for float (these
// pencils only weight search directions), the plain operations for double.
__device__ __forceinline__ float sg_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double sg_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float sg_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sg_rsqrt(double x) { return 1.0 / sqrt(x); }

// Same computation in either precision (R = float or double) with the order N fixed at
// compile time, so the 3 x 3 arrays live in registers; off_tol is the relative size of the
// off-diagonal part at which the Jacobi sweeps stop.
// Smallest eigenpair of the symmetric-definite pencil (A, B) of order N <= 3 with
// symmetric diagonal scaling, Cholesky of B and cyclic Jacobi rotations. Returns false
// if B is numerically singular.
template <typename R, int N>
__device__ bool small_geneig_n(const R A[3][3], const R B[3][3], R& theta, R coef[3], R off_tol) {
  R d[3], As[3][3], Bs[3][3], Lc[3][3] = {{0}}, iL[3], C[3][3], V[3][3];
#pragma unroll
  for (int i = 0; i < N; ++i) d[i] = sg_rsqrt(B[i][i]);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      As[i][j] = A[i][j] * d[i] * d[j];
      Bs[i][j] = B[i][j] * d[i] * d[j];
    }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    R s = Bs[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= Lc[j][k] * Lc[j][k];
    if (!(s > (R)1e-10)) return false;
    Lc[j][j] = sqrt(s);
    iL[j] = sg_rcp(Lc[j][j]);
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      R t = Bs[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= Lc[i][k] * Lc[j][k];
      Lc[i][j] = t * iL[j];
    }
  }
  // C = L^{-1} As L^{-T}: Y = L^{-1} As, then C = (L^{-1} Y^T)^T
  R Y[3][3];
#pragma unroll
  for (int c = 0; c < N; ++c)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      R t = As[i][c];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= Lc[i][k] * Y[k][c];
      Y[i][c] = t * iL[i];
    }
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      R t = Y[r][i];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= Lc[i][k] * C[r][k];
      C[r][i] = t * iL[i];
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) V[i][j] = (R)(i == j);
  for (int sweep = 0; sweep < 30; ++sweep) {
    R off = 0.0;
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int q = p + 1; q < N; ++q) off += C[p][q] * C[p][q];
    R dg = (R)0;
#pragma unroll
    for (int p = 0; p < N; ++p) dg += C[p][p] * C[p][p];
    if (off <= off_tol * dg) break;
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
      for (int q = p + 1; q < N; ++q) {
        if (C[p][q] == (R)0) continue;
        const R tau = (C[q][q] - C[p][p]) * sg_rcp((R)2 * C[p][q]);
        const R t = (tau >= 0 ? (R)1 : (R)-1) * sg_rcp(fabs(tau) + sqrt((R)1 + tau * tau));
        const R cs = sg_rsqrt((R)1 + t * t), sn = t * cs;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const R a = C[k][p], b = C[k][q];
          C[k][p] = cs * a - sn * b;
          C[k][q] = sn * a + cs * b;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const R a = C[p][k], b = C[q][k];
          C[p][k] = cs * a - sn * b;
          C[q][k] = sn * a + cs * b;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const R a = V[k][p], b = V[k][q];
          V[k][p] = cs * a - sn * b;
          V[k][q] = sn * a + cs * b;
        }
      }
  }
  int im = 0;
  R cm = C[0][0];
#pragma unroll
  for (int i = 1; i < N; ++i)
    if (C[i][i] < cm) {
      cm = C[i][i];
      im = i;
    }
  theta = cm;
  // coef = D L^{-T} v (the column of V chosen by select, no dynamic register indexing)
  R vm[3];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    vm[i] = V[i][0];
#pragma unroll
    for (int c = 1; c < N; ++c)
      if (im == c) vm[i] = V[i][c];
  }
  R y[3];
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    R t = vm[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) t -= Lc[k][i] * y[k];
    y[i] = t * iL[i];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) coef[i] = d[i] * y[i];
#pragma unroll
  for (int i = N; i < 3; ++i) coef[i] = (R)0;
  return true;
}

// ---------------------------------------------------------------- level-1 LOBPCG
template <typename T, int KK>
__global__ void __launch_bounds__(1024) k_level1(DevGeom G, GlobalLayout gl, Level1Args a) {
  __shared__ double scratch[32 * 12];
  __shared__ double red[12];
  __shared__ double sh_coef[4];
  __shared__ int sh_flag[2];
  const int p = blockIdx.x;
  const int g0 = a.grid_begin + p * a.nlev;
  const GridDesc& g = G.grids[g0];
  const long long vs = a.vstride;
  double* X = a.vec + (long long)p * 10 * vs;
  double *W = X + vs, *P = W + vs, *KX = P + vs, *MX = KX + vs, *KW = MX + vs, *MW = KW + vs, *KP = MW + vs,
         *MP = KP + vs, *R = MP + vs;
  T* xp = (T*)a.xpool;
  T* fp = (T*)a.fpool;
  const int nx = g.nx, ny = g.ny, pitch = g.pitch, nn = (nx + 1) * (ny + 1);
  const double h = level_h(G.H, 1), m12 = h * h / 12.0;

  auto apply_km = [&](const double* v, double* kv, double* mv) {
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const int i = q % (nx + 1), j = q / (nx + 1);
      const long long c = (long long)j * pitch + i;
      if (!is_unknown(G, g, i, j)) {
        kv[c] = 0.0;
        mv[c] = 0.0;
        continue;
      }
      const W4 w = edge_weights<KK>(G.kap, p, 1, i, j);
      kv[c] = apply_k<double, double>(v, c, pitch, w);
      mv[c] = m12 * apply_m12<double, double>(v, c, pitch);
    }
    __syncthreads();
  };

  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int i = q % (nx + 1), j = q / (nx + 1);
    const long long c = (long long)j * pitch + i;
    X[c] = is_unknown(G, g, i, j) ? 1.0 : 0.0;
    W[c] = P[c] = KP[c] = MP[c] = R[c] = 0.0;
  }
  __syncthreads();
  apply_km(X, KX, MX);
  double rho;
  {
    double v[2] = {0.0, 0.0};
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
      v[0] += X[c] * KX[c];
      v[1] += X[c] * MX[c];
    }
    block_sum<2>(v, scratch, red);
    rho = red[0] / red[1];
  }
  bool have_p = false;
  int it = 0;
  double res = 1.0;
  for (; it < a.max_iter; ++it) {
    {
      double v[2] = {0.0, 0.0};
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
        const double r = KX[c] - rho * MX[c];
        R[c] = r;
        v[0] += r * r;
        v[1] += MX[c] * MX[c];
      }
      block_sum<2>(v, scratch, red);
      res = sqrt(red[0]) / (rho * sqrt(red[1]));
    }
    if (res < a.tol) break;
    // preconditioner: one V-cycle for K w = r from w = 0
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
      fp[g.off + c] = (T)R[c];
      xp[g.off + c] = (T)0;
    }
    __syncthreads();
    blk_vcycle<T, KK>(G, G.grids + g0, a.nlev, xp, fp, a.pre, a.post, a.coarse_sweeps, (T)a.omega, nullptr);
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
      W[c] = (double)xp[g.off + c];
    }
    __syncthreads();
    apply_km(W, KW, MW);
    {
      double v[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = 0.0;
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
        const double x = X[c], w = W[c], pp = P[c];
        v[0] += x * KX[c]; v[1] += x * KW[c]; v[2] += x * KP[c];
        v[3] += w * KW[c]; v[4] += w * KP[c]; v[5] += pp * KP[c];
        v[6] += x * MX[c]; v[7] += x * MW[c]; v[8] += x * MP[c];
        v[9] += w * MW[c]; v[10] += w * MP[c]; v[11] += pp * MP[c];
      }
      block_sum<12>(v, scratch, red);
    }
    if (threadIdx.x == 0) {
      double A[3][3] = {{red[0], red[1], red[2]}, {red[1], red[3], red[4]}, {red[2], red[4], red[5]}};
      double Bm[3][3] = {{red[6], red[7], red[8]}, {red[7], red[9], red[10]}, {red[8], red[10], red[11]}};
      double th, cf[3];
      bool ok = have_p && small_geneig(3, A, Bm, th, cf);
      if (!ok) ok = small_geneig(2, A, Bm, th, cf);
      if (!ok) {
        th = rho;
        cf[0] = 1.0;
        cf[1] = cf[2] = 0.0;
      }
      // normalise x_new in the M-norm and keep p_new = cf1 w + cf2 p with unit M-norm
      const double bx = cf[0] * cf[0] * Bm[0][0] + cf[1] * cf[1] * Bm[1][1] + cf[2] * cf[2] * Bm[2][2] +
                        2.0 * (cf[0] * cf[1] * Bm[0][1] + cf[0] * cf[2] * Bm[0][2] + cf[1] * cf[2] * Bm[1][2]);
      const double bp = cf[1] * cf[1] * Bm[1][1] + cf[2] * cf[2] * Bm[2][2] + 2.0 * cf[1] * cf[2] * Bm[1][2];
      const double sx = 1.0 / sqrt(bx), sp = bp > 0 ? 1.0 / sqrt(bp) : 0.0;
      sh_coef[0] = cf[0] * sx;
      sh_coef[1] = cf[1];
      sh_coef[2] = cf[2];
      sh_coef[3] = th;
      red[0] = sx;
      red[1] = sp;
      sh_flag[0] = ok && bp > 0;
    }
    __syncthreads();
    const double ca = sh_coef[0], cb = sh_coef[1], cp = sh_coef[2], sx = red[0], sp = red[1];
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
      const double pn = cb * W[c] + cp * P[c], kpn = cb * KW[c] + cp * KP[c], mpn = cb * MW[c] + cp * MP[c];
      X[c] = ca * X[c] + sx * pn;
      KX[c] = ca * KX[c] + sx * kpn;
      MX[c] = ca * MX[c] + sx * mpn;
      P[c] = sp * pn;
      KP[c] = sp * kpn;
      MP[c] = sp * mpn;
    }
    rho = sh_coef[3];
    have_p = sh_flag[0] != 0;
    __syncthreads();
  }
  // recompute K x, M x exactly, the Rayleigh quotient, b(x,x) and the sign
  apply_km(X, KX, MX);
  double v[3] = {0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
    v[0] += X[c] * KX[c];
    v[1] += X[c] * MX[c];
    v[2] += X[c];
  }
  block_sum<3>(v, scratch, red);
  const double lam = red[0] / red[1];
  const double sc = (red[2] >= 0 ? 1.0 : -1.0) / sqrt(red[1]);
  double* out = a.ut1 + (long long)p * gl.bstride;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const long long c = (long long)(q / (nx + 1)) * pitch + q % (nx + 1);
    out[c] = sc * X[c];
  }
  const int ncoef = (G.ncx + 1) * (G.ncy + 1);
  for (int q = threadIdx.x; q < ncoef; q += blockDim.x) a.c[(long long)p * ncoef + q] = 0.0;
  if (threadIdx.x == 0) {
    a.c0[p] = 1.0;
    a.lam[p * a.lam_stride + 1] = lam;
    a.stat[p * a.stat_stride + MLEV_STAT_L1_IT] = it;
    a.stat[p * a.stat_stride + MLEV_STAT_L1_RES] = (long long)__double_as_longlong(res);
    if (it >= a.max_iter)
      atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_LEVEL1_NOCONV);
    if (!isfinite(lam))
      atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_NONFINITE);
  }
}

template <typename T>
void launch_level1(const DevGeom& G, const GlobalLayout& gl, const Level1Args& a, cudaStream_t s) {
  switch (G.kap.kind) {
    case MLEV_KAPPA_ONE: k_level1<T, MLEV_KAPPA_ONE><<<a.B, 1024, 0, s>>>(G, gl, a); break;
    case MLEV_KAPPA_PER_COARSE_CELL: k_level1<T, MLEV_KAPPA_PER_COARSE_CELL><<<a.B, 1024, 0, s>>>(G, gl, a); break;
    default: k_level1<T, MLEV_KAPPA_PER_FINE_ELEM><<<a.B, 1024, 0, s>>>(G, gl, a); break;
  }
}
template void launch_level1<float>(const DevGeom&, const GlobalLayout&, const Level1Args&, cudaStream_t);
template void launch_level1<double>(const DevGeom&, const GlobalLayout&, const Level1Args&, cudaStream_t);

// ---------------------------------------------------------------- level-1 LOBPCG on chip
// The iteration of k_level1 with every vector and the whole level-1 multigrid hierarchy in
// shared memory (compact row pitch nx + 1), used when they fit, and with the small Ritz
// step kept off the FP64 pipe: x, K x, M x and the residual r are FP64 (K x and M x are
// recomputed from x every iteration, so the residual test is exact), while the search
// directions w (one V-cycle on r) and p, their images and the 3 x 3 Rayleigh-Ritz pencil
// are FP32. The pencil is formed shifted by the FP64 Rayleigh quotient rho of x:
// (A - rho B)_{xw} = r^T w and (A - rho B)_{xx} = 0, so FP32 resolves the small
// coefficients of w and p; an FP32 coefficient error only makes a step slightly
// suboptimal. Layout: FP32 Gram partials [11][threads], 4 FP64 vectors, 6 FP32 vectors,
// then x (T) and f (T) of every level and the unknown masks. MINB is the register bound's
// blocks per SM: 1 (126 registers, no spills) for one or few problems, 2 (64 registers)
// when a batch has more problems than SMs and two blocks' shared memory fit one SM.
template <typename T, int KK, int MINB>
__global__ void __launch_bounds__(512, MINB) k_level1_sm(DevGeom G, GlobalLayout gl, Level1Args a) {
  extern __shared__ __align__(16) unsigned char l1_raw[];
  __shared__ SmGrid<T> lv[kTailMaxLev];
  __shared__ double red[4];
  __shared__ float gram[12];
  __shared__ float sh_coef[4];
  __shared__ double sh_rho[2];  // FP64 scalars formed by thread 0, read after the next barrier
  __shared__ int sh_flag, sh_stop;
  const int p = blockIdx.x, g0 = a.grid_begin + p * a.nlev, nlev = a.nlev;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const GridDesc& g = G.grids[g0];
  const int nx = g.nx, ny = g.ny, W = nx + 1, nn = W * (ny + 1);
  float* G11 = reinterpret_cast<float*>(l1_raw);   // [11][nt]
  double* X = reinterpret_cast<double*>(G11 + 12 * nt);
  double *KX = X + nn, *MX = KX + nn, *R = MX + nn;
  float* Wv = reinterpret_cast<float*>(R + nn);
  float *KW = Wv + nn, *MW = KW + nn, *P = MW + nn, *KP = P + nn, *MP = KP + nn;
  if (tid == 0) {
    long long tot = 0;
    for (int k = 0; k < nlev; ++k) {
      const GridDesc& gk = G.grids[g0 + k];
      tot += ((long long)(gk.nx + 1) * (gk.ny + 1) + 1) & ~1LL;
    }
    T* xb = reinterpret_cast<T*>(MP + nn);  // 6 nn floats after an 8-byte aligned start: aligned for T
    T* fb = xb + tot;
    uint8_t* mb = reinterpret_cast<uint8_t*>(fb + tot);
    long long off = 0;
    for (int k = 0; k < nlev; ++k) {
      const GridDesc& gk = G.grids[g0 + k];
      lv[k].x = xb + off;
      lv[k].f = fb + off;
      lv[k].m = mb + off;
      lv[k].nx = gk.nx;
      lv[k].ny = gk.ny;
      lv[k].W = gk.nx + 1;
      lv[k].g = &G.grids[g0 + k];
      off += ((long long)(gk.nx + 1) * (gk.ny + 1) + 1) & ~1LL;
    }
  }
  __syncthreads();
  for (int k = 0; k < nlev; ++k) {
    const GridDesc& gk = *lv[k].g;
    const int nk = lv[k].W * (lv[k].ny + 1);
    for (int q = tid; q < nk; q += nt) {
      const int j = q / lv[k].W, i = q - j * lv[k].W;
      lv[k].m[q] = is_unknown(G, gk, i, j);
    }
  }
  __syncthreads();
  const uint8_t* m0 = lv[0].m;
  const double h = level_h(G.H, 1), m12 = h * h / 12.0;
  const float m12f = (float)m12;
// every node (i, j) of level 1 once, flat over the block (no half-empty warp passes)
#define L1_FOR_NODES                                             \
  for (int n_ = tid, j = n_ / W, i = n_ - j * W; n_ < nn;        \
       n_ += nt, j = n_ / W, i = n_ - j * W)
  auto apply_km64 = [&]() {  // K x, M x in FP64
    L1_FOR_NODES {
      const int q = j * W + i;
      if (!m0[q]) {
        KX[q] = 0.0;
        MX[q] = 0.0;
        continue;
      }
      const W4 w = edge_weights<KK>(G.kap, p, 1, g.ox + i, g.oy + j);
      KX[q] = (w.e + w.w + w.n + w.s) * X[q] - w.e * X[q + 1] - w.w * X[q - 1] - w.n * X[q + W] - w.s * X[q - W];
      MX[q] = m12 * (6.0 * X[q] + X[q + 1] + X[q - 1] + X[q + W] + X[q - W] + X[q + W + 1] + X[q - W - 1]);
    }
    __syncthreads();
  };
  L1_FOR_NODES {
    const int q = j * W + i;
    X[q] = m0[q] ? 1.0 : 0.0;
    Wv[q] = P[q] = KP[q] = MP[q] = 0.f;
  }
  __syncthreads();
  apply_km64();
  bool have_p = false;
  int it = 0;
  double res = 1.0, rho = 0.0;
  // FP64 sums staged in the Gram buffer (free outside the Gram step), flat node loops (the
  // sums and the residual need no (i, j)); the stopping test compares squares
  double* stage = reinterpret_cast<double*>(G11);
  double r2 = 0.0, m2 = 1.0;
  for (; it < a.max_iter; ++it) {
    {  // FP64 Rayleigh quotient of x
      double v[2] = {0.0, 0.0};
      for (int q = tid; q < nn; q += nt) {
        v[0] += X[q] * KX[q];
        v[1] += X[q] * MX[q];
      }
      block_sum_t<2>(v, stage, red);
      // one thread divides: a warp's FP64 instruction holds its sub-partition's FP64 pipe
      // for 64 cycles whether one lane or 32 are active, so 16 warps each dividing would
      // cost as much as a pass over the grid
      if (tid == 0) sh_rho[0] = red[0] / red[1];
      __syncthreads();
      rho = sh_rho[0];
    }
    {
      double v[2] = {0.0, 0.0};
      for (int q = tid; q < nn; q += nt) {
        const double r = KX[q] - rho * MX[q];
        R[q] = r;
        v[0] += r * r;
        v[1] += MX[q] * MX[q];
      }
      block_sum_t<2>(v, stage, red);
      r2 = red[0];
      m2 = red[1];
    }
    // relative eigen-residual |r| / (rho |M x|) < tol, decided by thread 0 and read after
    // the barrier that follows the V-cycle's first loads
    if (tid == 0) sh_stop = r2 < a.tol * a.tol * rho * rho * m2;
    // preconditioner: one V-cycle for K w = r from w = 0, all grids on chip
    for (int q = tid; q < nn; q += nt) {
      lv[0].f[q] = m0[q] ? (T)R[q] : (T)0;
      lv[0].x[q] = (T)0;
    }
    __syncthreads();
    if (sh_stop) break;
    for (int d = 0; d + 1 < nlev; ++d) {
      tail_smooth<T, KK>(G, lv[d], a.pre, false, (T)a.omega);
      tail_restrict<T, KK>(G, lv[d], lv[d + 1], a.pre >= 1 && a.omega == 1.0);
    }
    tail_smooth<T, KK>(G, lv[nlev - 1], a.coarse_sweeps, false, (T)a.omega);
    for (int d = nlev - 2; d >= 0; --d) {
      tail_prolong<T>(lv[d], lv[d + 1], a.post >= 1 && a.omega == 1.0);
      tail_smooth<T, KK>(G, lv[d], a.post, true, (T)a.omega);
    }
    for (int q = tid; q < nn; q += nt) Wv[q] = (float)lv[0].x[q];
    __syncthreads();
    // K w, M w in FP32 and the FP32 Gram sums
    {
      float v[11];
#pragma unroll
      for (int k = 0; k < 11; ++k) v[k] = 0.f;
      L1_FOR_NODES {
        const int q = j * W + i;
        float kw = 0.f, mw = 0.f;
        if (m0[q]) {
          const EW<float> w = edge_weights_t<float, KK>(G.kap, p, 1, g.ox + i, g.oy + j);
          kw = (w.e + w.w + w.n + w.s) * Wv[q] - w.e * Wv[q + 1] - w.w * Wv[q - 1] - w.n * Wv[q + W] - w.s * Wv[q - W];
          mw = m12f * (6.f * Wv[q] + Wv[q + 1] + Wv[q - 1] + Wv[q + W] + Wv[q - W] + Wv[q + W + 1] + Wv[q - W - 1]);
        }
        KW[q] = kw;
        MW[q] = mw;
        const float w = Wv[q], pp = P[q], r = (float)R[q], x = (float)X[q], mx = (float)MX[q];
        v[0] += r * w;   v[1] += r * pp;   v[2] += w * kw;   v[3] += w * mw;
        v[4] += w * KP[q]; v[5] += w * MP[q]; v[6] += pp * KP[q]; v[7] += pp * MP[q];
        v[8] += x * mx;  v[9] += x * mw;   v[10] += x * MP[q];
      }
#pragma unroll
      for (int k = 0; k < 11; ++k) G11[k * nt + tid] = v[k];
      __syncthreads();
      const int lane = tid & 31, warp = tid >> 5;
      if (warp < 11) {
        float s = 0.f;
        for (int q = lane; q < nt; q += 32) s += G11[warp * nt + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) gram[warp] = s;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const float rf = (float)rho;
      const float As[3][3] = {{0.f, gram[0], gram[1]},
                              {gram[0], gram[2] - rf * gram[3], gram[4] - rf * gram[5]},
                              {gram[1], gram[4] - rf * gram[5], gram[6] - rf * gram[7]}};
      const float Bs[3][3] = {{gram[8], gram[9], gram[10]}, {gram[9], gram[3], gram[5]}, {gram[10], gram[5], gram[7]}};
      float th, cf[3];
      bool ok = have_p && small_geneig_n<float, 3>(As, Bs, th, cf, 1e-12f);
      if (!ok) ok = small_geneig_n<float, 2>(As, Bs, th, cf, 1e-12f);
      if (!ok) {
        cf[0] = 1.f;
        cf[1] = cf[2] = 0.f;
      }
      const float bx = cf[0] * cf[0] * Bs[0][0] + cf[1] * cf[1] * Bs[1][1] + cf[2] * cf[2] * Bs[2][2] +
                       2.f * (cf[0] * cf[1] * Bs[0][1] + cf[0] * cf[2] * Bs[0][2] + cf[1] * cf[2] * Bs[1][2]);
      const float bp = cf[1] * cf[1] * Bs[1][1] + cf[2] * cf[2] * Bs[2][2] + 2.f * cf[1] * cf[2] * Bs[1][2];
      const float sx = rsqrtf(bx), sp = bp > 0.f ? rsqrtf(bp) : 0.f;
      sh_coef[0] = cf[0] * sx;
      sh_coef[1] = cf[1] * sx;
      sh_coef[2] = cf[2] * sx;
      sh_coef[3] = sp / sx;  // p_new = sp (cf1 w + cf2 p)
      sh_flag = ok && bp > 0.f;
    }
    __syncthreads();
    // x <- ca x + cb w + cp p (FP64 accumulation); p <- s (cb w + cp p) with its images
    const double ca = sh_coef[0];
    const float cb = sh_coef[1], cp = sh_coef[2], sp = sh_coef[3];
    for (int q = tid; q < nn; q += nt) {
      const float pn = cb * Wv[q] + cp * P[q];
      X[q] = ca * X[q] + (double)pn;
      P[q] = sp * pn;
      KP[q] = sp * (cb * KW[q] + cp * KP[q]);
      MP[q] = sp * (cb * MW[q] + cp * MP[q]);
    }
    have_p = sh_flag != 0;
    __syncthreads();
    apply_km64();
  }
  double v[3] = {0.0, 0.0, 0.0};
  for (int q = tid; q < nn; q += nt) {
    v[0] += X[q] * KX[q];
    v[1] += X[q] * MX[q];
    v[2] += X[q];
  }
  block_sum_t<3>(v, stage, red);
  if (tid == 0) {
    sh_rho[0] = red[0] / red[1];
    sh_rho[1] = (red[2] >= 0 ? 1.0 : -1.0) / sqrt(red[1]);
  }
  __syncthreads();
  const double lam = sh_rho[0], sc = sh_rho[1];
  double* out = a.ut1 + (long long)p * gl.bstride;
  const int gp = gl.pitch[1 - MLEV_LMIN];
  L1_FOR_NODES { out[(long long)j * gp + i] = sc * X[j * W + i]; }
#undef L1_FOR_NODES
  const int ncoef = (G.ncx + 1) * (G.ncy + 1);
  for (int q = tid; q < ncoef; q += nt) a.c[(long long)p * ncoef + q] = 0.0;
  if (tid == 0) {
    res = sqrt(r2) / (rho * sqrt(m2));
    a.c0[p] = 1.0;
    a.lam[p * a.lam_stride + 1] = lam;
    a.stat[p * a.stat_stride + MLEV_STAT_L1_IT] = it;
    a.stat[p * a.stat_stride + MLEV_STAT_L1_RES] = (long long)__double_as_longlong(res);
    if (it >= a.max_iter)
      atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_LEVEL1_NOCONV);
    if (!isfinite(lam))
      atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_NONFINITE);
  }
}

size_t level1_smem_bytes(long long nn0, long long tot, int tsize) {
  return (size_t)(12 * 512 * 4 + 4 * nn0 * 8 + 6 * nn0 * 4 + 8 + 2 * tot * tsize + tot + 16);
}

template <typename T>
void launch_level1_sm(const DevGeom& G, const GlobalLayout& gl, const Level1Args& a, size_t smem, cudaStream_t s) {
  // two blocks per SM pay only when the batch fills every SM once and still has problems left
  int dev = 0, nsm = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const bool two = a.B > nsm && 2 * (smem + 4096) <= (size_t)smem_sm;
  switch (G.kap.kind) {
#define L1_LAUNCH(KKV, MB)                                                                                   \
  {                                                                                                          \
    static bool attr = false;                                                                                \
    if (!attr) {                                                                                             \
      cudaFuncSetAttribute(k_level1_sm<T, KKV, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kL1SmemMax); \
      attr = true;                                                                                           \
    }                                                                                                        \
    k_level1_sm<T, KKV, MB><<<a.B, dim3(32, 16), smem, s>>>(G, gl, a);                                       \
  }
#define L1_CASE(KKV)        \
  if (two)                  \
    L1_LAUNCH(KKV, 2)       \
  else                      \
    L1_LAUNCH(KKV, 1)
    case MLEV_KAPPA_ONE: L1_CASE(MLEV_KAPPA_ONE) break;
    case MLEV_KAPPA_PER_COARSE_CELL: L1_CASE(MLEV_KAPPA_PER_COARSE_CELL) break;
    default: L1_CASE(MLEV_KAPPA_PER_FINE_ELEM) break;
#undef L1_CASE
#undef L1_LAUNCH
  }
}
template void launch_level1_sm<float>(const DevGeom&, const GlobalLayout&, const Level1Args&, size_t, cudaStream_t);
template void launch_level1_sm<double>(const DevGeom&, const GlobalLayout&, const Level1Args&, size_t, cudaStream_t);

// ---------------------------------------------------------------- Rayleigh-Ritz
__global__ void __launch_bounds__(256) k_rr(DevGeom G, RRArgs a) {
  extern __shared__ double rr_sm[];
  __shared__ double scratch[8 * 4];
  __shared__ double red[4];
  __shared__ int flag;
  const int p = blockIdx.x, N = a.nhb, bw = a.bw, bw1 = bw + 1;
  const int ncx = G.ncx, ncy = G.ncy;
  const int npair = bw * (bw + 1) / 2;
  // band + vectors in shared memory when they fit (a.smem), else in the global scratch
  double* base = a.smem ? rr_sm : a.chol + (long long)p * ((long long)N * bw1 + 5LL * N);
  double* Lb = base;
  double* ga = Lb + (long long)N * bw1;
  double* gb = ga + N;
  double* wv = gb + N;
  double* y = wv + N;
  double* invD = y + N;
  int* pairs = reinterpret_cast<int*>(a.smem ? invD + N : rr_sm);
  const double* KH = a.KH + (long long)p * N * bw1;
  const double* MH = a.MH + (long long)p * N * bw1;
  const double* part = a.partials + (long long)p * ncx * ncy * 12;
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    int aa = 0;
    while ((aa + 1) * (aa + 2) / 2 <= q) ++aa;
    pairs[q] = (aa << 16) | (q - aa * (aa + 1) / 2);
  }
  // ---- reduce the per-cell partials: alpha, beta, sigma, g_a, g_b
  {
    double v[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < ncx * ncy; q += blockDim.x) {
      v[0] += part[q * 12 + 0];
      v[1] += part[q * 12 + 1];
      v[2] += part[q * 12 + 2];
    }
    block_sum<3>(v, scratch, red);
  }
  const double alpha = red[0], beta = red[1], sigma = red[2];
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int X = r % (ncx - 1) + 1, Y = r / (ncx - 1) + 1;
    double sa = 0.0, sb = 0.0;
    if (is_free(G, 0, ncx, ncy, X, Y)) {
      // node (X, Y) is corner 11 of cell (X-1, Y-1), 01 of (X, Y-1), 10 of (X-1, Y), 00 of (X, Y)
      const double* c11 = part + ((Y - 1) * ncx + (X - 1)) * 12;
      const double* c01 = part + ((Y - 1) * ncx + X) * 12;
      const double* c10 = part + (Y * ncx + (X - 1)) * 12;
      const double* c00 = part + (Y * ncx + X) * 12;
      sa = c00[3] + c10[4] + c01[5] + c11[6];
      sb = c00[7] + c10[8] + c01[9] + c11[10];
    }
    ga[r] = sa;
    gb[r] = sb;
  }
  __syncthreads();

  auto band_mv_m = [&](const double* v, int r) { return coarse_band_mv(MH, bw, bw - 1, v, r, N); };
  // factor S(mu) and solve S y = w(mu); false if S(mu) is not positive definite
  auto factor_solve = [&](double mu) {
    for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) Lb[q] = KH[q] - mu * MH[q];
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      wv[r] = ga[r] - mu * gb[r];
      y[r] = wv[r];
    }
    __syncthreads();
    if (!band_ldlt(Lb, invD, y, pairs, npair, N, bw, &flag)) return false;
    band_back(Lb, invD, y, N, bw);
    return true;
  };
  // f(mu) = alpha - mu beta - w^T y, f'(mu) = -beta + 2 g_b^T y - y^T M y
  auto eval = [&](double mu, double& f, double& fp) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      v[0] += wv[r] * y[r];
      v[1] += gb[r] * y[r];
      v[2] += y[r] * band_mv_m(y, r);
    }
    block_sum<3>(v, scratch, red);
    f = alpha - mu * beta - red[0];
    fp = -beta + 2.0 * red[1] - red[2];
  };

  // Newton from mu0 = alpha / beta (right of the root: f(mu0) = -w^T S^{-1} w <= 0),
  // safeguarded by the bracket [lo, hi]; accepted once the step is below 1e-9 relative
  // (the quadratic error is then at rounding level; y stays the solution at mu).
  double mu = alpha / beta, lo = 0.0, hi = INFINITY, lam = NAN;
  int it = 0, status = 0;
  bool have = false;
  for (; it < a.max_iter; ++it) {
    if (!factor_solve(mu)) {
      hi = mu;
      mu = 0.5 * (lo + hi);
      have = false;
      continue;
    }
    have = true;
    double f, fp;
    eval(mu, f, fp);
    if (f > 0.0) lo = mu;
    else hi = mu;
    const double step = (fp < 0.0) ? -f / fp : 0.0;
    if (fp < 0.0 && fabs(step) <= 1e-9 * fabs(mu)) {
      lam = mu + step;
      break;
    }
    double nmu = (fp < 0.0) ? mu + step : 0.5 * (lo + hi);
    if (!(nmu > lo && nmu < hi)) nmu = isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * mu;
    if (isfinite(hi) && hi - lo <= 1e-15 * hi) {
      lam = mu;
      break;
    }
    mu = nmu;
  }
  if (it >= a.max_iter) status |= MLEV_ST_RR_NOCONV;
  if (!(lam == lam)) lam = mu;
  if (!have && !factor_solve(mu)) status |= MLEV_ST_RR_BREAKDOWN;
  // y at lambda rather than at the last iterate mu (where Newton stops varies with the
  // input, and y(mu) differs from y(lambda) by O(lambda - mu) <= 1e-9): one correction step
  // y <- S(mu)^{-1} [w(lambda) + (lambda - mu) M y(mu)] with the factors of S(mu), error
  // O((lambda - mu)^2)
  if (have && lam != mu && isfinite(lam)) {
    const double dl = lam - mu;
    for (int r = threadIdx.x; r < N; r += blockDim.x) wv[r] = ga[r] - lam * gb[r] + dl * band_mv_m(y, r);
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) y[r] = wv[r];
    __syncthreads();
    band_fwd(Lb, invD, y, N, bw);
    band_back(Lb, invD, y, N, bw);
  }
  // eigenvector c = [-y ; 1], scaled to b(u,u) = 1 and int u > 0
  double v[3] = {0.0, 0.0, 0.0};
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    v[0] += y[r] * band_mv_m(y, r);
    v[1] += gb[r] * y[r];
    v[2] += y[r];
  }
  block_sum<3>(v, scratch, red);
  const double bn = red[0] - 2.0 * red[1] + beta;       // b(u,u) with c_H = -y, c_0 = 1
  const double S = (double)(1LL << (2 * a.L));          // sum over fine nodes of a coarse hat = H^2 / h^2
  const double integral = sigma - S * red[2];
  const double sc = (integral >= 0 ? 1.0 : -1.0) / sqrt(bn);
  const int ncoef = (ncx + 1) * (ncy + 1);
  double* cp = a.c + (long long)p * ncoef;
  for (int q = threadIdx.x; q < ncoef; q += blockDim.x) cp[q] = 0.0;
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int X = r % (ncx - 1) + 1, Y = r / (ncx - 1) + 1;
    cp[Y * (ncx + 1) + X] = is_free(G, 0, ncx, ncy, X, Y) ? -sc * y[r] : 0.0;
  }
  if (threadIdx.x == 0) {
    a.c0[p] = sc;
    a.lam[p * (a.n + 1) + a.L] = lam;
    a.stat[p * a.stat_stride + MLEV_STAT_RR_IT + a.L] = it + 1;
    if (!isfinite(lam) || !isfinite(sc)) status |= MLEV_ST_NONFINITE;
    if (status) atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)status);
  }
}

// Mixed-precision Rayleigh-Ritz (MLEV_PREC_MIXED): the Newton iteration of k_rr with the
// serial linear algebra moved off the FP64 pipe. S(sigma) is factored in FP32 (band
// LDL^T); every solve S(mu) y = w(mu) is FP64 iterative refinement y += S(sigma)^{-1} r
// (FP32 register-window solves by one warp), r = w - S(mu) y (FP64 band products from
// K_H and M_H staged in shared memory). It converges while |mu - sigma| is small against
// the distance of mu to the spectrum of (K_H, M_H); the factors are rebuilt at the current
// mu when it stalls.
// f(mu) is evaluated as alpha - mu beta - (w^T y + y^T r), the variational form of
// w^T S^{-1} w, whose error is quadratic in the error of y.
__global__ void __launch_bounds__(256) k_rr_mixed(DevGeom G, RRArgs a) {
  extern __shared__ double rr_sm[];
  __shared__ double stage[4 * 256];  // FP64 block sums, one warp per quantity (block_sum_t)
  __shared__ double red[4];
  __shared__ double sh_bc[2];  // scalars formed by thread 0 and broadcast at the next barrier
  __shared__ int bflag;
  const int p = blockIdx.x, N = a.nhb, bw = a.bw, bw1 = bw + 1;
  const int ncx = G.ncx, ncy = G.ncy;
  const int npair = bw * (bw + 1) / 2;
  double* base = a.smem ? rr_sm : a.chol + (long long)p * ((long long)N * bw1 + 5LL * N);
  double* ga = base;
  double* gb = ga + N;
  double* wv = gb + N;
  double* y = wv + N;
  double* r = y + N;
  double* kh_s = r + N;                                   // staged K_H, M_H (shared-memory mode)
  double* mh_s = kh_s + (long long)N * bw1;
  double* sm_s = mh_s + (long long)N * bw1;               // S(mu) of the current mu (FP64)
  float* Lb = reinterpret_cast<float*>(a.smem ? sm_s + (long long)N * bw1 : r + N);
  float* invD = Lb + (long long)N * bw1;
  float* r32 = invD + N;                                    // N + 32 entries, the tail kept at 0
  const int bsz = bw - 1, nbk = bsz > 0 ? N / bsz : 0;     // row blocks (blocked solves)
  const int BS = bsz <= 16 ? 16 : 32;                      // padded tile edge
  const int TS = BS * (BS + 4);                            // tile with row stride BS + 4
  // blocked mode (16-byte aligned): P_I^{-1}, W_I, W_I^T tiles, the padded right-hand side
  // yp and solution xp (block I at I * BS), 2 work tiles
  float* Dinv = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(r32 + N + 32) + 15) & ~uintptr_t(15));
  const long long tiles = a.blocked ? (long long)nbk * TS : 0, vecs = a.blocked ? (long long)nbk * BS : 0;
  float* Loff = Dinv + tiles;
  float* LT = Loff + tiles;
  float* yp = LT + tiles;
  float* xp = yp + vecs;
  float* bwork = xp + vecs;
  int* pairs = reinterpret_cast<int*>(a.smem ? bwork + (a.blocked ? 2 * TS : 0) : reinterpret_cast<float*>(rr_sm));
  // Set-up is a few rounds of L2 latency: the copies into shared memory (the factors of
  // S(sigma) prepared ahead, K_H and M_H) are issued first as asynchronous copies, then the
  // independent loads of the partials and the previous eigenvector, and one wait at the end.
  const bool pre_in = a.use_pre && a.blocked && a.smem;
  int pre_ok = 0;
  double pre_sig = NAN;
  if (pre_in) {
    // factors of S(sigma) from the inner-product kernel (rr_prefactor_block), copied whether
    // or not they are valid (invalid ones are rebuilt by factor() before any use)
    const unsigned char* pp = a.pre + (long long)p * a.pre_stride;
    const float* src = reinterpret_cast<const float*>(pp + 16);
    for (long long q = threadIdx.x; q < 3 * tiles / 4; q += blockDim.x) cp_async16(Dinv + 4 * q, src + 4 * q);
    pre_ok = *reinterpret_cast<const int*>(pp + 8);
    pre_sig = *reinterpret_cast<const double*>(pp);
  }
  const double* KH = a.KH + (long long)p * N * bw1;
  const double* MH = a.MH + (long long)p * N * bw1;
  if (a.smem) {
    if (a.blocked && bw >= 3) {
      // only the nonzero diagonals d = 0, 1, b, b + 1 are read in blocked mode (products,
      // S(mu), the block factor): stage those
      for (int q = threadIdx.x; q < 4 * N; q += blockDim.x) {
        const long long e = (long long)(q >> 2) * bw1 + coarse_band_diag(q & 3, bw - 1);
        cp_async8(kh_s + e, KH + e);
        cp_async8(mh_s + e, MH + e);
      }
    } else {
      for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) {
        cp_async8(kh_s + q, KH + q);
        cp_async8(mh_s + q, MH + q);
      }
    }
    for (int q = threadIdx.x; q < 32; q += blockDim.x) r32[N + q] = 0.f;
    for (long long q = threadIdx.x; q < 2 * vecs; q += blockDim.x) yp[q] = 0.f;  // padding stays 0
  }
  double smu = NAN;  // mu of the S band in sm_s (shared-memory mode)
  // r_q = w_q - (S(mu) y)_q, from the staged S(mu) band when it is current (only the
  // diagonals d = 0, 1, b, b + 1 are nonzero: coarse_band_mv)
  const int bb = bw - 1;
  auto resid_row = [&](const double* v, int q, double mu) {
    if (a.smem && smu == mu) return wv[q] - coarse_band_mv(sm_s, bw, bb, v, q, N);
    const double sk = coarse_band_mv(KH, bw, bb, v, q, N), sm = coarse_band_mv(MH, bw, bb, v, q, N);
    return wv[q] - (sk - mu * sm);
  };
  // S(mu) into sm_s: the four nonzero diagonals (all that the products and the block factor read)
  auto stage_s = [&](double mu) {
    if (bb >= 2 && bw == bb + 1) {
      for (int q = threadIdx.x; q < 4 * N; q += blockDim.x) {
        const long long e = (long long)(q >> 2) * bw1 + coarse_band_diag(q & 3, bb);
        sm_s[e] = kh_s[e] - mu * mh_s[e];
      }
    } else {
      for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) sm_s[q] = kh_s[q] - mu * mh_s[q];
    }
    smu = mu;
  };
  const double* part = a.partials + (long long)p * ncx * ncy * 12;
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    int aa = 0;
    while ((aa + 1) * (aa + 2) / 2 <= q) ++aa;
    pairs[q] = (aa << 16) | (q - aa * (aa + 1) / 2);
  }
  // g_a, g_b from the per-cell partials, and y from the previous level's eigenvector,
  // y = -c_H / c_0, whose coarse part differs from this level's by the small change of
  // u_{h_k} between levels (the previous solution warm-starts the first solve). c_prev and
  // this level's output c may be the same buffer: it is read here, written at the end.
  {
    const int ncoef0 = (ncx + 1) * (ncy + 1);
    const double* cpv = a.c_prev + (long long)p * ncoef0;
    const double c0v = a.c0_prev[p];
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      const int X = q % (ncx - 1) + 1, Y = q / (ncx - 1) + 1;
      double sa = 0.0, sb = 0.0, yq = 0.0;
      if (is_free(G, 0, ncx, ncy, X, Y)) {
        const double* c11 = part + ((Y - 1) * ncx + (X - 1)) * 12;
        const double* c01 = part + ((Y - 1) * ncx + X) * 12;
        const double* c10 = part + (Y * ncx + (X - 1)) * 12;
        const double* c00 = part + (Y * ncx + X) * 12;
        sa = c00[3] + c10[4] + c01[5] + c11[6];
        sb = c00[7] + c10[8] + c01[9] + c11[10];
        if (c0v != 0.0) yq = -cpv[Y * (ncx + 1) + X] / c0v;
      }
      ga[q] = sa;
      gb[q] = sb;
      y[q] = yq;
    }
  }
  {
    double v[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < ncx * ncy; q += blockDim.x) {
      v[0] += part[q * 12 + 0];
      v[1] += part[q * 12 + 1];
      v[2] += part[q * 12 + 2];
    }
    block_sum_t<3>(v, stage, red);
  }
  const double alpha = red[0], beta = red[1], sigma = red[2];
  // FP64 scalar work is formed by one thread: a warp's FP64 instruction holds its
  // sub-partition's FP64 pipe for 64 cycles whether one lane or 32 are active, so every
  // warp repeating a division costs the block as much as a vector operation
  if (threadIdx.x == 0) sh_bc[0] = alpha / beta;
  cp_async_wait_all();
  __syncthreads();
  if (a.smem) {
    KH = kh_s;
    MH = mh_s;
  }
  auto band_mv = [&](const double* M, const double* v, int q) { return coarse_band_mv(M, bw, bb, v, q, N); };
  double sig = NAN;  // shift of the current factors
  // FP32 factors of S(mu); false if S(mu) is not positive definite. Blocked mode: the block
  // LDL^T by grid rows (P_I^{-1} in Dinv, W_I in Loff) from the staged FP64 band S(mu);
  // otherwise the column band LDL^T with off-diagonals scaled to L.
  auto factor = [&](double mu) {
    sig = mu;
    if (a.blocked) {
      if (smu != mu) stage_s(mu);
      __syncthreads();
      return BS == 16 ? block_ldlt_f<16>(sm_s, bw1, bsz, nbk, Dinv, Loff, LT, bwork, &bflag)
                      : block_ldlt_f<32>(sm_s, bw1, bsz, nbk, Dinv, Loff, LT, bwork, &bflag);
    }
    for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) Lb[q] = (float)(KH[q] - mu * MH[q]);
    if (!band_ldlt_f(Lb, invD, pairs, npair, N, bw)) return false;
    for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) {
      const int i = (int)(q / bw1), d = (int)(q % bw1);
      if (d > 0 && i - d >= 0) Lb[q] *= invD[i - d];
    }
    __syncthreads();
    return true;
  };
  // w = w(mu) and r = w - S(mu) y for the current y (the previous solution warm-starts the
  // next solve)
  auto start = [&](double mu) {
    for (int q = threadIdx.x; q < N; q += blockDim.x) wv[q] = ga[q] - mu * gb[q];
    if (a.smem && smu != mu) stage_s(mu);
    __syncthreads();
    for (int q = threadIdx.x; q < N; q += blockDim.x) r[q] = resid_row(y, q, mu);
    __syncthreads();
  };
  // y += S(sigma)^{-1} r (FP32 factors), then r = w - S(mu) y in FP64; returns |r|^2 / |w|^2
  auto refine = [&](double mu) {
    if (a.blocked) {
      for (int q = threadIdx.x; q < N; q += blockDim.x) yp[(q / bsz) * BS + q % bsz] = (float)r[q];
      __syncthreads();
      if (BS == 16)
        block_solve_f<16>(Dinv, Loff, LT, yp, xp, bsz, nbk);
      else
        block_solve_f<32>(Dinv, Loff, LT, yp, xp, bsz, nbk);
      for (int q = threadIdx.x; q < N; q += blockDim.x) y[q] += (double)xp[(q / bsz) * BS + q % bsz];
    } else {
      for (int q = threadIdx.x; q < N; q += blockDim.x) r32[q] = (float)r[q];
      __syncthreads();
      band_solve_shfl(Lb, bw1, invD, r32, N, bw);
      for (int q = threadIdx.x; q < N; q += blockDim.x) y[q] += (double)r32[q];
    }
    __syncthreads();
    double v[2] = {0.0, 0.0};
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      const double rq = resid_row(y, q, mu);
      r[q] = rq;
      v[0] += rq * rq;
      v[1] += wv[q] * wv[q];
    }
    block_sum_t<2>(v, stage, red);
    // FP32 ratio: it is only compared against the targets and the previous ratio
    return red[1] > 0.0 ? (double)((float)red[0] / (float)red[1]) : 0.0;
  };
  // refine to rel^2 <= target; false if the iteration stalls first (then refactor at mu)
  auto solve = [&](double mu, double target) {
    start(mu);
    double prev = INFINITY;
    for (int k = 0; k < 16; ++k) {
      const double rel = refine(mu);
      if (rel <= target) return true;
      if (!(rel < 0.1 * prev)) return false;
      prev = rel;
    }
    return false;
  };
  auto eval = [&](double mu, double& f, double& fp) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
      v[0] += wv[q] * y[q];
      v[1] += y[q] * r[q];
      v[2] += gb[q] * y[q];
      v[3] += y[q] * band_mv(MH, y, q);
    }
    block_sum_t<4>(v, stage, red);
    f = alpha - mu * beta - (red[0] + red[1]);
    fp = -beta + 2.0 * red[2] - red[3];
  };
  // squared relative residuals: Newton steps need y to ~1e-6 (the variational f then has a
  // relative error ~1e-12); the eigenvector to ~1e-9 (or until the residual stops falling):
  // its error enters the next level's eigenvalue squared (1e-18), and the returned u at 1e-9
  // is far inside the 1e-6 eigenvector bar of the mixed path
  const double kNewtonTarget = 1e-12, kFinalTarget = 1e-18;
  // Newton stops when its step is below kStep relative: f is concave with its pole at the
  // smallest coarse eigenvalue, a distance d of about 1 % of mu away, so the error left after
  // the last step is about step^2 / d, under 1e-12 relative (the mixed path's bar is 1e-8)
  const double kStep = 1e-7;
  double mu = sh_bc[0], lo = 0.0, hi = INFINITY, lam = NAN;
  int it = 0, status = 0;
  bool have = false, factored = false;
  if (pre_in && pre_ok) {
    // the factors of S(sigma) copied at set-up are valid
    sig = pre_sig;
    factored = true;
    // Newton from the extrapolated shift: it lies within ~1e-7 of lambda_L where alpha / beta
    // lies ~1e-4 above it, which saves a step (S(sigma) factored, so sigma is below the pole;
    // from either side of the root the safeguarded iteration converges)
    if (sig > 0.0 && sig < mu) mu = sig;
  }
  for (; it < a.max_iter; ++it) {
    bool ok = factored && solve(mu, kNewtonTarget);
    if (!ok) {
      if (!factor(mu)) {
        factored = false;
        hi = mu;
        mu = 0.5 * (lo + hi);
        have = false;
        continue;
      }
      factored = true;
      solve(mu, kNewtonTarget);
    }
    have = true;
    double f, fp;
    eval(mu, f, fp);
    if (f > 0.0) lo = mu;
    else hi = mu;
    // the step in FP32 division: its relative error 1e-7 only perturbs the next iterate, and
    // the accepted last step is below kStep |mu|, so lambda gains an error under 1e-14
    const double step = (fp < 0.0) ? (double)(-(float)f / (float)fp) : 0.0;
    if (fp < 0.0 && fabs(step) <= kStep * fabs(mu)) {
      lam = mu + step;
      break;
    }
    double nmu = (fp < 0.0) ? mu + step : 0.5 * (lo + hi);
    if (!(nmu > lo && nmu < hi)) nmu = isfinite(hi) ? 0.5 * (lo + hi) : 2.0 * mu;
    if (isfinite(hi) && hi - lo <= 1e-15 * hi) {
      lam = mu;
      break;
    }
    mu = nmu;
  }
  if (it >= a.max_iter) status |= MLEV_ST_RR_NOCONV;
  if (!(lam == lam)) lam = mu;
  if (!have) {
    if (factor(mu)) {
      factored = true;
      have = true;
    } else {
      status |= MLEV_ST_RR_BREAKDOWN;
    }
  }
  // y = S(mu)^{-1} w to the FP64 floor for the eigenvector; a stall with factors taken at
  // another shift refactors once (a stall at the same shift is the rounding floor)
  // (at lambda, not at the last Newton iterate, so the eigenvector does not depend on where
  // Newton stopped)
  const double mfin = isfinite(lam) ? lam : mu;
  if (have && !solve(mfin, kFinalTarget) && sig != mfin && factor(mfin)) solve(mfin, kFinalTarget);
  double v[3] = {0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    v[0] += y[q] * band_mv(MH, y, q);
    v[1] += gb[q] * y[q];
    v[2] += y[q];
  }
  block_sum_t<3>(v, stage, red);
  if (threadIdx.x == 0) {
    const double bn = red[0] - 2.0 * red[1] + beta;
    const double S = (double)(1LL << (2 * a.L));
    const double integral = sigma - S * red[2];
    sh_bc[1] = (integral >= 0 ? 1.0 : -1.0) / sqrt(bn);
  }
  const int ncoef = (ncx + 1) * (ncy + 1);
  double* cp = a.c + (long long)p * ncoef;
  for (int q = threadIdx.x; q < ncoef; q += blockDim.x) cp[q] = 0.0;
  __syncthreads();
  const double sc = sh_bc[1];
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int X = q % (ncx - 1) + 1, Y = q / (ncx - 1) + 1;
    cp[Y * (ncx + 1) + X] = is_free(G, 0, ncx, ncy, X, Y) ? -sc * y[q] : 0.0;
  }
  if (threadIdx.x == 0) {
    a.c0[p] = sc;
    a.lam[p * (a.n + 1) + a.L] = lam;
    a.stat[p * a.stat_stride + MLEV_STAT_RR_IT + a.L] = it + 1;
    if (!isfinite(lam) || !isfinite(sc)) status |= MLEV_ST_NONFINITE;
    if (status) atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)status);
  }
}

size_t rr_prefactor_smem(int nhb, int bw) {
  const int bsz = bw - 1;
  if (bsz <= 0 || bsz > 32) return (size_t)-1;
  const size_t bs = bsz <= 16 ? 16 : 32;
  return (size_t)nhb * (bw + 1) * 8 + 16 + (3 * (size_t)(nhb / bsz) + 2) * bs * (bs + 4) * 4;
}

// Shared memory of k_rr_mixed: 5 FP64 vectors, K_H, M_H and S(mu), the FP32 band, 2 FP32
// vectors, the row-blocked factors (blocked mode) and the pair table.
size_t rr_mixed_smem_bytes(int nhb, int bw, int blocked) {
  const size_t bsz = bw - 1, bs = bsz <= 16 ? 16 : 32;
  const size_t ts = bs * (bs + 4);  // padded tile
  // 3 tile sets, yp and xp, 2 work tiles, 4 floats of alignment slack
  const size_t blk = blocked && bsz > 0 ? 3 * (nhb / bsz) * ts + 2 * (nhb / bsz) * bs + 2 * ts + 4 : 0;
  return (size_t)nhb * 5 * 8 + 3 * (size_t)nhb * (bw + 1) * 8 +
         ((size_t)nhb * (bw + 1) + 2 * (size_t)nhb + 32 + blk + 2) * 4 + (size_t)(bw * (bw + 1) / 2) * 4 + 16;
}
// The mixed kernel keeps one factorisation pair per thread (bw (bw + 1) / 2 <= 256) and the
// warp solve's window in one warp's lanes (bw <= 31); wider coarse grids use the FP64 kernel.
int rr_mixed_supported(int nhb, int bw) { return bw * (bw + 1) / 2 <= 256 && bw <= 31 && nhb > 0; }

// Shared memory of the Rayleigh-Ritz kernel when its band system is kept on chip.
size_t rr_smem_bytes(int nhb, int bw) {
  return ((size_t)nhb * (bw + 1) + 5 * (size_t)nhb) * 8 + (size_t)(bw * (bw + 1) / 2) * 4;
}

void launch_rr(const DevGeom& G, const RRArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, kRRSmemMax);
    cudaFuncSetAttribute(k_rr_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, kRRSmemMax);
    attr = true;
  }
  const size_t pairs_only = (size_t)(a.bw * (a.bw + 1) / 2) * 4;
  if (a.mixed) {
    const size_t smem = a.smem ? rr_mixed_smem_bytes(a.nhb, a.bw, a.blocked) : pairs_only;
    k_rr_mixed<<<a.B, 256, smem, s>>>(G, a);
    return;
  }
  const size_t smem = a.smem ? rr_smem_bytes(a.nhb, a.bw) : pairs_only;
  k_rr<<<a.B, 256, smem, s>>>(G, a);
}

}  // namespace mlev
