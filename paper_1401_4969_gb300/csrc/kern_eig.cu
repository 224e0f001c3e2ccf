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

  auto band_mv_m = [&](const double* v, int r) {
    double my = MH[(long long)r * bw1] * v[r];
    for (int d = 1; d <= bw; ++d) {
      if (r - d >= 0) my += MH[(long long)r * bw1 + d] * v[r - d];
      if (r + d < N) my += MH[(long long)(r + d) * bw1 + d] * v[r + d];
    }
    return my;
  };
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

// Shared memory of the Rayleigh-Ritz kernel when its band system is kept on chip.
size_t rr_smem_bytes(int nhb, int bw) {
  return ((size_t)nhb * (bw + 1) + 5 * (size_t)nhb) * 8 + (size_t)(bw * (bw + 1) / 2) * 4;
}

void launch_rr(const DevGeom& G, const RRArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, kRRSmemMax);
    attr = true;
  }
  const size_t smem = a.smem ? rr_smem_bytes(a.nhb, a.bw) : (size_t)(a.bw * (a.bw + 1) / 2) * 4;
  k_rr<<<a.B, 256, smem, s>>>(G, a);
}

}  // namespace mlev
