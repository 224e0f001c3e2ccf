// Reverse sweep of Algorithm 4.2: d lambda_{h_n} / d kappa by the adjoint method.
//
// Every step of the forward map is differentiated exactly (the local and strip solves
// as exact solves, the two eigenproblems as exact eigenpairs), and the sweep runs from
// level n down to level 1:
//
// * Rayleigh-Ritz step (Algorithm 4.1 step 3, Eq. Eigen_Augment_Problem). For the pencil
//   (A, B) of order N_H + 1 in the basis Q = [coarse hats, u~] with eigenpair (lambda, c),
//   c^T B c = 1, and adjoints (lambar, cbar = Q^T ubar), the bordered system
//   [[A - lambda B, B c], [c^T B, 0]] [z; sigma] = [cbar - B c (c^T cbar); 0] gives
//   Abar = lambar c c^T - (c z^T + z c^T) / 2 and Bbar = -lambda Abar - (c^T cbar) c c^T / 2.
//   The system is reduced to three banded solves with S(lambda) = K_H - lambda M_H and a
//   2 x 2 system (k_rr_adj).
// * The adjoint of u~ is then c_u ubar + 2 K Q Abar[:, u] + 2 M Q Bbar[:, u] on the free
//   nodes (k_adj_ut); the kappa-derivative of a(Qc, Qc') is the element form of Qc and
//   Qc' (k_grad_aug).
// * G_{m+1} problem (Eq. G_m+1_Problem): one strip solve with the adjoint as right-hand
//   side (the strip matrix is symmetric, so the same multigrid), then its coupling to the
//   glued values and to u_{h_k} (k_strip_adj_post, k_adj_uin).
// * Gluing and auxiliary problems (Eq. Aux_Problem): the adjoint restricted to closed G_j
//   is the right-hand side of one local solve per subdomain (the masked gather); the
//   local solutions e^j are recomputed, not stored, and each subdomain adds
//   -t_j^T dK (u_in + e^j) to the gradient (k_grad_local).
// * Embedding u_{h_k} -> V_{h_{k+1}}: the transpose of P1 interpolation (k_restrict_adj).
// * Level 1 (Algorithm 4.2 step 1): (K_1 - lambda_1 M_1) z = ubar - M_1 u (u^T ubar) with
//   z M-orthogonal to u, by projected conjugate gradients preconditioned with the level-1
//   multigrid (k_level1_adj).
//
// A derivative with respect to the coefficient of a level-l triangle is stored per level
// (a(.,.) is linear in it: dK_T is the element stiffness with kappa = 1) and spread at the
// end to the finest descendants, each with weight 4^{l-n} (a coarser triangle's
// coefficient is the mean of its four children's).
#include "kern_band.cuh"
#include "kern_blk.cuh"
#include "kern_coarse.cuh"
#include "kern_launch.h"

namespace mlev {

constexpr int AX = 32, AY = 8;

__host__ __device__ __forceinline__ int lix(int l) { return l - MLEV_LMIN; }

static dim3 node_grid(const GlobalLayout& gl, int L, int B) {
  return dim3((gl.nx[lix(L)] + 1 + AX - 1) / AX, (gl.ny[lix(L)] + 1 + AY - 1) / AY, B);
}
static dim3 cell_grid(const GlobalLayout& gl, int L, int B) {
  return dim3((gl.nx[lix(L)] + AX - 1) / AX, (gl.ny[lix(L)] + AY - 1) / AY, B);
}

// Label of a free node of level L >= 2 in the quarter-cell map: j + 1 if it lies in the
// closed set G_j (a node on the boundary of G_j belongs to it), 0 on G_{m+1}.
__device__ __forceinline__ int closed_label(const DevGeom& G, int L, int x, int y) {
  const int s = L - 2, qx = 4 * G.ncx;
  const int xa = (x - 1) >> s, xb = x >> s, ya = (y - 1) >> s, yb = y >> s;
  return max(max((int)G.qlabel[ya * qx + xa], (int)G.qlabel[ya * qx + xb]),
             max((int)G.qlabel[yb * qx + xa], (int)G.qlabel[yb * qx + xb]));
}

// a^T K_T b for the lower and upper triangle of one cell with kappa = 1, from the values
// at the corners 00, 10, 01, 11. On the SW-NE triangulation the gradient of a P1 function
// is ((a10 - a00) / h, (a11 - a10) / h) on the lower triangle and
// ((a11 - a01) / h, (a01 - a00) / h) on the upper one; the area h^2 / 2 cancels h^-2.
__device__ __forceinline__ void elem_pair(const double a[4], const double b[4], double& lo, double& up) {
  lo = 0.5 * ((a[1] - a[0]) * (b[1] - b[0]) + (a[3] - a[1]) * (b[3] - b[1]));
  up = 0.5 * ((a[3] - a[2]) * (b[3] - b[2]) + (a[2] - a[0]) * (b[2] - b[0]));
}

// ------------------------------------------------ local right-hand sides restricted to G_j
// Job j's right-hand side is R on the nodes of closed G_j and 0 on the rest of Omega_j.
template <typename T>
__global__ void __launch_bounds__(256) k_gather_masked(DevGeom G, GlobalLayout gl, const Tile* __restrict__ tiles, T* X,
                                                       T* F, double* X64, const double* __restrict__ R) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  const long long c = (long long)j * g.pitch + i;
  X[g.off + c] = (T)0;
  if (X64) X64[g.off64 + c] = 0.0;
  double r = 0.0;
  if (is_unknown(G, g, i, j)) {
    const int x = g.ox + i, y = g.oy + j, sub = g.job - g.problem * G.m;
    if (closed_label(G, g.level, x, y) == sub + 1)
      r = R[(long long)g.problem * gl.bstride + (long long)y * gl.pitch[lix(g.level)] + x];
  }
  F[g.off + c] = (T)r;
}

template <typename T, int KK>
__global__ void __launch_bounds__(256) k_refine_residual_masked(DevGeom G, GlobalLayout gl,
                                                                const Tile* __restrict__ tiles, T* F,
                                                                const double* __restrict__ X64,
                                                                const double* __restrict__ R) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (!is_unknown(G, g, i, j)) return;
  const long long c = (long long)j * g.pitch + i;
  const int x = g.ox + i, y = g.oy + j, sub = g.job - g.problem * G.m;
  const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, x, y);
  const double f = closed_label(G, g.level, x, y) == sub + 1
                       ? R[(long long)g.problem * gl.bstride + (long long)y * gl.pitch[lix(g.level)] + x]
                       : 0.0;
  F[g.off + c] = (T)(f - apply_k<double, double>(X64 + g.off64, c, g.pitch, w));
}

// ------------------------------------------------ cbar = Q^T ubar, per T_H cell
// part2[p][cell][5]: 0 = sum u~ ubar, 1..4 = the cell's share of P_H^T ubar at its corners
// 00, 10, 01, 11 (same ownership of fine nodes as the forward inner products).
__global__ void __launch_bounds__(256) k_cbar(DevGeom G, GlobalLayout gl, int L, const double* ut, const double* ubar,
                                              double* part2) {
  __shared__ double scratch[8 * 5];
  __shared__ double outv[5];
  const int ci = blockIdx.x, cj = blockIdx.y, p = blockIdx.z;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  const int S = 1 << L;
  const double invS = 1.0 / S;
  const double* u = ut + (long long)p * gl.bstride;
  const double* ub = ubar + (long long)p * gl.bstride;
  if (G.cell_in[cj * G.ncx + ci]) {
    for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
      const int ri = q & (S - 1), rj = q >> L;
      const int i = (ci << L) + ri, j = (cj << L) + rj;
      if (!is_free(G, L, nx, ny, i, j)) continue;
      const long long c = (long long)j * pitch + i;
      const double x = ub[c];
      acc[0] += u[c] * x;
      const double s = ri * invS, t = rj * invS;
      if (ri >= rj) {
        acc[1] += (1.0 - s) * x;
        acc[2] += (s - t) * x;
        acc[4] += t * x;
      } else {
        acc[1] += (1.0 - t) * x;
        acc[3] += (t - s) * x;
        acc[4] += s * x;
      }
    }
  }
  block_sum<5>(acc, scratch, outv);
  if (threadIdx.x < 5) part2[((long long)p * G.ncx * G.ncy + cj * G.ncx + ci) * 5 + threadIdx.x] = outv[threadIdx.x];
}

// ------------------------------------------------ Rayleigh-Ritz adjoint (one block per problem)
__global__ void __launch_bounds__(256) k_rr_adj(DevGeom G, RRAdjArgs a) {
  extern __shared__ double ra_sm[];
  __shared__ double scratch[8 * 5];
  __shared__ double red[5];
  __shared__ double sh[2];
  __shared__ int flag;
  const int p = blockIdx.x, N = a.nhb, bw = a.bw, bw1 = bw + 1;
  const int ncx = G.ncx, ncy = G.ncy, ncoef = (ncx + 1) * (ncy + 1);
  const int npair = bw * (bw + 1) / 2;
  double* base = a.smem ? ra_sm : a.scratch + (long long)p * ((long long)N * bw1 + 10LL * N);
  double* Lb = base;
  double* ga = Lb + (long long)N * bw1;
  double* gb = ga + N;
  double* wv = gb + N;
  double* yw = wv + N;
  double* yb = yw + N;
  double* yr = yb + N;
  double* cP = yr + N;
  double* cb = cP + N;
  double* bP = cb + N;
  double* invD = bP + N;
  int* pairs = reinterpret_cast<int*>(a.smem ? invD + N : ra_sm);
  const double* KH = a.KH + (long long)p * N * bw1;
  const double* MH = a.MH + (long long)p * N * bw1;
  const double* part = a.partials + (long long)p * ncx * ncy * 12;
  const double* part2 = a.part2 + (long long)p * ncx * ncy * 5;
  const double* cin = a.c + (long long)p * ncoef;
  const double cu = a.c0[p];
  const double lam = a.lam[p * (a.n + 1) + a.L], lb = a.lambar[p * (a.n + 1) + a.L];
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    int aa = 0;
    while ((aa + 1) * (aa + 2) / 2 <= q) ++aa;
    pairs[q] = (aa << 16) | (q - aa * (aa + 1) / 2);
  }
  {
    double v[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < ncx * ncy; q += blockDim.x) {
      v[0] += part[q * 12 + 0];
      v[1] += part[q * 12 + 1];
      v[2] += part2[q * 5 + 0];
    }
    block_sum<3>(v, scratch, red);
  }
  const double alpha = red[0], beta = red[1], cbu = red[2];
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int X = r % (ncx - 1) + 1, Y = r / (ncx - 1) + 1;
    double sa = 0.0, sb = 0.0, sc = 0.0, cv = 0.0;
    if (is_free(G, 0, ncx, ncy, X, Y)) {
      const int q11 = (Y - 1) * ncx + (X - 1), q01 = (Y - 1) * ncx + X, q10 = Y * ncx + (X - 1), q00 = Y * ncx + X;
      sa = part[q00 * 12 + 3] + part[q10 * 12 + 4] + part[q01 * 12 + 5] + part[q11 * 12 + 6];
      sb = part[q00 * 12 + 7] + part[q10 * 12 + 8] + part[q01 * 12 + 9] + part[q11 * 12 + 10];
      sc = part2[q00 * 5 + 1] + part2[q10 * 5 + 2] + part2[q01 * 5 + 3] + part2[q11 * 5 + 4];
      cv = cin[Y * (ncx + 1) + X];
    }
    ga[r] = sa;
    gb[r] = sb;
    cb[r] = sc;
    cP[r] = cv;
  }
  __syncthreads();
  auto band_mv_m = [&](const double* v, int r) { return coarse_band_mv(MH, bw, bw - 1, v, r, N); };
  // b = B c, s = c^T cbar
  {
    double v[2] = {0.0, 0.0};
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      bP[r] = band_mv_m(cP, r) + gb[r] * cu;
      v[0] += gb[r] * cP[r];
      v[1] += cP[r] * cb[r];
    }
    block_sum<2>(v, scratch, red);
  }
  const double bu = red[0] + beta * cu, sc = red[1] + cu * cbu;
  const double rhs_u = cbu - bu * sc;
  for (long long q = threadIdx.x; q < (long long)N * bw1; q += blockDim.x) Lb[q] = KH[q] - lam * MH[q];
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    wv[r] = ga[r] - lam * gb[r];
    yw[r] = wv[r];
    yb[r] = bP[r];
    yr[r] = cb[r] - bP[r] * sc;
  }
  __syncthreads();
  double* cf = a.coef + (long long)p * a.cstride;
  if (!band_ldlt(Lb, invD, yw, pairs, npair, N, bw, &flag)) {
    for (int q = threadIdx.x; q < a.cstride; q += blockDim.x) cf[q] = 0.0;
    if (threadIdx.x == 0)
      atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_RR_BREAKDOWN);
    return;
  }
  band_back(Lb, invD, yw, N, bw);
  band_fwd(Lb, invD, yb, N, bw);
  band_back(Lb, invD, yb, N, bw);
  band_fwd(Lb, invD, yr, N, bw);
  band_back(Lb, invD, yr, N, bw);
  {
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      v[0] += wv[r] * yw[r];
      v[1] += wv[r] * yb[r];
      v[2] += wv[r] * yr[r];
      v[3] += bP[r] * yb[r];
      v[4] += bP[r] * yr[r];
    }
    block_sum<5>(v, scratch, red);
  }
  if (threadIdx.x == 0) {
    // [[f, m], [m, -q]] [z_u; sigma] = [rhs_u - w^T y_r; -b^T y_r]
    const double f = alpha - lam * beta - red[0], m = bu - red[1], q = red[3];
    const double r0 = rhs_u - red[2], r1 = -red[4];
    const double det = -f * q - m * m;
    sh[0] = (-q * r0 - m * r1) / det;
    sh[1] = (f * r1 - m * r0) / det;
  }
  __syncthreads();
  const double zu = sh[0], sigma = sh[1];
  for (int q = threadIdx.x; q < 3 * ncoef; q += blockDim.x) cf[q] = 0.0;
  __syncthreads();
  const double gamma = lb * cu - 0.5 * zu;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int X = r % (ncx - 1) + 1, Y = r / (ncx - 1) + 1;
    if (!is_free(G, 0, ncx, ncy, X, Y)) continue;
    const double zp = yr[r] - yw[r] * zu - yb[r] * sigma;
    const double qa = gamma * cP[r] - 0.5 * cu * zp;  // coarse part of Q Abar[:, u]
    const int o = Y * (ncx + 1) + X;
    cf[o] = zp;
    cf[ncoef + o] = 2.0 * qa;
    cf[2 * ncoef + o] = 2.0 * lam * qa + sc * cu * cP[r];
  }
  if (threadIdx.x == 0) {
    const double qu = gamma * cu - 0.5 * cu * zu;   // u~ part of Q Abar[:, u]
    double* s = cf + 3 * ncoef;
    s[ADJ_CU] = cu;
    s[ADJ_ZU] = zu;
    s[ADJ_KAU] = 2.0 * qu;
    s[ADJ_MAU] = 2.0 * lam * qu + sc * cu * cu;
    s[ADJ_LAMBAR] = lb;
    s[ADJ_LAM] = lam;
    s[ADJ_SC] = sc;
    s[ADJ_SIGMA] = sigma;
    if (!isfinite(zu) || !isfinite(sigma))
      atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_NONFINITE);
  }
}

size_t rr_adj_smem_bytes(int nhb, int bw) {
  return ((size_t)nhb * (bw + 1) + 10 * (size_t)nhb) * 8 + (size_t)(bw * (bw + 1) / 2) * 4;
}

// ------------------------------------------------ adjoint of u~ from the Rayleigh-Ritz step
// utbar = c_u ubar + K (P kac + ka_u u~) - M (P mac + ma_u u~) on free nodes, 0 elsewhere.
template <int KK>
__global__ void __launch_bounds__(256) k_adj_ut(DevGeom G, GlobalLayout gl, int L, const double* ut,
                                                const double* ubar, const double* coef, int cstride, double* utbar) {
  const int p = blockIdx.z;
  const int i = blockIdx.x * AX + threadIdx.x, j = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  if (i > nx || j > ny) return;
  const long long base = (long long)p * gl.bstride, c = (long long)j * pitch + i;
  if (!is_free(G, L, nx, ny, i, j)) {
    utbar[base + c] = 0.0;
    return;
  }
  const int ncoef = (G.ncx + 1) * (G.ncy + 1);
  const double* cf = coef + (long long)p * cstride;
  const double* kac = cf + ncoef;
  const double* mac = cf + 2 * ncoef;
  const double* sc = cf + 3 * ncoef;
  const double kau = sc[ADJ_KAU], mau = sc[ADJ_MAU], cu = sc[ADJ_CU];
  const double* u = ut + base;
  // stencil nodes: 0 c, 1 E, 2 W, 3 N, 4 S, 5 NE, 6 SW
  const int di[7] = {0, 1, -1, 0, 0, 1, -1}, dj[7] = {0, 0, 0, 1, -1, 1, -1};
  double fk[5], fm[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int x = i + di[k], y = j + dj[k];
    const double uv = u[c + dj[k] * (long long)pitch + di[k]];
    fm[k] = coarse_eval(G, mac, L, x, y) + mau * uv;
    if (k < 5) fk[k] = coarse_eval(G, kac, L, x, y) + kau * uv;
  }
  const W4 w = edge_weights<KK>(G.kap, p, L, i, j);
  const double h = level_h(G.H, L);
  const double kf = (w.e + w.w + w.n + w.s) * fk[0] - w.e * fk[1] - w.w * fk[2] - w.n * fk[3] - w.s * fk[4];
  const double mf = (h * h / 12.0) * (6.0 * fm[0] + fm[1] + fm[2] + fm[3] + fm[4] + fm[5] + fm[6]);
  utbar[base + c] = cu * ubar[base + c] + kf - mf;
}

// ------------------------------------------------ element contributions
__device__ __forceinline__ double aug_value(const DevGeom& G, const GlobalLayout& gl, const AugField& f, int p, int L,
                                            int x, int y) {
  double v = (f.s ? f.s[(long long)p * f.sstride] : 1.0) *
             f.f[(long long)p * gl.bstride + (long long)y * gl.pitch[lix(L)] + x];
  if (f.c) v += coarse_eval(G, f.c + (long long)p * f.cstride, L, x, y);
  return v;
}

// gl_lvl[p][cell][t] += w11 * f1^T K_T f1 + w12 * f1^T K_T f2 on every level-L cell.
__global__ void __launch_bounds__(256) k_grad_aug(DevGeom G, GlobalLayout gl, int L, AugField f1, AugField f2,
                                                  const double* w11, int w11_stride, double w12, double* gl_lvl) {
  const int p = blockIdx.z;
  const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)];
  if (x >= nx || y >= ny) return;
  double a[4], b[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = aug_value(G, gl, f1, p, L, x + (k & 1), y + (k >> 1));
    b[k] = aug_value(G, gl, f2, p, L, x + (k & 1), y + (k >> 1));
  }
  double l11, u11, l12, u12;
  elem_pair(a, a, l11, u11);
  elem_pair(a, b, l12, u12);
  const double ww = w11[(long long)p * w11_stride];
  double* g = gl_lvl + ((long long)p * ny * nx + (long long)y * nx + x) * 2;
  g[0] += ww * l11 + w12 * l12;
  g[1] += ww * u11 + w12 * u12;
}

__global__ void __launch_bounds__(256) k_grad_pair(DevGeom G, GlobalLayout gl, int L, double w, const double* fa,
                                                   const double* fb, double* gl_lvl) {
  const int p = blockIdx.z;
  const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  if (x >= nx || y >= ny) return;
  const long long c = (long long)p * gl.bstride + (long long)y * pitch + x;
  const double a[4] = {fa[c], fa[c + 1], fa[c + pitch], fa[c + pitch + 1]};
  const double b[4] = {fb[c], fb[c + 1], fb[c + pitch], fb[c + pitch + 1]};
  double lo, up;
  elem_pair(a, b, lo, up);
  double* g = gl_lvl + ((long long)p * ny * nx + (long long)y * nx + x) * 2;
  g[0] += w * lo;
  g[1] += w * up;
}

// -t_j^T dK (u_in + e^j) summed over the subdomains whose window holds the cell, in
// subdomain order (deterministic, no atomics).
__global__ void __launch_bounds__(256) k_grad_local(DevGeom G, GlobalLayout gl, int L, const double* Tb,
                                                    const double* E, int use64, const double* uin, double* gl_lvl) {
  const int p = blockIdx.z;
  const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  if (x >= nx || y >= ny) return;
  if (!G.cell_in[(y >> L) * G.ncx + (x >> L)]) return;
  const long long gc = (long long)p * gl.bstride + (long long)y * pitch + x;
  const double ui[4] = {uin[gc], uin[gc + 1], uin[gc + pitch], uin[gc + pitch + 1]};
  double slo = 0.0, sup = 0.0;
  for (int sj = 0; sj < G.m; ++sj) {
    const GridDesc& g = G.grids[G.sub_top[p * G.m + sj]];
    const int i = x - g.ox, j = y - g.oy;
    if (i < 0 || j < 0 || i >= g.nx || j >= g.ny) continue;
    const long long o = (use64 ? g.off64 : g.off) + (long long)j * g.pitch + i;
    double t[4], v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ii = i + (k & 1), jj = j + (k >> 1);
      const long long ok = o + (long long)(k >> 1) * g.pitch + (k & 1);
      const bool un = is_unknown(G, g, ii, jj);
      t[k] = un ? Tb[ok] : 0.0;
      v[k] = ui[k] + (un ? E[ok] : 0.0);
    }
    double lo, up;
    elem_pair(t, v, lo, up);
    slo += lo;
    sup += up;
  }
  double* gg = gl_lvl + ((long long)p * ny * nx + (long long)y * nx + x) * 2;
  gg[0] -= slo;
  gg[1] -= sup;
}

// rbar = sum_j t_j (extended by zero) on every free node.
__global__ void __launch_bounds__(256) k_rbar(DevGeom G, GlobalLayout gl, int L, const double* Tb, int use64,
                                              double* rbar) {
  const int p = blockIdx.z;
  const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  if (x > nx || y > ny) return;
  double s = 0.0;
  if (is_free(G, L, nx, ny, x, y)) {
    for (int sj = 0; sj < G.m; ++sj) {
      const GridDesc& g = G.grids[G.sub_top[p * G.m + sj]];
      const int i = x - g.ox, j = y - g.oy;
      if (i < 1 || j < 1 || i >= g.nx || j >= g.ny || !is_unknown(G, g, i, j)) continue;
      s += Tb[(use64 ? g.off64 : g.off) + (long long)j * g.pitch + i];
    }
  }
  rbar[(long long)p * gl.bstride + (long long)y * pitch + x] = s;
}

// After the strip solve: utbar <- utbar - K sbar off the strip, 0 on the strip and off the free nodes.
template <int KK>
__global__ void __launch_bounds__(256) k_strip_adj_post(DevGeom G, GlobalLayout gl, int L, double* utbar,
                                                        const double* sbar) {
  const int p = blockIdx.z;
  const int i = blockIdx.x * AX + threadIdx.x, j = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  if (i > nx || j > ny) return;
  const long long base = (long long)p * gl.bstride, c = (long long)j * pitch + i;
  if (!is_free(G, L, nx, ny, i, j) || closed_label(G, L, i, j) == 0) {
    utbar[base + c] = 0.0;
    return;
  }
  const W4 w = edge_weights<KK>(G.kap, p, L, i, j);
  utbar[base + c] -= apply_k<double, double>(sbar + base, c, pitch, w);
}

// utbar <- utbar + lambda_k M (sbar + rbar) - K rbar (the adjoint of u_in), and the block
// partials of lambdabar_k = u_in^T M (sbar + rbar).
template <int KK>
__global__ void __launch_bounds__(256) k_adj_uin(DevGeom G, GlobalLayout gl, int L, double* utbar, const double* sbar,
                                                 const double* rbar, const double* uin, const double* lam,
                                                 int lam_stride, double* lbpart, int nblk_stride) {
  __shared__ double scratch[8];
  __shared__ double outv[1];
  const int p = blockIdx.z;  // 1-D blocks of AX * AY threads (block_sum wants a linear id)
  const int i = blockIdx.x * AX + threadIdx.x % AX, j = blockIdx.y * AY + threadIdx.x / AX;
  const int nx = gl.nx[lix(L)], ny = gl.ny[lix(L)], pitch = gl.pitch[lix(L)];
  double acc[1] = {0.0};
  if (i <= nx && j <= ny) {
    const long long base = (long long)p * gl.bstride, c = (long long)j * pitch + i;
    if (!is_free(G, L, nx, ny, i, j)) {
      utbar[base + c] = 0.0;
    } else {
      const double* sb = sbar + base;
      const double* rb = rbar + base;
      const double h = level_h(G.H, L);
      const double lamk = lam[p * lam_stride + (L - 1)];
      const double mq = (h * h / 12.0) * (apply_m12<double, double>(sb, c, pitch) + apply_m12<double, double>(rb, c, pitch));
      const W4 w = edge_weights<KK>(G.kap, p, L, i, j);
      utbar[base + c] += lamk * mq - apply_k<double, double>(rb, c, pitch, w);
      acc[0] = uin[base + c] * mq;
    }
  }
  block_sum<1>(acc, scratch, outv);
  if (threadIdx.x == 0)
    lbpart[(long long)p * nblk_stride + blockIdx.y * gridDim.x + blockIdx.x] = outv[0];
}

__global__ void __launch_bounds__(256) k_lambar_finalize(int nblk, int nblk_stride, const double* lbpart,
                                                         double* lambar, int lam_stride, int k) {
  __shared__ double scratch[8];
  __shared__ double outv[1];
  const int p = blockIdx.x;
  double acc[1] = {0.0};
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) acc[0] += lbpart[(long long)p * nblk_stride + q];
  block_sum<1>(acc, scratch, outv);
  if (threadIdx.x == 0) lambar[p * lam_stride + k] = outv[0];
}

__global__ void k_lambar_init(int B, int n, const double* dl, double* lambar) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B * (n + 1)) return;
  const int p = q / (n + 1), k = q % (n + 1);
  lambar[q] = k == n ? dl[p] : 0.0;
}

// ubar_k = I^T uinbar (transpose of the P1 embedding of level k into level k+1), 0 off the
// free nodes of level k.
__global__ void __launch_bounds__(256) k_restrict_adj(DevGeom G, GlobalLayout gl, int k, const double* fine,
                                                      double* coarse) {
  const int p = blockIdx.z;
  const int I = blockIdx.x * AX + threadIdx.x, J = blockIdx.y * AY + threadIdx.y;
  const int nx = gl.nx[lix(k)], ny = gl.ny[lix(k)], pc = gl.pitch[lix(k)], pf = gl.pitch[lix(k + 1)];
  if (I > nx || J > ny) return;
  const long long base = (long long)p * gl.bstride;
  double v = 0.0;
  if (is_free(G, k, nx, ny, I, J)) {
    const double* f = fine + base;
    const long long c = (long long)(2 * J) * pf + 2 * I;
    v = f[c] + 0.5 * (f[c + 1] + f[c - 1] + f[c + pf] + f[c - pf] + f[c + pf + 1] + f[c - pf - 1]);
  }
  coarse[base + (long long)J * pc + I] = v;
}

// ------------------------------------------------ level-1 eigenvector adjoint
// (K_1 - lambda_1 M_1) z = ubar - M_1 u (u^T ubar), u^T M_1 z = 0, by flexible projected
// conjugate gradients: the preconditioner is Pi C Pi^T with C one level-1 V-cycle for K_1,
// Pi = I - u (M u)^T (onto the M-orthogonal complement of u) and Pi^T = I - (M u) u^T.
template <typename T, int KK>
__global__ void __launch_bounds__(1024) k_level1_adj(DevGeom G, GlobalLayout gl, Level1AdjArgs a) {
  __shared__ double scratch[32 * 4];
  __shared__ double red[4];
  const int p = blockIdx.x;
  const int g0 = a.grid_begin + p * a.nlev;
  const GridDesc& g = G.grids[g0];
  const long long vs = a.vstride;
  double* U = a.vec + (long long)p * 10 * vs;
  double *MU = U + vs, *Z = MU + vs, *R = Z + vs, *P = R + vs, *AP = P + vs, *W = AP + vs, *WO = W + vs;
  T* xp = (T*)a.xpool;
  T* fp = (T*)a.fpool;
  const int nx = g.nx, ny = g.ny, pitch = g.pitch, nn = (nx + 1) * (ny + 1);
  const double h = level_h(G.H, 1), m12 = h * h / 12.0;
  const double lam = a.lam[p * a.lam_stride + 1];
  const double* u1 = a.ut1 + (long long)p * gl.bstride;
  const double* ub = a.ubar1 + (long long)p * gl.bstride;
  auto cidx = [&](int q) { return (long long)(q / (nx + 1)) * pitch + q % (nx + 1); };
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int i = q % (nx + 1), j = q / (nx + 1);
    const long long c = (long long)j * pitch + i;
    U[c] = is_unknown(G, g, i, j) ? u1[c] : 0.0;
    Z[c] = P[c] = AP[c] = W[c] = WO[c] = 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int i = q % (nx + 1), j = q / (nx + 1);
    const long long c = (long long)j * pitch + i;
    MU[c] = is_unknown(G, g, i, j) ? m12 * apply_m12<double, double>(U, c, pitch) : 0.0;
  }
  __syncthreads();
  {
    double v[2] = {0.0, 0.0};
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = cidx(q);
      v[0] += U[c] * ub[c];
      v[1] += U[c] * MU[c];
    }
    block_sum<2>(v, scratch, red);
  }
  const double s = red[0] / red[1], umu = red[1];
  double rr0;
  {
    double v[1] = {0.0};
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = cidx(q);
      R[c] = ub[c] - MU[c] * s;  // ubar and M u vanish off the unknowns
      v[0] += R[c] * R[c];
    }
    block_sum<1>(v, scratch, red);
    rr0 = red[0];
  }
  // w = Pi C Pi^T r
  auto precondition = [&]() {
    double v[1] = {0.0};
    for (int q = threadIdx.x; q < nn; q += blockDim.x) v[0] += U[cidx(q)] * R[cidx(q)];
    block_sum<1>(v, scratch, red);
    const double ur = red[0] / umu;
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = cidx(q);
      fp[g.off + c] = (T)(R[c] - MU[c] * ur);
      xp[g.off + c] = (T)0;
    }
    __syncthreads();
    blk_vcycle<T, KK>(G, G.grids + g0, a.nlev, xp, fp, a.pre, a.post, a.coarse_sweeps, (T)a.omega, nullptr);
    double v2[1] = {0.0};
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = cidx(q);
      W[c] = (double)xp[g.off + c];
      v2[0] += MU[c] * W[c];
    }
    block_sum<1>(v2, scratch, red);
    const double mw = red[0] / umu;
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
      const long long c = cidx(q);
      W[c] -= U[c] * mw;
    }
    __syncthreads();
  };
  int it = 0;
  bool conv = rr0 == 0.0;
  if (!conv) {
    precondition();
    double rho;
    {
      double v[1] = {0.0};
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const long long c = cidx(q);
        P[c] = W[c];
        v[0] += R[c] * W[c];
      }
      block_sum<1>(v, scratch, red);
      rho = red[0];
    }
    for (; it < a.max_iter; ++it) {
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const int i = q % (nx + 1), j = q / (nx + 1);
        const long long c = (long long)j * pitch + i;
        if (!is_unknown(G, g, i, j)) {
          AP[c] = 0.0;
          continue;
        }
        const W4 w = edge_weights<KK>(G.kap, p, 1, i, j);
        AP[c] = apply_k<double, double>(P, c, pitch, w) - lam * m12 * apply_m12<double, double>(P, c, pitch);
      }
      __syncthreads();
      double pap;
      {
        double v[1] = {0.0};
        for (int q = threadIdx.x; q < nn; q += blockDim.x) v[0] += P[cidx(q)] * AP[cidx(q)];
        block_sum<1>(v, scratch, red);
        pap = red[0];
      }
      if (!(pap > 0.0)) break;
      const double alpha = rho / pap;
      // convergence on Pi^T r: u is an eigenvector only up to the level-1 eigen-residual, so
      // the component of r along M u is the system's inconsistency, not solver error
      double rr;
      {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = threadIdx.x; q < nn; q += blockDim.x) {
          const long long c = cidx(q);
          Z[c] += alpha * P[c];
          R[c] -= alpha * AP[c];
          WO[c] = W[c];
          v[0] += R[c] * R[c];
          v[1] += U[c] * R[c];
          v[2] += MU[c] * R[c];
          v[3] += MU[c] * MU[c];
        }
        block_sum<4>(v, scratch, red);
        const double cu = red[1] / umu;
        rr = fmax(red[0] - 2.0 * cu * red[2] + cu * cu * red[3], 0.0);
      }
      if (rr <= a.tol * a.tol * rr0) {
        conv = true;
        ++it;
        break;
      }
      precondition();
      double rho_new, rwo;
      {
        double v[2] = {0.0, 0.0};
        for (int q = threadIdx.x; q < nn; q += blockDim.x) {
          const long long c = cidx(q);
          v[0] += R[c] * W[c];
          v[1] += R[c] * WO[c];
        }
        block_sum<2>(v, scratch, red);
        rho_new = red[0];
        rwo = red[1];
      }
      const double beta = (rho_new - rwo) / rho;
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const long long c = cidx(q);
        P[c] = W[c] + beta * P[c];
      }
      rho = rho_new;
      __syncthreads();
    }
  }
  // z <- Pi z (removes rounding drift along u), written in the global level-1 layout
  {
    double v[1] = {0.0};
    for (int q = threadIdx.x; q < nn; q += blockDim.x) v[0] += MU[cidx(q)] * Z[cidx(q)];
    block_sum<1>(v, scratch, red);
  }
  const double mz = red[0] / umu;
  double* out = a.zout + (long long)p * gl.bstride;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const long long c = cidx(q);
    out[c] = Z[c] - U[c] * mz;
  }
  if (threadIdx.x == 0 && !conv)
    atomicOr((unsigned long long*)&a.stat[p * a.stat_stride + MLEV_STAT_FLAGS], (unsigned long long)MLEV_ST_ADJ_NOCONV);
}

// ------------------------------------------------ spreading the per-level gradients
// layout MLEV_GRAD_FINE_ELEM: out[p][fy][fx][t] = sum_l 4^{l-n} G_l[ancestor]; a finest
// triangle (t) of fine cell (fx, fy) lies in the level-l triangle of cell (fx >> s, fy >> s),
// s = n - l, that is lower if the local cell (li, lj) has li > lj, upper if li < lj, and
// of its own type on the diagonal.
__global__ void __launch_bounds__(256) k_grad_spread_fine(GlobalLayout gl, int n, GradLevels lv, const double* glb,
                                                          double* out) {
  const int p = blockIdx.z;
  const int fx = blockIdx.x * AX + threadIdx.x, fy = blockIdx.y * AY + threadIdx.y;
  const int fnx = gl.nx[lix(n)], fny = gl.ny[lix(n)];
  if (fx >= fnx || fy >= fny) return;
  double acc[2] = {0.0, 0.0};
  for (int l = 1; l <= n; ++l) {
    const int s = n - l, mask = (1 << s) - 1;
    const int li = fx & mask, lj = fy & mask;
    const int nxl = gl.nx[lix(l)], nyl = gl.ny[lix(l)];
    const double* gg = glb + lv.off[l] + ((long long)p * nyl * nxl + (long long)(fy >> s) * nxl + (fx >> s)) * 2;
    const double wgt = 1.0 / (double)(1LL << (2 * s));
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int tl = li > lj ? 0 : (li < lj ? 1 : t);
      acc[t] += wgt * gg[tl];
    }
  }
  double* o = out + ((long long)p * fny * fnx + (long long)fy * fnx + fx) * 2;
  o[0] = acc[0];
  o[1] = acc[1];
}

// layout MLEV_GRAD_COARSE_CELL: out[p][cy][cx] = sum over every level of the gradients of
// the triangles inside T_H cell (cx, cy) (the chain rule for a coefficient constant per cell).
__global__ void __launch_bounds__(256) k_grad_spread_cell(GlobalLayout gl, int n, int ncx, int ncy, GradLevels lv,
                                                          const double* glb, double* out) {
  __shared__ double scratch[8];
  __shared__ double outv[1];
  const int cx = blockIdx.x, cy = blockIdx.y, p = blockIdx.z;
  double acc[1] = {0.0};
  for (int l = 1; l <= n; ++l) {
    const int S = 1 << l, nxl = gl.nx[lix(l)], nyl = gl.ny[lix(l)];
    const double* gg = glb + lv.off[l] + (long long)p * nyl * nxl * 2;
    for (int q = threadIdx.x; q < S * S * 2; q += blockDim.x) {
      const int t = q & 1, r = q >> 1, ri = r % S, rj = r / S;
      acc[0] += gg[((long long)(cy * S + rj) * nxl + cx * S + ri) * 2 + t];
    }
  }
  block_sum<1>(acc, scratch, outv);
  if (threadIdx.x == 0) out[(long long)p * ncx * ncy + cy * ncx + cx] = outv[0];
}

// ------------------------------------------------------------------ launchers
#define MLEV_ADJ_KK(kk, ...)                         \
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

template <typename T>
void launch_gather_masked(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* X, T* F, double* X64,
                          const double* R, cudaStream_t s) {
  if (!n) return;
  k_gather_masked<T><<<n, dim3(AX, AY), 0, s>>>(G, gl, tiles, X, F, X64, R);
}
template <typename T>
void launch_refine_residual_masked(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* F,
                                   const double* X64, const double* R, cudaStream_t s) {
  if (!n) return;
  MLEV_ADJ_KK(G.kap.kind, (k_refine_residual_masked<T, KK><<<n, dim3(AX, AY), 0, s>>>(G, gl, tiles, F, X64, R)));
}
template void launch_gather_masked<float>(const DevGeom&, const GlobalLayout&, const Tile*, int, float*, float*,
                                          double*, const double*, cudaStream_t);
template void launch_gather_masked<double>(const DevGeom&, const GlobalLayout&, const Tile*, int, double*, double*,
                                           double*, const double*, cudaStream_t);
template void launch_refine_residual_masked<float>(const DevGeom&, const GlobalLayout&, const Tile*, int, float*,
                                                   const double*, const double*, cudaStream_t);
template void launch_refine_residual_masked<double>(const DevGeom&, const GlobalLayout&, const Tile*, int, double*,
                                                    const double*, const double*, cudaStream_t);

void launch_cbar(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* ut, const double* ubar,
                 double* part2, cudaStream_t s) {
  k_cbar<<<dim3(G.ncx, G.ncy, B), 256, 0, s>>>(G, gl, L, ut, ubar, part2);
}

void launch_rr_adj(const DevGeom& G, const RRAdjArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rr_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, kRRSmemMax);
    attr = true;
  }
  const size_t smem = a.smem ? rr_adj_smem_bytes(a.nhb, a.bw) : (size_t)(a.bw * (a.bw + 1) / 2) * 4;
  k_rr_adj<<<a.B, 256, smem, s>>>(G, a);
}

void launch_adj_ut(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* ut, const double* ubar,
                   const double* coef, int cstride, double* utbar, cudaStream_t s) {
  MLEV_ADJ_KK(G.kap.kind,
              (k_adj_ut<KK><<<node_grid(gl, L, B), dim3(AX, AY), 0, s>>>(G, gl, L, ut, ubar, coef, cstride, utbar)));
}

void launch_grad_aug(const DevGeom& G, const GlobalLayout& gl, int L, int B, const AugField& f1, const AugField& f2,
                     const double* w11, int w11_stride, double w12, double* gl_lvl, cudaStream_t s) {
  k_grad_aug<<<cell_grid(gl, L, B), dim3(AX, AY), 0, s>>>(G, gl, L, f1, f2, w11, w11_stride, w12, gl_lvl);
}

void launch_grad_pair(const DevGeom& G, const GlobalLayout& gl, int L, int B, double w, const double* a,
                      const double* b, double* gl_lvl, cudaStream_t s) {
  k_grad_pair<<<cell_grid(gl, L, B), dim3(AX, AY), 0, s>>>(G, gl, L, w, a, b, gl_lvl);
}

void launch_strip_adj_post(const DevGeom& G, const GlobalLayout& gl, int L, int B, double* utbar, const double* sbar,
                           cudaStream_t s) {
  MLEV_ADJ_KK(G.kap.kind, (k_strip_adj_post<KK><<<node_grid(gl, L, B), dim3(AX, AY), 0, s>>>(G, gl, L, utbar, sbar)));
}

void launch_grad_local(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* T_, const double* E,
                       int use64, const double* uin, double* gl_lvl, cudaStream_t s) {
  k_grad_local<<<cell_grid(gl, L, B), dim3(AX, AY), 0, s>>>(G, gl, L, T_, E, use64, uin, gl_lvl);
}

void launch_rbar(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* T_, int use64, double* rbar,
                 cudaStream_t s) {
  k_rbar<<<node_grid(gl, L, B), dim3(AX, AY), 0, s>>>(G, gl, L, T_, use64, rbar);
}

int adj_uin_blocks(const GlobalLayout& gl, int L) {
  const dim3 g = node_grid(gl, L, 1);
  return (int)(g.x * g.y);
}

void launch_adj_uin(const DevGeom& G, const GlobalLayout& gl, int L, int B, double* utbar, const double* sbar,
                    const double* rbar, const double* uin, const double* lam, int lam_stride, double* lbpart,
                    int nblk_stride, cudaStream_t s) {
  MLEV_ADJ_KK(G.kap.kind, (k_adj_uin<KK><<<node_grid(gl, L, B), AX * AY, 0, s>>>(
                              G, gl, L, utbar, sbar, rbar, uin, lam, lam_stride, lbpart, nblk_stride)));
}

void launch_lambar_finalize(int B, int nblk, int nblk_stride, const double* lbpart, double* lambar, int lam_stride,
                            int k, cudaStream_t s) {
  k_lambar_finalize<<<B, 256, 0, s>>>(nblk, nblk_stride, lbpart, lambar, lam_stride, k);
}

void launch_lambar_init(int B, int n, const double* dl, double* lambar, cudaStream_t s) {
  const int tot = B * (n + 1);
  k_lambar_init<<<(tot + 127) / 128, 128, 0, s>>>(B, n, dl, lambar);
}

void launch_restrict_adj(const DevGeom& G, const GlobalLayout& gl, int k, int B, const double* fine, double* coarse,
                         cudaStream_t s) {
  k_restrict_adj<<<node_grid(gl, k, B), dim3(AX, AY), 0, s>>>(G, gl, k, fine, coarse);
}

template <typename T>
void launch_level1_adj(const DevGeom& G, const GlobalLayout& gl, const Level1AdjArgs& a, cudaStream_t s) {
  MLEV_ADJ_KK(G.kap.kind, (k_level1_adj<T, KK><<<a.B, 1024, 0, s>>>(G, gl, a)));
}
template void launch_level1_adj<float>(const DevGeom&, const GlobalLayout&, const Level1AdjArgs&, cudaStream_t);
template void launch_level1_adj<double>(const DevGeom&, const GlobalLayout&, const Level1AdjArgs&, cudaStream_t);

void launch_grad_spread(const DevGeom& G, const GlobalLayout& gl, int n, int B, const GradLevels& lv,
                        const double* glbase, int layout, double* out, cudaStream_t s) {
  if (layout == MLEV_GRAD_COARSE_CELL)
    k_grad_spread_cell<<<dim3(G.ncx, G.ncy, B), 256, 0, s>>>(gl, n, G.ncx, G.ncy, lv, glbase, out);
  else
    k_grad_spread_fine<<<cell_grid(gl, n, B), dim3(AX, AY), 0, s>>>(gl, n, lv, glbase, out);
}

}  // namespace mlev
