// Kernels on whole-domain fields of one level (all FP64): the embedding of
// u_{h_k} into V_{h_{k+1}}, the right-hand side of the auxiliary problems, the
// gluing of step 2, the G_{m+1} right-hand side, the inner products of step 3,
// and set-up kernels for kappa and the coarse matrices.
#include "kern_band.cuh"
#include "kern_coarse.cuh"
#include "kern_launch.h"
#include "kern_tail.cuh"

namespace mlev {

constexpr int GX = 32, GY = 8;

__host__ __device__ __forceinline__ int lidx(int l) { return l - MLEV_LMIN; }

// Exact embedding V_{h_{L-1}} -> V_{h_L} of a pitched level-(L-1) field at node (i, j).
__device__ __forceinline__ double embed(const double* u, int pitch, int i, int j) {
  const int I = i >> 1, J = j >> 1;
  if (!(i & 1) && !(j & 1)) return u[(long long)J * pitch + I];
  if ((i & 1) && !(j & 1)) return 0.5 * (u[(long long)J * pitch + I] + u[(long long)J * pitch + I + 1]);
  if (!(i & 1) && (j & 1)) return 0.5 * (u[(long long)J * pitch + I] + u[(long long)(J + 1) * pitch + I]);
  return 0.5 * (u[(long long)J * pitch + I] + u[(long long)(J + 1) * pitch + I + 1]);
}

// u_in = c0 * u~_{L-1} + sum_i c_i phi_i on level L (u_{h_k} of Algorithm 4.1 as an
// element of V_{h_{k+1}}), zero on dOmega.
__global__ void __launch_bounds__(256) k_interp(DevGeom G, GlobalLayout gl, LevelArgs a) {
  const int p = blockIdx.z, L = a.L;
  const int i = blockIdx.x * GX + threadIdx.x, j = blockIdx.y * GY + threadIdx.y;
  const int nx = gl.nx[lidx(L)], ny = gl.ny[lidx(L)];
  if (i > nx || j > ny) return;
  const long long idx = (long long)p * gl.bstride + (long long)j * gl.pitch[lidx(L)] + i;
  if (!is_free(G, L, nx, ny, i, j)) {
    a.uin[idx] = 0.0;
    return;
  }
  const double* prev = a.ut_prev + (long long)p * gl.bstride;
  const double v = embed(prev, gl.pitch[lidx(L - 1)], i, j);
  a.uin[idx] = a.c0[p] * v + coarse_eval(G, a.c + (long long)p * (G.ncx + 1) * (G.ncy + 1), L, i, j);
}

// Right-hand side of Eq. Aux_Problem in nodal form: r = lambda_k M u - K u on free nodes.
template <int KK>
__global__ void __launch_bounds__(256) k_rhs(DevGeom G, GlobalLayout gl, LevelArgs a) {
  const int p = blockIdx.z, L = a.L;
  const int i = blockIdx.x * GX + threadIdx.x, j = blockIdx.y * GY + threadIdx.y;
  const int nx = gl.nx[lidx(L)], ny = gl.ny[lidx(L)], pitch = gl.pitch[lidx(L)];
  if (i > nx || j > ny) return;
  const long long base = (long long)p * gl.bstride, c = (long long)j * pitch + i;
  if (!is_free(G, L, nx, ny, i, j)) {
    a.r[base + c] = 0.0;
    return;
  }
  const double lam = a.lam[p * a.lam_stride + (L - 1)];
  const double* u = a.uin + base;
  if (KK == MLEV_KAPPA_ONE) {
    double ku, mu;
    apply_km_one<double, double>(u, c, pitch, ku, mu);
    a.r[base + c] = (lam * a.m12) * mu - ku;
    return;
  }
  const W4 w = edge_weights<KK>(G.kap, p, L, i, j);
  a.r[base + c] = lam * a.m12 * apply_m12<double, double>(u, c, pitch) - apply_k<double, double>(u, c, pitch, w);
}

// Step 2 of Algorithm 4.1: u~ = u_in + e^j on closed G_j, u_in on G_{m+1} (corrected
// later by the G_{m+1} solve), 0 on dOmega. e^j is read from the FP64 pool E, or widened from
// the FP32 multigrid pool E32 when that holds the whole solution (one pass, mixed precision).
__global__ void __launch_bounds__(256) k_glue(DevGeom G, GlobalLayout gl, LevelArgs a, const double* E, int use64,
                                              const float* E32) {
  const int p = blockIdx.z, L = a.L;
  const int i = blockIdx.x * GX + threadIdx.x, j = blockIdx.y * GY + threadIdx.y;
  const int nx = gl.nx[lidx(L)], ny = gl.ny[lidx(L)], pitch = gl.pitch[lidx(L)];
  if (i > nx || j > ny) return;
  const long long idx = (long long)p * gl.bstride + (long long)j * pitch + i;
  if (!is_free(G, L, nx, ny, i, j)) {
    a.ut[idx] = 0.0;
    return;
  }
  const int s = L - 2, qx = 4 * G.ncx;
  const int xa = (i - 1) >> s, xb = i >> s, ya = (j - 1) >> s, yb = j >> s;
  int lab = max(max((int)G.qlabel[ya * qx + xa], (int)G.qlabel[ya * qx + xb]),
                max((int)G.qlabel[yb * qx + xa], (int)G.qlabel[yb * qx + xb]));
  double v = a.uin[idx];
  if (lab > 0) {
    const GridDesc& g = G.grids[G.sub_top[p * G.m + lab - 1]];
    const long long c = (long long)(j - g.oy) * g.pitch + (i - g.ox);
    v += E32 ? (double)E32[g.off + c] : E[(use64 ? g.off64 : g.off) + c];
  }
  a.ut[idx] = v;
}

// Right-hand side of Eq. G_m+1_Problem for the correction d = u~^{m+1} - u_in on
// G_{m+1}: R = lambda_k M u_in - K u~ (u~ = glued values, u_in on the strip). Stored in
// FP64 in the global R field (for refinement) and as T in the strip's finest grid.
template <typename T, int KK>
__global__ void __launch_bounds__(256) k_strip_rhs(DevGeom G, GlobalLayout gl, LevelArgs a, const Tile* __restrict__ tiles,
                                                   T* X, T* F, double* X64) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  const long long c = (long long)j * g.pitch + i;
  X[g.off + c] = (T)0;
  if (X64) X64[g.off64 + c] = 0.0;
  if (!is_unknown(G, g, i, j)) {
    F[g.off + c] = (T)0;
    return;
  }
  const int L = g.level, p = g.problem, pitch = gl.pitch[lidx(L)];
  const long long base = (long long)p * gl.bstride, gc = (long long)j * pitch + i;
  const double lam = a.lam[p * a.lam_stride + (L - 1)];
  const W4 w = edge_weights<KK>(G.kap, p, L, i, j);
  const double r = lam * a.m12 * apply_m12<double, double>(a.uin + base, gc, pitch) -
                   apply_k<double, double>(a.ut + base, gc, pitch, w);
  a.r[base + gc] = r;
  F[g.off + c] = (T)r;
}

__global__ void __launch_bounds__(256) k_strip_update(DevGeom G, GlobalLayout gl, LevelArgs a, const Tile* __restrict__ tiles,
                                                      const double* E, int use64, const float* E32) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (!is_unknown(G, g, i, j)) return;
  const long long c = (long long)j * g.pitch + i;
  a.ut[(long long)g.problem * gl.bstride + (long long)j * gl.pitch[lidx(g.level)] + i] +=
      E32 ? (double)E32[g.off + c] : E[(use64 ? g.off64 : g.off) + c];
}

// Step 3 inputs on one T_H cell: alpha = a(u~,u~), beta = b(u~,u~), sigma = sum of u~,
// and the cell's share of g_a = P_H^T K u~, g_b = P_H^T M u~ at its four corners, summed
// by the nt threads tid = 0 .. nt-1 into acc (each thread's partial sums).
// partials[p][cell][12]: 0 alpha, 1 beta, 2 sigma, 3..6 K-part at corners 00,10,01,11,
// 7..10 M-part at corners 00,10,01,11.
template <int KK>
__device__ __forceinline__ void aug_cell(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, int p, int ci,
                                         int cj, int tid, int nt, double (&acc)[11]) {
#pragma unroll
  for (int k = 0; k < 11; ++k) acc[k] = 0.0;
  if (!G.cell_in[cj * G.ncx + ci]) return;
  const int L = a.L;
  const int nx = gl.nx[lidx(L)], ny = gl.ny[lidx(L)], pitch = gl.pitch[lidx(L)];
  const int S = 1 << L;
  const double invS = pow2(-L);
  const double* u = a.ut + (long long)p * gl.bstride;
  // Thread layout: a fixed column ri of the cell (s = ri / S) and every nt/S-th row. The
  // hats of the cell's corners are linear in t = rj / S on each triangle (lower rj <= ri:
  // 1 - s, s - t, 0, t; upper: 1 - t, 0, t - s, s), so per thread and column it suffices
  // to sum ku, t ku, mu, t mu over the lower and the upper nodes; the weights are applied
  // once per column and h^2 / 12 once at the end.
  const int cstep = S < nt ? S : nt, rstep = S < nt ? nt / S : 1;
  for (int ri = tid % cstep; ri < S; ri += cstep) {
    const double s = ri * invS, dt = rstep * invS;
    double skl = 0.0, tkl = 0.0, sml = 0.0, tml = 0.0, sku = 0.0, tku = 0.0, smu = 0.0, tmu = 0.0;
    int rj = S < nt ? tid / S : 0;
    double t = rj * invS;
    for (; rj < S; rj += rstep, t += dt) {
      const int i = (ci << L) + ri, j = (cj << L) + rj;
      if (!is_free(G, L, nx, ny, i, j)) continue;
      const long long c = (long long)j * pitch + i;
      const double uc = u[c];
      double ku, mu;  // K u and M u / (h^2 / 12)
      if (KK == MLEV_KAPPA_ONE) {
        apply_km_one<double, double>(u, c, pitch, ku, mu);
      } else {
        const W4 w = edge_weights<KK>(G.kap, p, L, i, j);
        ku = apply_k<double, double>(u, c, pitch, w);
        mu = apply_m12<double, double>(u, c, pitch);
      }
      acc[0] += uc * ku;
      acc[1] += uc * mu;
      acc[2] += uc;
      if (rj > ri) {  // upper triangle
        sku += ku;
        tku += t * ku;
        smu += mu;
        tmu += t * mu;
      } else {
        skl += ku;
        tkl += t * ku;
        sml += mu;
        tml += t * mu;
      }
    }
    acc[3] += (1.0 - s) * skl + sku - tku;
    acc[4] += s * skl - tkl;
    acc[5] += tku - s * sku;
    acc[6] += tkl + s * sku;
    acc[7] += (1.0 - s) * sml + smu - tmu;
    acc[8] += s * sml - tml;
    acc[9] += tmu - s * smu;
    acc[10] += tml + s * smu;
  }
  acc[1] *= a.m12;
#pragma unroll
  for (int k = 7; k < 11; ++k) acc[k] *= a.m12;
}

// One block of 256 threads per T_H cell (cells of 64 x 64 fine nodes or more).
template <int KK, bool PRE>
__global__ void __launch_bounds__(256) k_aug(DevGeom G, GlobalLayout gl, LevelArgs a, double* partials,
                                             RRPrefactor pf) {
  extern __shared__ double aug_dyn[];
  __shared__ double stage[11 * 256];
  __shared__ double outv[11];
  __shared__ int pflag;
  // with PRE, blocks [0, B) prepare the Rayleigh-Ritz factors (first, so they start first),
  // then one block per coarse cell of each batch member (a separate instantiation, so the
  // plain kernel keeps its default shared-memory configuration)
  const long long npre = PRE ? a.B : 0;
  if (PRE && (long long)blockIdx.x < npre) {
    const int p = blockIdx.x;
    const long long band = (long long)pf.nhb * (pf.bw + 1);
    rr_prefactor_block(pf.KH + p * band, pf.MH + p * band, a.lam + (long long)p * a.lam_stride, a.L, pf.nhb, pf.bw,
                       pf.out + p * pf.stride, aug_dyn, &pflag);
    return;
  }
  const long long q = (long long)blockIdx.x - npre;
  const int ncell = G.ncx * G.ncy;
  const int p = (int)(q / ncell), ci = (int)(q % ncell) % G.ncx, cj = (int)(q % ncell) / G.ncx;
  double acc[11];
  aug_cell<KK>(G, gl, a, p, ci, cj, threadIdx.x, blockDim.x, acc);
  block_sum_t<11>(acc, stage, outv);
  if (threadIdx.x < 11) partials[((long long)p * G.ncx * G.ncy + cj * G.ncx + ci) * 12 + threadIdx.x] = outv[threadIdx.x];
}

// One warp per T_H cell, 8 cells per block (cells of at most 32 x 32 fine nodes, where a
// block per cell would give each thread a node or two and spend its time in the block
// reduction); the sums are reduced by shuffles within the warp.
template <int KK, bool PRE>
__global__ void __launch_bounds__(256) k_aug_warp(DevGeom G, GlobalLayout gl, LevelArgs a, double* partials,
                                                  RRPrefactor pf) {
  extern __shared__ double aug_dyn[];
  __shared__ int pflag;
  const long long npre = PRE ? a.B : 0;
  if (PRE && (long long)blockIdx.x < npre) {
    const int p = blockIdx.x;
    const long long band = (long long)pf.nhb * (pf.bw + 1);
    rr_prefactor_block(pf.KH + p * band, pf.MH + p * band, a.lam + (long long)p * a.lam_stride, a.L, pf.nhb, pf.bw,
                       pf.out + p * pf.stride, aug_dyn, &pflag);
    return;
  }
  const int ncell = G.ncx * G.ncy;
  const long long q = ((long long)blockIdx.x - npre) * 8 + (threadIdx.x >> 5);
  if (q >= (long long)a.B * ncell) return;
  const int lane = threadIdx.x & 31;
  const int p = (int)(q / ncell), ci = (int)(q % ncell) % G.ncx, cj = (int)(q % ncell) / G.ncx;
  double acc[11];
  aug_cell<KK>(G, gl, a, p, ci, cj, lane, 32, acc);
#pragma unroll
  for (int k = 0; k < 11; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  if (lane == 0) {
    double* out = partials + ((long long)p * ncell + cj * G.ncx + ci) * 12;
#pragma unroll
    for (int k = 0; k < 11; ++k) out[k] = acc[k];
  }
}

// u_out = c0 u~ + P_H c on level L, dense (ny+1) x (nx+1) per problem.
__global__ void __launch_bounds__(256) k_output_u(DevGeom G, GlobalLayout gl, int L, const double* ut, const double* c,
                                                  const double* c0, double* out) {
  const int p = blockIdx.z;
  const int i = blockIdx.x * GX + threadIdx.x, j = blockIdx.y * GY + threadIdx.y;
  const int nx = gl.nx[lidx(L)], ny = gl.ny[lidx(L)];
  if (i > nx || j > ny) return;
  double v = 0.0;
  if (is_free(G, L, nx, ny, i, j))
    v = c0[p] * ut[(long long)p * gl.bstride + (long long)j * gl.pitch[lidx(L)] + i] +
        coarse_eval(G, c + (long long)p * (G.ncx + 1) * (G.ncy + 1), L, i, j);
  out[(long long)p * (nx + 1) * (ny + 1) + (long long)j * (nx + 1) + i] = v;
}

// Finest-level triangle values copied into the per-level table (and its FP32 copy).
__global__ void k_kappa_copy_fine(KappaDev kv, int n, int B, const double* src, double* lvl, float* lvl_f) {
  const long long per = (long long)lvl_cells_x(kv, n) * lvl_cells_y(kv, n) * 2;
  const long long tot = per * B;
  const long long off = kv.lvl_off[lidx(n)];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    lvl[off + q] = src[q];
    lvl_f[off + q] = (float)src[q];
  }
}

// FP32 copy of the per-coarse-cell coefficient.
__global__ void k_kappa_to_f(long long tot, const double* src, float* dst) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x)
    dst[q] = (float)src[q];
}

// Triangle values of level l as the mean of their four children on level l+1 (the
// exact P1 stiffness of the coarser triangle; children as in regular refinement).
template <int KK>
__global__ void k_kappa_average(KappaDev kv, int l, int B, double* lvl, float* lvl_f) {
  const int nx = lvl_cells_x(kv, l), ny = lvl_cells_y(kv, l);
  const long long tot = (long long)nx * ny * B;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(q / ((long long)nx * ny));
    const int r = (int)(q % ((long long)nx * ny));
    const int x = r % nx, y = r / nx;
    const int X = 2 * x, Y = 2 * y;
    const double lo = 0.25 * (kap_tri<KK>(kv, p, l + 1, X, Y, 0) + kap_tri<KK>(kv, p, l + 1, X + 1, Y, 0) +
                              kap_tri<KK>(kv, p, l + 1, X + 1, Y + 1, 0) + kap_tri<KK>(kv, p, l + 1, X + 1, Y, 1));
    const double up = 0.25 * (kap_tri<KK>(kv, p, l + 1, X, Y, 1) + kap_tri<KK>(kv, p, l + 1, X + 1, Y + 1, 1) +
                              kap_tri<KK>(kv, p, l + 1, X, Y + 1, 1) + kap_tri<KK>(kv, p, l + 1, X, Y + 1, 0));
    const long long o = kv.lvl_off[lidx(l)] + (long long)p * kv.lvl_bstride[lidx(l)] + (long long)r * 2;
    lvl[o] = lo;
    lvl[o + 1] = up;
    lvl_f[o] = (float)lo;
    lvl_f[o + 1] = (float)up;
  }
}

// Coarse pencil (K_H, M_H) in symmetric band storage: row r = (Y-1)(ncx-1) + (X-1) for
// the T_H node (X, Y); entry [r][d] = A(r, r-d), d = 0..bw. Nodes on dOmega become
// identity rows of K_H (zero rows of M_H) so the band stays regular.
template <int KK>
__global__ void k_band_setup(DevGeom G, int B, int nhb, int bw, double* KH, double* MH) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nhb * B) return;
  const int p = q / nhb, r = q % nhb;
  const int X = r % (G.ncx - 1) + 1, Y = r / (G.ncx - 1) + 1;
  double* kr = KH + ((long long)p * nhb + r) * (bw + 1);
  double* mr = MH + ((long long)p * nhb + r) * (bw + 1);
  for (int d = 0; d <= bw; ++d) kr[d] = mr[d] = 0.0;
  if (!is_free(G, 0, G.ncx, G.ncy, X, Y)) {
    kr[0] = 1.0;
    return;
  }
  const double H2 = G.H * G.H;
  const W4 w = edge_weights<KK>(G.kap, p, 0, X, Y);
  kr[0] = w.e + w.w + w.n + w.s;
  mr[0] = H2 / 2.0;
  if (X > 1 && is_free(G, 0, G.ncx, G.ncy, X - 1, Y)) {
    kr[1] = -w.w;
    mr[1] = H2 / 12.0;
  }
  if (Y > 1 && is_free(G, 0, G.ncx, G.ncy, X, Y - 1)) {
    kr[G.ncx - 1] = -w.s;
    mr[G.ncx - 1] = H2 / 12.0;
  }
  if (X > 1 && Y > 1 && is_free(G, 0, G.ncx, G.ncy, X - 1, Y - 1)) mr[G.ncx] = H2 / 12.0;
}

__global__ void k_lambda_out(int B, int n, const double* lam, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < B) out[p] = lam[p * (n + 1) + n];
}

// ------------------------------------------------------------------ launchers
#define MLEV_DISPATCH_KK(kk, ...)                    \
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

static dim3 global_grid(const GlobalLayout& gl, int L, int B) {
  return dim3((gl.nx[lidx(L)] + 1 + GX - 1) / GX, (gl.ny[lidx(L)] + 1 + GY - 1) / GY, B);
}

void launch_interp(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, cudaStream_t s) {
  k_interp<<<global_grid(gl, a.L, a.B), dim3(GX, GY), 0, s>>>(G, gl, a);
}
void launch_rhs(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, cudaStream_t s) {
  MLEV_DISPATCH_KK(G.kap.kind, (k_rhs<KK><<<global_grid(gl, a.L, a.B), dim3(GX, GY), 0, s>>>(G, gl, a)));
}
void launch_glue(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, const double* E, int use64, const float* E32,
                 cudaStream_t s) {
  k_glue<<<global_grid(gl, a.L, a.B), dim3(GX, GY), 0, s>>>(G, gl, a, E, use64, E32);
}
template <typename T>
void launch_strip_rhs(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, const Tile* tiles, int n, T* X,
                      T* F, double* X64, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_strip_rhs<T, KK><<<n, dim3(GX, GY), 0, s>>>(G, gl, a, tiles, X, F, X64)));
}
template void launch_strip_rhs<float>(const DevGeom&, const GlobalLayout&, const LevelArgs&, const Tile*, int, float*,
                                      float*, double*, cudaStream_t);
template void launch_strip_rhs<double>(const DevGeom&, const GlobalLayout&, const LevelArgs&, const Tile*, int,
                                       double*, double*, double*, cudaStream_t);
void launch_strip_update(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, const Tile* tiles, int n,
                         const double* E, int use64, const float* E32, cudaStream_t s) {
  if (!n) return;
  k_strip_update<<<n, dim3(GX, GY), 0, s>>>(G, gl, a, tiles, E, use64, E32);
}
template <int KK>
static void launch_aug_kk(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, double* partials,
                          const RRPrefactor* pf, cudaStream_t s) {
  const long long cells = (long long)a.B * G.ncx * G.ncy;
  const bool warp = a.L <= 5;  // cells of at most 32 x 32 fine nodes
  if (!pf) {
    if (warp)
      k_aug_warp<KK, false><<<(unsigned)((cells + 7) / 8), 256, 0, s>>>(G, gl, a, partials, RRPrefactor{});
    else
      k_aug<KK, false><<<(unsigned)cells, 256, 0, s>>>(G, gl, a, partials, RRPrefactor{});
    return;
  }
  static bool attr = false, attr_w = false;
  if (warp) {
    if (!attr_w) {
      cudaFuncSetAttribute(k_aug_warp<KK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRRSmemMax);
      attr_w = true;
    }
    const long long nb = (long long)a.B + (cells + 7) / 8;
    k_aug_warp<KK, true><<<(unsigned)nb, 256, rr_prefactor_smem(pf->nhb, pf->bw), s>>>(G, gl, a, partials, *pf);
    return;
  }
  if (!attr) {
    cudaFuncSetAttribute(k_aug<KK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRRSmemMax);
    attr = true;
  }
  const long long nb = (long long)a.B * (G.ncx * G.ncy + 1);
  k_aug<KK, true><<<(unsigned)nb, 256, rr_prefactor_smem(pf->nhb, pf->bw), s>>>(G, gl, a, partials, *pf);
}
void launch_aug(const DevGeom& G, const GlobalLayout& gl, const LevelArgs& a, double* partials, const RRPrefactor* pf,
                cudaStream_t s) {
  MLEV_DISPATCH_KK(G.kap.kind, (launch_aug_kk<KK>(G, gl, a, partials, pf, s)));
}
void launch_output_u(const DevGeom& G, const GlobalLayout& gl, int L, int B, const double* ut, const double* c,
                     const double* c0, double* u_out, cudaStream_t s) {
  k_output_u<<<global_grid(gl, L, B), dim3(GX, GY), 0, s>>>(G, gl, L, ut, c, c0, u_out);
}
void launch_kappa_copy_fine(const KappaDev& kv, int n, int B, const double* src, double* lvl, float* lvl_f,
                            cudaStream_t s) {
  k_kappa_copy_fine<<<1024, 256, 0, s>>>(kv, n, B, src, lvl, lvl_f);
}
void launch_kappa_to_f(long long count, const double* src, float* dst, cudaStream_t s) {
  k_kappa_to_f<<<256, 256, 0, s>>>(count, src, dst);
}
void launch_kappa_average(const KappaDev& kv, int l, int B, double* lvl, float* lvl_f, cudaStream_t s) {
  MLEV_DISPATCH_KK(kv.kind, (k_kappa_average<KK><<<1024, 256, 0, s>>>(kv, l, B, lvl, lvl_f)));
}
void launch_band_setup(const DevGeom& G, int B, int nhb, int bw, double* KH, double* MH, cudaStream_t s) {
  const int n = nhb * B;
  MLEV_DISPATCH_KK(G.kap.kind, (k_band_setup<KK><<<(n + 127) / 128, 128, 0, s>>>(G, B, nhb, bw, KH, MH)));
}
void launch_lambda_out(int B, int n, const double* lam, double* out, cudaStream_t s) {
  k_lambda_out<<<(B + 127) / 128, 128, 0, s>>>(B, n, lam, out);
}

}  // namespace mlev
