// Batched geometric multigrid for the masked SPD problems of Algorithm 4.1:
// the auxiliary problems on Omega_j (Eq. Aux_Problem) and the G_{m+1} problem
// (Eq. G_m+1_Problem). Every launch covers the grids of one depth of ALL jobs of all
// batch members through a tile list, so uneven subdomains share one launch.
//
// Hierarchy: the spaces V_{0h_l}(region) for l = top .. coarsest are nested because
// every region is a union of cells of its coarsest level, so prolongation is exact P1
// interpolation on the SW-NE mesh (the coarse hat's values 1 at the node and 1/2 at the
// midpoints of its six incident edges E, W, N, S, NE, SW), restriction is its
// transpose, and rediscretisation with the level's kappa equals the Galerkin
// operator. The smoother is red-black Gauss-Seidel (the stiffness is a 5-point
// stencil, so colours decouple).
#include "kern_launch.h"

namespace mlev {

constexpr int TX = 32, TY = 8;
constexpr int kCoarsestSmemMax = 220 * 1024;

// One thread per node of the colour: a tile's 32 columns hold 16 nodes of each colour per
// row (x0 is a multiple of 32), so the 16 x 8 threads take column x0 + 2 tx + ((color + j) & 1).
template <typename T, int KK>
__global__ void __launch_bounds__(128) k_smooth(DevGeom G, const Tile* __restrict__ tiles, T* X, const T* __restrict__ F,
                                                int color, T omega) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int j = t.y0 + threadIdx.y, i = t.x0 + 2 * threadIdx.x + ((color + j) & 1);
  if (!is_unknown(G, g, i, j)) return;
  T* x = X + g.off;
  const long long c = (long long)j * g.pitch + i;
  const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  const T s = F[g.off + c] + (T)w.e * x[c + 1] + (T)w.w * x[c - 1] + (T)w.n * x[c + g.pitch] + (T)w.s * x[c - g.pitch];
  x[c] += omega * (div_diag<T>(s, (T)(w.e + w.w + w.n + w.s)) - x[c]);
}

// r = f - A x at node (i, j) of grid g (0 off the unknowns).
template <typename T, int KK>
__device__ __forceinline__ T residual_at(const DevGeom& G, const GridDesc& g, const T* X, const T* F, int i, int j) {
  if (!is_unknown(G, g, i, j)) return (T)0;
  const long long c = (long long)j * g.pitch + i;
  const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  return F[g.off + c] - apply_k<T, T>(X + g.off, c, g.pitch, w);
}

// Coarse grid (tiles over depth d+1): f_c = P^T (f - A x)_fine, x_c = 0. With `black_zero`
// the fine grid was just pre-smoothed by plain Gauss-Seidel (omega = 1) ending with the black
// half-sweep: the residual of every black node (odd i + j) is then zero, since each was
// relaxed against its red neighbours and black nodes do not couple, so of the seven fine
// nodes of the coarse hat only the red ones (the node itself, NE and SW) contribute.
template <typename T, int KK>
__global__ void __launch_bounds__(256) k_restrict(DevGeom G, const Tile* __restrict__ tiles, T* X, T* F,
                                                  int black_zero) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& gc = G.grids[t.grid];
  const GridDesc& gf = G.grids[t.grid - 1];
  const int I = t.x0 + threadIdx.x, J = t.y0 + threadIdx.y;
  if (I > gc.nx || J > gc.ny) return;
  const long long cc = (long long)J * gc.pitch + I;
  X[gc.off + cc] = (T)0;
  if (!is_unknown(G, gc, I, J)) return;
  const int i = 2 * I, j = 2 * J;
  T acc = residual_at<T, KK>(G, gf, X, F, i, j);
  T half = residual_at<T, KK>(G, gf, X, F, i + 1, j + 1) + residual_at<T, KK>(G, gf, X, F, i - 1, j - 1);
  if (!black_zero)
    half += residual_at<T, KK>(G, gf, X, F, i + 1, j) + residual_at<T, KK>(G, gf, X, F, i - 1, j) +
            residual_at<T, KK>(G, gf, X, F, i, j + 1) + residual_at<T, KK>(G, gf, X, F, i, j - 1);
  F[gc.off + cc] = acc + (T)0.5 * half;
}

// Fine grid (tiles over depth d): x += P x_c. With `red_only` the post-smoothing that follows
// starts with a plain Gauss-Seidel (omega = 1) black half-sweep, which sets every black node
// from its red neighbours alone, so only the red nodes take the correction.
// RED: 16 x 8 threads, one per red node of the 32 x 8 tile (x0 even: column x0 + 2 tx + (j & 1)).
template <typename T, bool RED>
__global__ void __launch_bounds__(256) k_prolong(DevGeom G, const Tile* __restrict__ tiles, T* X) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& gf = G.grids[t.grid];
  const GridDesc& gc = G.grids[t.grid + 1];
  const int j = t.y0 + threadIdx.y, i = RED ? t.x0 + 2 * threadIdx.x + (j & 1) : t.x0 + threadIdx.x;
  if (!is_unknown(G, gf, i, j)) return;
  const T* xc = X + gc.off;
  const int I = i >> 1, J = j >> 1;
  T v;
  if (!(i & 1) && !(j & 1))
    v = xc[(long long)J * gc.pitch + I];
  else if ((i & 1) && !(j & 1))
    v = (T)0.5 * (xc[(long long)J * gc.pitch + I] + xc[(long long)J * gc.pitch + I + 1]);
  else if (!(i & 1) && (j & 1))
    v = (T)0.5 * (xc[(long long)J * gc.pitch + I] + xc[(long long)(J + 1) * gc.pitch + I]);
  else
    v = (T)0.5 * (xc[(long long)J * gc.pitch + I] + xc[(long long)(J + 1) * gc.pitch + I + 1]);
  X[gf.off + (long long)j * gf.pitch + i] += v;
}

// Coarsest grids: one block per job, `sweeps` symmetric red-black sweeps.
template <typename T, int KK>
__global__ void __launch_bounds__(256) k_coarsest(DevGeom G, const Tile* __restrict__ tiles, T* X, const T* __restrict__ F,
                                                  int sweeps, T omega) {
  const GridDesc& g = G.grids[tiles[blockIdx.x].grid];
  const int nn = (g.nx + 1) * (g.ny + 1);
  T* x = X + g.off;
  for (int s = 0; s < sweeps; ++s) {
    for (int color = 0; color < 2; ++color) {
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const int i = q % (g.nx + 1), j = q / (g.nx + 1);
        if (((i + j) & 1) != color || !is_unknown(G, g, i, j)) continue;
        const long long c = (long long)j * g.pitch + i;
        const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
        const T v = F[g.off + c] + (T)w.e * x[c + 1] + (T)w.w * x[c - 1] + (T)w.n * x[c + g.pitch] +
                    (T)w.s * x[c - g.pitch];
        x[c] += omega * (div_diag<T>(v, (T)(w.e + w.w + w.n + w.s)) - x[c]);
      }
      __syncthreads();
    }
  }
}

// Exact solve on the coarsest grid of every subdomain job (its T_H window, at most
// MLEV_DIRECT_MAX nodes): the matrix of the window's interior nodes (identity rows for
// nodes that are not unknowns) is assembled in FP64 and inverted by Gauss-Jordan
// elimination without pivoting (SPD), once per solve; the inverse is kept in T.
template <typename T, int KK>
__global__ void __launch_bounds__(256) k_coarse_inverse(DevGeom G, const Tile* __restrict__ tiles, T* inv, int nd_max) {
  extern __shared__ double smA[];
  const GridDesc& g = G.grids[tiles[blockIdx.x].grid];
  const int nx1 = g.nx - 1, ny1 = g.ny - 1, nd = nx1 * ny1;
  double* A = smA;            // nd x nd
  double* colk = A + nd * nd; // nd
  for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) A[q] = 0.0;
  __syncthreads();
  for (int r = threadIdx.x; r < nd; r += blockDim.x) {
    const int i = r % nx1 + 1, j = r / nx1 + 1;
    if (!is_unknown(G, g, i, j)) {
      A[r * nd + r] = 1.0;
      continue;
    }
    const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
    A[r * nd + r] = w.e + w.w + w.n + w.s;
    if (i + 1 <= nx1 && is_unknown(G, g, i + 1, j)) A[r * nd + r + 1] = -w.e;
    if (i - 1 >= 1 && is_unknown(G, g, i - 1, j)) A[r * nd + r - 1] = -w.w;
    if (j + 1 <= ny1 && is_unknown(G, g, i, j + 1)) A[r * nd + r + nx1] = -w.n;
    if (j - 1 >= 1 && is_unknown(G, g, i, j - 1)) A[r * nd + r - nx1] = -w.s;
  }
  for (int k = 0; k < nd; ++k) {
    __syncthreads();
    const double ip = 1.0 / A[k * nd + k];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) colk[i] = (i == k) ? 0.0 : A[i * nd + k];
    __syncthreads();
    for (int c = threadIdx.x; c < nd; c += blockDim.x) A[k * nd + c] = (c == k ? 1.0 : A[k * nd + c]) * ip;
    __syncthreads();
    for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) {
      const int i = q / nd, c = q % nd;
      if (i == k) continue;
      A[q] = (c == k ? 0.0 : A[q]) - colk[i] * A[k * nd + c];
    }
  }
  __syncthreads();
  T* out = inv + (long long)g.job * nd_max * nd_max;
  for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) out[q] = (T)A[q];
}

template <typename T>
__global__ void __launch_bounds__(128) k_coarsest_direct(DevGeom G, const Tile* __restrict__ tiles, T* X,
                                                         const T* __restrict__ F, const T* __restrict__ inv,
                                                         int nd_max) {
  extern __shared__ unsigned char smraw[];
  T* f = reinterpret_cast<T*>(smraw);
  const GridDesc& g = G.grids[tiles[blockIdx.x].grid];
  const int nx1 = g.nx - 1, ny1 = g.ny - 1, nd = nx1 * ny1;
  for (int r = threadIdx.x; r < nd; r += blockDim.x) {
    const int i = r % nx1 + 1, j = r / nx1 + 1;
    f[r] = is_unknown(G, g, i, j) ? F[g.off + (long long)j * g.pitch + i] : (T)0;
  }
  __syncthreads();
  const T* A = inv + (long long)g.job * nd_max * nd_max;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < nd; r += nw) {  // one warp per row of the inverse
    T sacc = (T)0;
    for (int c = lane; c < nd; c += 32) sacc += A[r * nd + c] * f[c];
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
    if (lane == 0) {
      const int i = r % nx1 + 1, j = r / nx1 + 1;
      X[g.off + (long long)j * g.pitch + i] = is_unknown(G, g, i, j) ? sacc : (T)0;
    }
  }
}

// Coarsest grid staged in shared memory (the strip's T_{h_2} window): per-node weights
// and inverse diagonals are computed once, then `sweeps` red-black sweeps run from
// shared memory with one block of 1024 threads per job.
template <typename T, int KK>
__global__ void __launch_bounds__(1024) k_coarsest_smem(DevGeom G, const Tile* __restrict__ tiles, T* X,
                                                        const T* __restrict__ F, int sweeps, T omega) {
  constexpr bool kOne = (KK == MLEV_KAPPA_ONE);  // unit weights: store none
  extern __shared__ unsigned char smraw[];
  const GridDesc& g = G.grids[tiles[blockIdx.x].grid];
  const int W = g.nx + 1, nn = W * (g.ny + 1);
  T* x = reinterpret_cast<T*>(smraw);
  T* f = x + nn;
  T* idg = f + nn;  // inverse diagonal; 0 marks a node that is not an unknown
  T* we = idg + nn;
  T* ww = we + (kOne ? 0 : nn);
  T* wn = ww + (kOne ? 0 : nn);
  T* wsx = wn + (kOne ? 0 : nn);
  // block 32 x 32: rows by threadIdx.y, columns by threadIdx.x
  for (int j = threadIdx.y; j <= g.ny; j += blockDim.y)
    for (int i = threadIdx.x; i <= g.nx; i += blockDim.x) {
      const int q = j * W + i;
      const long long c = (long long)j * g.pitch + i;
      x[q] = X[g.off + c];
      if (is_unknown(G, g, i, j)) {
        const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
        f[q] = F[g.off + c];
        idg[q] = (T)1 / (w.e + w.w + w.n + w.s);
        if (!kOne) {
          we[q] = (T)w.e; ww[q] = (T)w.w; wn[q] = (T)w.n; wsx[q] = (T)w.s;
        }
      } else {
        f[q] = (T)0;
        idg[q] = (T)0;
      }
    }
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      for (int j = 1 + threadIdx.y; j < g.ny; j += blockDim.y) {
        const int i0 = ((color + j) & 1) ? 1 : 2;
        for (int i = i0 + 2 * threadIdx.x; i < g.nx; i += 2 * blockDim.x) {
          const int q = j * W + i;
          if (idg[q] == (T)0) continue;
          T v;
          if (kOne)
            v = f[q] + x[q + 1] + x[q - 1] + x[q + W] + x[q - W];
          else
            v = f[q] + we[q] * x[q + 1] + ww[q] * x[q - 1] + wn[q] * x[q + W] + wsx[q] * x[q - W];
          x[q] += omega * (v * idg[q] - x[q]);
        }
      }
      __syncthreads();
    }
  for (int j = threadIdx.y; j <= g.ny; j += blockDim.y)
    for (int i = threadIdx.x; i <= g.nx; i += blockDim.x) X[g.off + (long long)j * g.pitch + i] = x[j * W + i];
}

// Finest grids of subdomain jobs: f = R (global residual of Eq. Aux_Problem restricted
// to Omega_j) and, when the FP64 accumulator is in use, x64 = 0 (x starts at zero: the
// caller clears the whole pool before).
template <typename T>
__global__ void __launch_bounds__(256) k_gather(DevGeom G, GlobalLayout gl, const Tile* __restrict__ tiles, T* X, T* F,
                                                double* X64, const double* __restrict__ R) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  const long long c = (long long)j * g.pitch + i;
  if (X64) X64[g.off64 + c] = 0.0;  // X itself: the caller clears the whole pool first
  const int li = g.level - MLEV_LMIN;
  const double r = is_unknown(G, g, i, j)
                       ? R[(long long)g.problem * gl.bstride + (long long)(g.oy + j) * gl.pitch[li] + g.ox + i]
                       : 0.0;
  F[g.off + c] = (T)r;
}

// Mixed precision, step A: x64 += x, x = 0 on the finest grids.
template <typename T>
__global__ void __launch_bounds__(256) k_accumulate(DevGeom G, const Tile* __restrict__ tiles, T* X, double* X64) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  const long long c = (long long)j * g.pitch + i;
  X64[g.off64 + c] += (double)X[g.off + c];
  X[g.off + c] = (T)0;
}

// Mixed precision, step B: f = (float)(R - A x64) in FP64 on the finest grids.
template <typename T, int KK>
__global__ void __launch_bounds__(256) k_refine_residual(DevGeom G, GlobalLayout gl, const Tile* __restrict__ tiles, T* F,
                                                         const double* __restrict__ X64, const double* __restrict__ R) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (!is_unknown(G, g, i, j)) return;
  const long long c = (long long)j * g.pitch + i;
  const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  const int li = g.level - MLEV_LMIN;
  const double r = R[(long long)g.problem * gl.bstride + (long long)(g.oy + j) * gl.pitch[li] + g.ox + i] -
                   apply_k<double, double>(X64 + g.off64, c, g.pitch, w);
  F[g.off + c] = (T)r;
}

// Diagnostics: ||R - A e||^2 and ||R||^2 per job on its finest grid (FP64), e in the FP64
// pool at off64 (mixed) or off (FP64 mode). Accumulated with atomics: order-dependent in
// the last bits, used only for reporting.
template <int KK>
__global__ void __launch_bounds__(256) k_job_resnorm(DevGeom G, GlobalLayout gl, const Tile* __restrict__ tiles,
                                                     const double* __restrict__ E, int use64,
                                                     const double* __restrict__ R, double* acc) {
  __shared__ double scratch[8 * 2];
  __shared__ double out[2];
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x % TX, j = t.y0 + threadIdx.x / TX;
  double v[2] = {0.0, 0.0};
  if (is_unknown(G, g, i, j)) {
    const long long c = (long long)j * g.pitch + i;
    const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
    const int li = g.level - MLEV_LMIN;
    const double f = R[(long long)g.problem * gl.bstride + (long long)(g.oy + j) * gl.pitch[li] + g.ox + i];
    const double r = f - apply_k<double, double>(E + (use64 ? g.off64 : g.off), c, g.pitch, w);
    v[0] = r * r;
    v[1] = f * f;
  }
  block_sum<2>(v, scratch, out);
  if (threadIdx.x == 0 && (out[0] != 0.0 || out[1] != 0.0)) {
    atomicAdd(&acc[2 * g.job], out[0]);
    atomicAdd(&acc[2 * g.job + 1], out[1]);
  }
}

// max over the jobs [first, first + count) of problem p of sqrt(rr / ff) -> stat slot.
__global__ void k_resnorm_finalize(const double* acc, int B, int jobs_per_problem, int first_kind_sub,
                                   int m, long long* stat, int stat_stride, int slot) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B) return;
  double mx = 0.0;
  if (first_kind_sub) {
    for (int j = 0; j < m; ++j) {
      const double* a = acc + 2 * (p * m + j);
      if (a[1] > 0) mx = fmax(mx, sqrt(a[0] / a[1]));
    }
  } else {
    const double* a = acc + 2 * (B * m + p);
    if (a[1] > 0) mx = sqrt(a[0] / a[1]);
  }
  stat[p * stat_stride + slot] = __double_as_longlong(mx);
  (void)jobs_per_problem;
}

// ------------------------------------------------------------------ launchers
#define MLEV_DISPATCH_KK(kk, ...)                                  \
  switch (kk) {                                                    \
    case MLEV_KAPPA_ONE: {                                         \
      constexpr int KK = MLEV_KAPPA_ONE;                           \
      __VA_ARGS__;                                                 \
    } break;                                                       \
    case MLEV_KAPPA_PER_COARSE_CELL: {                             \
      constexpr int KK = MLEV_KAPPA_PER_COARSE_CELL;               \
      __VA_ARGS__;                                                 \
    } break;                                                       \
    default: {                                                     \
      constexpr int KK = MLEV_KAPPA_PER_FINE_ELEM;                 \
      __VA_ARGS__;                                                 \
    } break;                                                       \
  }

template <typename T>
void launch_smooth(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, int color, double omega, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_smooth<T, KK><<<n, dim3(TX / 2, TY), 0, s>>>(G, tiles, X, F, color, (T)omega)));
}
template <typename T>
void launch_restrict(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, int black_zero, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_restrict<T, KK><<<n, dim3(TX, TY), 0, s>>>(G, tiles, X, F, black_zero)));
}
template <typename T>
void launch_prolong(const DevGeom& G, const Tile* tiles, int n, T* X, int red_only, cudaStream_t s) {
  if (!n) return;
  if (red_only)
    k_prolong<T, true><<<n, dim3(TX / 2, TY), 0, s>>>(G, tiles, X);
  else
    k_prolong<T, false><<<n, dim3(TX, TY), 0, s>>>(G, tiles, X);
}
template <typename T>
void launch_coarsest(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, int sweeps, double omega,
                     cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_coarsest<T, KK><<<n, 256, 0, s>>>(G, tiles, X, F, sweeps, (T)omega)));
}
template <typename T>
void launch_gather(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* X, T* F, double* X64,
                   const double* R, cudaStream_t s) {
  if (!n) return;
  k_gather<T><<<n, dim3(TX, TY), 0, s>>>(G, gl, tiles, X, F, X64, R);
}
template <typename T>
void launch_accumulate(const DevGeom& G, const Tile* tiles, int n, T* X, double* X64, cudaStream_t s) {
  if (!n) return;
  k_accumulate<T><<<n, dim3(TX, TY), 0, s>>>(G, tiles, X, X64);
}
template <typename T>
void launch_refine_residual(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, T* F, const double* X64,
                            const double* R, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_refine_residual<T, KK><<<n, dim3(TX, TY), 0, s>>>(G, gl, tiles, F, X64, R)));
}

template <typename T>
void launch_coarse_inverse(const DevGeom& G, const Tile* tiles, int n, T* inv, int nd_max, cudaStream_t s) {
  if (!n) return;
  const size_t smem = ((size_t)nd_max * nd_max + nd_max) * sizeof(double);
  MLEV_DISPATCH_KK(G.kap.kind, ({
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_coarse_inverse<T, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr = true;
    }
    k_coarse_inverse<T, KK><<<n, 256, smem, s>>>(G, tiles, inv, nd_max);
  }));
}
template <typename T>
void launch_coarsest_direct(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, const T* inv, int nd_max,
                            cudaStream_t s) {
  if (!n) return;
  k_coarsest_direct<T><<<n, 128, (size_t)nd_max * sizeof(T), s>>>(G, tiles, X, F, inv, nd_max);
}
// Bytes of shared memory the staged coarsest kernel needs for a grid of `nodes` nodes.
size_t coarsest_smem_bytes(int kappa_kind, int nodes, int tsize) {
  return (size_t)(kappa_kind == MLEV_KAPPA_ONE ? 3 : 7) * nodes * tsize;
}

template <typename T>
void launch_coarsest_smem(const DevGeom& G, const Tile* tiles, int n, int max_nodes, T* X, const T* F, int sweeps,
                          double omega, cudaStream_t s) {
  if (!n) return;
  const size_t smem = coarsest_smem_bytes(G.kap.kind, max_nodes, sizeof(T));
  MLEV_DISPATCH_KK(G.kap.kind, ({
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_coarsest_smem<T, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCoarsestSmemMax);
      attr = true;
    }
    k_coarsest_smem<T, KK><<<n, dim3(32, 32), smem, s>>>(G, tiles, X, F, sweeps, (T)omega);
  }));
}

void launch_job_resnorm(const DevGeom& G, const GlobalLayout& gl, const Tile* tiles, int n, const double* E, int use64,
                        const double* R, double* acc, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_job_resnorm<KK><<<n, 256, 0, s>>>(G, gl, tiles, E, use64, R, acc)));
}
void launch_resnorm_finalize(const double* acc, int B, int m, int subdomains, long long* stat, int stat_stride,
                             int slot, cudaStream_t s) {
  k_resnorm_finalize<<<(B + 127) / 128, 128, 0, s>>>(acc, B, m + 1, subdomains, m, stat, stat_stride, slot);
}

#define MLEV_INST(T)                                                                                             \
  template void launch_smooth<T>(const DevGeom&, const Tile*, int, T*, const T*, int, double, cudaStream_t);     \
  template void launch_restrict<T>(const DevGeom&, const Tile*, int, T*, T*, int, cudaStream_t);                 \
  template void launch_prolong<T>(const DevGeom&, const Tile*, int, T*, int, cudaStream_t);                      \
  template void launch_coarsest<T>(const DevGeom&, const Tile*, int, T*, const T*, int, double, cudaStream_t);   \
  template void launch_gather<T>(const DevGeom&, const GlobalLayout&, const Tile*, int, T*, T*, double*,         \
                                 const double*, cudaStream_t);                                                   \
  template void launch_accumulate<T>(const DevGeom&, const Tile*, int, T*, double*, cudaStream_t);               \
  template void launch_refine_residual<T>(const DevGeom&, const GlobalLayout&, const Tile*, int, T*,             \
                                          const double*, const double*, cudaStream_t);                           \
  template void launch_coarse_inverse<T>(const DevGeom&, const Tile*, int, T*, int, cudaStream_t);               \
  template void launch_coarsest_direct<T>(const DevGeom&, const Tile*, int, T*, const T*, const T*, int,         \
                                          cudaStream_t);                                                         \
  template void launch_coarsest_smem<T>(const DevGeom&, const Tile*, int, int, T*, const T*, int, double,        \
                                        cudaStream_t);
MLEV_INST(float)
MLEV_INST(double)

}  // namespace mlev
