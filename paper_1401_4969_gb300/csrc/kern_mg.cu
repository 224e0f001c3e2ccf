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

template <typename T, int KK>
__global__ void __launch_bounds__(256) k_smooth(DevGeom G, const Tile* __restrict__ tiles, T* X, const T* __restrict__ F,
                                                int color, T omega) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (((i + j) & 1) != color || !is_unknown(G, g, i, j)) return;
  T* x = X + g.off;
  const long long c = (long long)j * g.pitch + i;
  const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  const T s = F[g.off + c] + (T)w.e * x[c + 1] + (T)w.w * x[c - 1] + (T)w.n * x[c + g.pitch] + (T)w.s * x[c - g.pitch];
  x[c] += omega * (s / (T)(w.e + w.w + w.n + w.s) - x[c]);
}

// r = f - A x at node (i, j) of grid g (0 off the unknowns).
template <typename T, int KK>
__device__ __forceinline__ T residual_at(const DevGeom& G, const GridDesc& g, const T* X, const T* F, int i, int j) {
  if (!is_unknown(G, g, i, j)) return (T)0;
  const long long c = (long long)j * g.pitch + i;
  const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  return F[g.off + c] - apply_k<T, T>(X + g.off, c, g.pitch, w);
}

// Coarse grid (tiles over depth d+1): f_c = P^T (f - A x)_fine, x_c = 0.
template <typename T, int KK>
__global__ void __launch_bounds__(256) k_restrict(DevGeom G, const Tile* __restrict__ tiles, T* X, T* F) {
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
  T half = residual_at<T, KK>(G, gf, X, F, i + 1, j) + residual_at<T, KK>(G, gf, X, F, i - 1, j) +
           residual_at<T, KK>(G, gf, X, F, i, j + 1) + residual_at<T, KK>(G, gf, X, F, i, j - 1) +
           residual_at<T, KK>(G, gf, X, F, i + 1, j + 1) + residual_at<T, KK>(G, gf, X, F, i - 1, j - 1);
  F[gc.off + cc] = acc + (T)0.5 * half;
}

// Fine grid (tiles over depth d): x += P x_c.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(DevGeom G, const Tile* __restrict__ tiles, T* X) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& gf = G.grids[t.grid];
  const GridDesc& gc = G.grids[t.grid + 1];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
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
        const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
        const T v = F[g.off + c] + (T)w.e * x[c + 1] + (T)w.w * x[c - 1] + (T)w.n * x[c + g.pitch] +
                    (T)w.s * x[c - g.pitch];
        x[c] += omega * (v / (T)(w.e + w.w + w.n + w.s) - x[c]);
      }
      __syncthreads();
    }
  }
}

// Finest grids of subdomain jobs: f = R (global residual of Eq. Aux_Problem restricted
// to Omega_j), x = 0, x64 = 0.
template <typename T>
__global__ void __launch_bounds__(256) k_gather(DevGeom G, GlobalLayout gl, const Tile* __restrict__ tiles, T* X, T* F,
                                                double* X64, const double* __restrict__ R) {
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const int i = t.x0 + threadIdx.x, j = t.y0 + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  const long long c = (long long)j * g.pitch + i;
  X[g.off + c] = (T)0;
  if (X64) X64[g.off64 + c] = 0.0;
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
  MLEV_DISPATCH_KK(G.kap.kind, (k_smooth<T, KK><<<n, dim3(TX, TY), 0, s>>>(G, tiles, X, F, color, (T)omega)));
}
template <typename T>
void launch_restrict(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK(G.kap.kind, (k_restrict<T, KK><<<n, dim3(TX, TY), 0, s>>>(G, tiles, X, F)));
}
template <typename T>
void launch_prolong(const DevGeom& G, const Tile* tiles, int n, T* X, cudaStream_t s) {
  if (!n) return;
  k_prolong<T><<<n, dim3(TX, TY), 0, s>>>(G, tiles, X);
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
  template void launch_restrict<T>(const DevGeom&, const Tile*, int, T*, T*, cudaStream_t);                      \
  template void launch_prolong<T>(const DevGeom&, const Tile*, int, T*, cudaStream_t);                           \
  template void launch_coarsest<T>(const DevGeom&, const Tile*, int, T*, const T*, int, double, cudaStream_t);   \
  template void launch_gather<T>(const DevGeom&, const GlobalLayout&, const Tile*, int, T*, T*, double*,         \
                                 const double*, cudaStream_t);                                                   \
  template void launch_accumulate<T>(const DevGeom&, const Tile*, int, T*, double*, cudaStream_t);               \
  template void launch_refine_residual<T>(const DevGeom&, const GlobalLayout&, const Tile*, int, T*,             \
                                          const double*, const double*, cudaStream_t);
MLEV_INST(float)
MLEV_INST(double)

}  // namespace mlev
