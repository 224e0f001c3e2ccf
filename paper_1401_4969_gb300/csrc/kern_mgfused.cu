// Fused multigrid kernels for the masked SPD problems of Algorithm 4.1 (the auxiliary
// problems on Omega_j and the G_{m+1} problem). Same arithmetic as kern_mg.cu, fewer
// launches and fewer passes over memory:
//
// * k_mg_down: on one 64x64 output tile of a fine grid, NU red-black Gauss-Seidel sweeps,
//   the residual f - A x and its restriction P^T r to the coarse grid, in shared memory.
//   The tile is loaded with a halo of 2*NU + 2 nodes; every half-sweep shrinks the valid
//   region by one node, so the outputs equal those of the global sweeps (temporal
//   blocking). Writes the smoothed x of the tile, f and x = 0 on the coarse nodes it owns.
// * k_mg_up: prolongation x += P x_c and NU sweeps (colours in reverse order) on one tile
//   with a halo of 2*NU.
// * k_mg_tail: one block per job runs the rest of the V-cycle (all grids from a depth on,
//   down to the coarsest solve and back) on copies of those grids in shared memory.
#include "kern_blk.cuh"
#include "kern_launch.h"

namespace mlev {

constexpr int FT = 64;  // output tile edge of the fused kernels (nodes)

// Thread block of the fused kernels: 32 x 8 threads; loops below walk rows with threadIdx.y
// and, within a row, either every node (stride 32) or the nodes of one colour (stride 64).
template <typename T, int KK>
__device__ __forceinline__ void tile_half_sweep(const DevGeom& G, const GridDesc& g, T* xs, const T* fs,
                                                const uint8_t* uk, int RW, int rx0, int ry0, int lo, int hi, int color,
                                                T omega) {
  for (int b = lo + threadIdx.y; b <= hi; b += blockDim.y) {
    // first a >= lo in this row with (rx0 + a + ry0 + b) even == colour parity
    const int a0 = lo + (((rx0 + lo + ry0 + b) & 1) != color);
    for (int a = a0 + 2 * threadIdx.x; a <= hi; a += 2 * blockDim.x) {
      const int q = b * RW + a;
      if (!uk[q]) continue;
      const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + rx0 + a, g.oy + ry0 + b);
      const T v = fs[q] + (T)w.e * xs[q + 1] + (T)w.w * xs[q - 1] + (T)w.n * xs[q + RW] + (T)w.s * xs[q - RW];
      xs[q] += omega * (v / (T)(w.e + w.w + w.n + w.s) - xs[q]);
    }
  }
}

template <typename T, int KK, int NU>
__global__ void __launch_bounds__(256) k_mg_down(DevGeom G, const Tile* __restrict__ tiles, T* X, T* F, T omega) {
  constexpr int HALO = 2 * NU + 2;
  constexpr int RW = FT + 2 * HALO;
  extern __shared__ unsigned char sm_raw[];
  T* xs = reinterpret_cast<T*>(sm_raw);
  T* fs = xs + RW * RW;
  uint8_t* uk = reinterpret_cast<uint8_t*>(fs + RW * RW);
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const GridDesc& gc = G.grids[t.grid + 1];
  const int rx0 = t.x0 - HALO, ry0 = t.y0 - HALO;
  for (int b = threadIdx.y; b < RW; b += blockDim.y)
    for (int a = threadIdx.x; a < RW; a += blockDim.x) {
      const int q = b * RW + a, i = rx0 + a, j = ry0 + b;
      const bool in = i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
      const bool u = is_unknown(G, g, i, j);
      const long long c = (long long)j * g.pitch + i;
      xs[q] = in ? X[g.off + c] : (T)0;
      fs[q] = u ? F[g.off + c] : (T)0;
      uk[q] = u;
    }
  __syncthreads();
  for (int s = 0; s < 2 * NU; ++s) {
    tile_half_sweep<T, KK>(G, g, xs, fs, uk, RW, rx0, ry0, s + 1, RW - 2 - s, s & 1, omega);
    __syncthreads();
  }
  {  // residual in place where the restriction needs it
    const int lo = 2 * NU + 1, hi = RW - 2 - 2 * NU;
    for (int b = lo + threadIdx.y; b <= hi; b += blockDim.y)
      for (int a = lo + threadIdx.x; a <= hi; a += blockDim.x) {
        const int q = b * RW + a;
        if (!uk[q]) continue;
        const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + rx0 + a, g.oy + ry0 + b);
        fs[q] -= (T)(w.e + w.w + w.n + w.s) * xs[q] - (T)w.e * xs[q + 1] - (T)w.w * xs[q - 1] -
                 (T)w.n * xs[q + RW] - (T)w.s * xs[q - RW];
      }
  }
  __syncthreads();
  for (int bb = threadIdx.y; bb < FT; bb += blockDim.y)
    for (int aa = threadIdx.x; aa < FT; aa += blockDim.x) {
      const int i = t.x0 + aa, j = t.y0 + bb, q = (bb + HALO) * RW + aa + HALO;
      if (i <= g.nx && j <= g.ny && uk[q]) X[g.off + (long long)j * g.pitch + i] = xs[q];
    }
  constexpr int CT = FT / 2;
  for (int jj = threadIdx.y; jj < CT; jj += blockDim.y)
    for (int ii = threadIdx.x; ii < CT; ii += blockDim.x) {
      const int J = (t.y0 >> 1) + jj, I = (t.x0 >> 1) + ii;
      if (I > gc.nx || J > gc.ny) continue;
      const long long cc = (long long)J * gc.pitch + I;
      X[gc.off + cc] = (T)0;
      if (!is_unknown(G, gc, I, J)) continue;
      const int q = (2 * J - ry0) * RW + (2 * I - rx0);
      F[gc.off + cc] =
          fs[q] + (T)0.5 * (fs[q + 1] + fs[q - 1] + fs[q + RW] + fs[q - RW] + fs[q + RW + 1] + fs[q - RW - 1]);
    }
}

template <typename T, int KK, int NU>
__global__ void __launch_bounds__(256) k_mg_up(DevGeom G, const Tile* __restrict__ tiles, T* X, const T* __restrict__ F,
                                               T omega) {
  constexpr int HALO = 2 * NU;
  constexpr int RW = FT + 2 * HALO;
  extern __shared__ unsigned char sm_raw[];
  T* xs = reinterpret_cast<T*>(sm_raw);
  T* fs = xs + RW * RW;
  uint8_t* uk = reinterpret_cast<uint8_t*>(fs + RW * RW);
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const GridDesc& gc = G.grids[t.grid + 1];
  const T* xc = X + gc.off;
  const int rx0 = t.x0 - HALO, ry0 = t.y0 - HALO;
  for (int b = threadIdx.y; b < RW; b += blockDim.y)
    for (int a = threadIdx.x; a < RW; a += blockDim.x) {
      const int q = b * RW + a, i = rx0 + a, j = ry0 + b;
      const bool in = i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
      const bool u = is_unknown(G, g, i, j);
      const long long c = (long long)j * g.pitch + i;
      T x = in ? X[g.off + c] : (T)0;
      if (u) {  // x += P x_c (exact P1 interpolation on the SW-NE mesh)
        const int I = i >> 1, J = j >> 1;
        const long long cj = (long long)J * gc.pitch + I;
        if (!(i & 1) && !(j & 1)) x += xc[cj];
        else if ((i & 1) && !(j & 1)) x += (T)0.5 * (xc[cj] + xc[cj + 1]);
        else if (!(i & 1) && (j & 1)) x += (T)0.5 * (xc[cj] + xc[cj + gc.pitch]);
        else x += (T)0.5 * (xc[cj] + xc[cj + gc.pitch + 1]);
      }
      xs[q] = x;
      fs[q] = u ? F[g.off + c] : (T)0;
      uk[q] = u;
    }
  __syncthreads();
  for (int s = 0; s < 2 * NU; ++s) {
    tile_half_sweep<T, KK>(G, g, xs, fs, uk, RW, rx0, ry0, s + 1, RW - 2 - s, 1 - (s & 1), omega);
    __syncthreads();
  }
  for (int bb = threadIdx.y; bb < FT; bb += blockDim.y)
    for (int aa = threadIdx.x; aa < FT; aa += blockDim.x) {
      const int i = t.x0 + aa, j = t.y0 + bb, q = (bb + HALO) * RW + aa + HALO;
      if (i <= g.nx && j <= g.ny && uk[q]) X[g.off + (long long)j * g.pitch + i] = xs[q];
    }
}

constexpr int kTailMaxLev = 16;

// Shared-memory grid of the tail: compact row pitch W = nx + 1, x / f values and a mask of
// the unknowns; `g` is the job's original descriptor (coordinates, level, coefficient).
template <typename T>
struct SmGrid {
  T* x;
  T* f;
  uint8_t* m;
  int nx, ny, W;
  const GridDesc* g;
};

// Red-black sweeps with a 32 x 16 thread block: thread (tx, ty) visits rows ty + 1, ty + 17,
// ... and, in each row, the nodes of the current colour with stride 64.
template <typename T, int KK>
__device__ void tail_smooth(const DevGeom& G, const SmGrid<T>& s, int sweeps, bool reverse, T omega) {
  const GridDesc& g = *s.g;
  for (int it = 0; it < sweeps; ++it)
    for (int cc = 0; cc < 2; ++cc) {
      const int color = reverse ? 1 - cc : cc;
      for (int j = 1 + threadIdx.y; j < s.ny; j += blockDim.y) {
        const int i0 = ((color + j) & 1) ? 1 : 2;
        for (int i = i0 + 2 * threadIdx.x; i < s.nx; i += 2 * blockDim.x) {
          const int q = j * s.W + i;
          if (!s.m[q]) continue;
          const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
          const T v = s.f[q] + (T)w.e * s.x[q + 1] + (T)w.w * s.x[q - 1] + (T)w.n * s.x[q + s.W] +
                      (T)w.s * s.x[q - s.W];
          s.x[q] += omega * (v / (T)(w.e + w.w + w.n + w.s) - s.x[q]);
        }
      }
      __syncthreads();
    }
}

template <typename T, int KK>
__device__ __forceinline__ T tail_res(const DevGeom& G, const SmGrid<T>& s, int i, int j) {
  const int q = j * s.W + i;
  if (!s.m[q]) return (T)0;
  const GridDesc& g = *s.g;
  const W4 w = edge_weights<KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  return s.f[q] - ((T)(w.e + w.w + w.n + w.s) * s.x[q] - (T)w.e * s.x[q + 1] - (T)w.w * s.x[q - 1] -
                   (T)w.n * s.x[q + s.W] - (T)w.s * s.x[q - s.W]);
}

template <typename T, int KK>
__device__ void tail_restrict(const DevGeom& G, const SmGrid<T>& fi, const SmGrid<T>& co) {
  for (int J = threadIdx.y; J <= co.ny; J += blockDim.y)
    for (int I = threadIdx.x; I <= co.nx; I += blockDim.x) {
      const int q = J * co.W + I;
      co.x[q] = (T)0;
      if (!co.m[q]) continue;
      const int i = 2 * I, j = 2 * J;
      const T half = tail_res<T, KK>(G, fi, i + 1, j) + tail_res<T, KK>(G, fi, i - 1, j) +
                     tail_res<T, KK>(G, fi, i, j + 1) + tail_res<T, KK>(G, fi, i, j - 1) +
                     tail_res<T, KK>(G, fi, i + 1, j + 1) + tail_res<T, KK>(G, fi, i - 1, j - 1);
      co.f[q] = tail_res<T, KK>(G, fi, i, j) + (T)0.5 * half;
    }
  __syncthreads();
}

template <typename T>
__device__ void tail_prolong(const SmGrid<T>& fi, const SmGrid<T>& co) {
  for (int j = 1 + threadIdx.y; j < fi.ny; j += blockDim.y)
    for (int i = 1 + threadIdx.x; i < fi.nx; i += blockDim.x) {
      const int q = j * fi.W + i;
      if (!fi.m[q]) continue;
      const int I = i >> 1, J = j >> 1, c = J * co.W + I;
      T v;
      if (!(i & 1) && !(j & 1)) v = co.x[c];
      else if ((i & 1) && !(j & 1)) v = (T)0.5 * (co.x[c] + co.x[c + 1]);
      else if (!(i & 1) && (j & 1)) v = (T)0.5 * (co.x[c] + co.x[c + co.W]);
      else v = (T)0.5 * (co.x[c] + co.x[c + co.W + 1]);
      fi.x[q] += v;
    }
  __syncthreads();
}

template <typename T>
__device__ void tail_direct(const SmGrid<T>& s, const T* __restrict__ inv, T* fbuf) {
  const int nx1 = s.nx - 1, nd = nx1 * (s.ny - 1);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int r = tid; r < nd; r += nt) {
    const int j = r / nx1 + 1, i = r - (j - 1) * nx1 + 1, q = j * s.W + i;
    fbuf[r] = s.m[q] ? s.f[q] : (T)0;
  }
  __syncthreads();
  for (int r = tid; r < nd; r += nt) {
    const int j = r / nx1 + 1, i = r - (j - 1) * nx1 + 1, q = j * s.W + i;
    T acc = (T)0;
    for (int c = 0; c < nd; ++c) acc += inv[r * nd + c] * fbuf[c];
    s.x[q] = s.m[q] ? acc : (T)0;
  }
  __syncthreads();
}

// tiles[b].grid = the job's grid at the first tail depth; its coarser grids follow it.
template <typename T, int KK>
__global__ void __launch_bounds__(512) k_mg_tail(DevGeom G, const Tile* __restrict__ tiles, T* X, T* F,
                                                 const T* __restrict__ inv, int nd_max, int nlev, int pre, int post,
                                                 int csweeps, T omega, int load_x) {
  extern __shared__ unsigned char sm_raw[];
  __shared__ SmGrid<T> lv[kTailMaxLev];
  const int gi0 = tiles[blockIdx.x].grid;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  if (tid == 0) {
    long long tot = 0;
    for (int k = 0; k < nlev; ++k) {
      const GridDesc& g = G.grids[gi0 + k];
      tot += (long long)(g.nx + 1) * (g.ny + 1);
      tot = (tot + 1) & ~1LL;
    }
    T* xb = reinterpret_cast<T*>(sm_raw);
    T* fb = xb + tot;
    uint8_t* mb = reinterpret_cast<uint8_t*>(fb + tot + nd_max);
    long long off = 0;
    for (int k = 0; k < nlev; ++k) {
      const GridDesc& g = G.grids[gi0 + k];
      lv[k].x = xb + off;
      lv[k].f = fb + off;
      lv[k].m = mb + off;
      lv[k].nx = g.nx;
      lv[k].ny = g.ny;
      lv[k].W = g.nx + 1;
      lv[k].g = &G.grids[gi0 + k];
      off += (long long)(g.nx + 1) * (g.ny + 1);
      off = (off + 1) & ~1LL;
    }
  }
  __syncthreads();
  T* fbuf = lv[0].f + 0;  // placeholder, replaced below
  {
    // fbuf follows the f values of all levels (nd_max entries)
    long long tot = 0;
    for (int k = 0; k < nlev; ++k) {
      tot += (long long)(lv[k].nx + 1) * (lv[k].ny + 1);
      tot = (tot + 1) & ~1LL;
    }
    fbuf = reinterpret_cast<T*>(sm_raw) + 2 * tot;
  }
  for (int k = 0; k < nlev; ++k) {
    const GridDesc& g = *lv[k].g;
    const int nn = lv[k].W * (lv[k].ny + 1);
    for (int q = tid; q < nn; q += nt) {
      const int j = q / lv[k].W, i = q - j * lv[k].W;
      const bool u = is_unknown(G, g, i, j);
      lv[k].m[q] = u;
      if (k == 0) {
        const long long c = (long long)j * g.pitch + i;
        lv[0].x[q] = load_x ? X[g.off + c] : (T)0;
        lv[0].f[q] = u ? F[g.off + c] : (T)0;
      }
    }
  }
  __syncthreads();
  const T* jinv = inv ? inv + (long long)lv[0].g->job * nd_max * nd_max : nullptr;
  for (int d = 0; d + 1 < nlev; ++d) {
    tail_smooth<T, KK>(G, lv[d], pre, false, omega);
    tail_restrict<T, KK>(G, lv[d], lv[d + 1]);
  }
  if (jinv)
    tail_direct<T>(lv[nlev - 1], jinv, fbuf);
  else
    tail_smooth<T, KK>(G, lv[nlev - 1], csweeps, false, omega);
  for (int d = nlev - 2; d >= 0; --d) {
    tail_prolong<T>(lv[d], lv[d + 1]);
    tail_smooth<T, KK>(G, lv[d], post, true, omega);
  }
  const GridDesc& g0 = *lv[0].g;
  const int nn0 = lv[0].W * (lv[0].ny + 1);
  for (int q = tid; q < nn0; q += nt) {
    const int j = q / lv[0].W, i = q - j * lv[0].W;
    X[g0.off + (long long)j * g0.pitch + i] = lv[0].x[q];
  }
}

// ------------------------------------------------------------------ launchers
#define MLEV_DISPATCH_KK2(kk, ...)                   \
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

template <typename T, int NU>
size_t down_smem() {
  constexpr int RW = FT + 2 * (2 * NU + 2);
  return (size_t)RW * RW * (2 * sizeof(T) + 1);
}
template <typename T, int NU>
size_t up_smem() {
  constexpr int RW = FT + 2 * (2 * NU);
  return (size_t)RW * RW * (2 * sizeof(T) + 1);
}

template <typename T, int KK, int NU>
void down_one(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, double omega, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mg_down<T, KK, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)down_smem<T, NU>());
    attr = true;
  }
  k_mg_down<T, KK, NU><<<n, dim3(32, 8), down_smem<T, NU>(), s>>>(G, tiles, X, F, (T)omega);
}
template <typename T, int KK, int NU>
void up_one(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, double omega, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mg_up<T, KK, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)up_smem<T, NU>());
    attr = true;
  }
  k_mg_up<T, KK, NU><<<n, dim3(32, 8), up_smem<T, NU>(), s>>>(G, tiles, X, F, (T)omega);
}

template <typename T>
void launch_mg_down(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, int nu, double omega, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK2(G.kap.kind, {
    if (nu == 1) down_one<T, KK, 1>(G, tiles, n, X, F, omega, s);
    else down_one<T, KK, 2>(G, tiles, n, X, F, omega, s);
  });
}
template <typename T>
void launch_mg_up(const DevGeom& G, const Tile* tiles, int n, T* X, const T* F, int nu, double omega, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK2(G.kap.kind, {
    if (nu == 1) up_one<T, KK, 1>(G, tiles, n, X, F, omega, s);
    else up_one<T, KK, 2>(G, tiles, n, X, F, omega, s);
  });
}
template <typename T>
void launch_mg_tail(const DevGeom& G, const Tile* tiles, int n, T* X, T* F, const T* inv, int nd_max, int nlev,
                    int pre, int post, int csweeps, double omega, int load_x, size_t smem, cudaStream_t s) {
  if (!n) return;
  MLEV_DISPATCH_KK2(G.kap.kind, {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_mg_tail<T, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemMax);
      attr = true;
    }
    k_mg_tail<T, KK><<<n, dim3(32, 16), smem, s>>>(G, tiles, X, F, inv, nd_max, nlev, pre, post, csweeps, (T)omega,
                                                   load_x);
  });
}

#define MLEV_INST_F(T)                                                                                      \
  template void launch_mg_down<T>(const DevGeom&, const Tile*, int, T*, T*, int, double, cudaStream_t);     \
  template void launch_mg_up<T>(const DevGeom&, const Tile*, int, T*, const T*, int, double, cudaStream_t); \
  template void launch_mg_tail<T>(const DevGeom&, const Tile*, int, T*, T*, const T*, int, int, int, int,   \
                                  int, double, int, size_t, cudaStream_t);
MLEV_INST_F(float)
MLEV_INST_F(double)

}  // namespace mlev
