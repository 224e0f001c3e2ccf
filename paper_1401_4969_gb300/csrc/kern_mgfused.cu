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
#include "kern_tail.cuh"

namespace mlev {

constexpr int FT = 64;  // output tile edge of the fused kernels (nodes)

// ---------------------------------------------------------------- TMA / mbarrier (inline PTX)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 2-D tiled bulk tensor copy global -> shared; x must be a multiple of 16 bytes / element size.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((unsigned long long)tmap) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase 0 of the barrier: gives up after ~2^22 polls and flags a timeout
// (the block then computes on whatever arrived; the solve reports MLEV_ETIMEOUT).
__device__ __forceinline__ void mbar_wait0(unsigned long long* bar, unsigned long long* status) {
  for (unsigned it = 0; !mbar_try_wait(bar, 0); ++it)
    if (it > (1u << 22)) {
      if (threadIdx.x == 0 && threadIdx.y == 0 && status) atomicOr(status, (unsigned long long)MLEV_ST_TIMEOUT);
      break;
    }
}

__device__ __forceinline__ const void* grid_map(const DevGeom& G, const GridDesc& g, int which) {
  return G.tmaps + (long long)(g.tmap + which) * MLEV_TMAP_BYTES;
}

// Thread block of the fused kernels: 32 x 8 threads; loops walk rows with threadIdx.y and,
// within a row, either every node (stride 32) or the nodes of one colour (stride 64).
// Tiles live in the TMA box layout: row pitch SW = MLEV_TMA_FBW; region node (a, b) is at
// q = (b + oy) * SW + a + ox.
template <typename T, int KK>
__device__ __forceinline__ void tile_half_sweep(const DevGeom& G, const GridDesc& g, T* xs, const T* fs,
                                                const uint8_t* uk, int ox, int oy, int rx0, int ry0, int lo, int hi,
                                                int color, T omega) {
  constexpr int SW = MLEV_TMA_FBW;
  for (int b = lo + threadIdx.y; b <= hi; b += blockDim.y) {
    const int a0 = lo + (((rx0 + lo + ry0 + b) & 1) != color);
    for (int a = a0 + 2 * threadIdx.x; a <= hi; a += 2 * blockDim.x) {
      const int q = (b + oy) * SW + a + ox;
      if (!uk[q]) continue;
      const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + rx0 + a, g.oy + ry0 + b);
      const T v = fs[q] + (T)w.e * xs[q + 1] + (T)w.w * xs[q - 1] + (T)w.n * xs[q + SW] + (T)w.s * xs[q - SW];
      xs[q] += omega * (div_diag<T>(v, (T)(w.e + w.w + w.n + w.s)) - xs[q]);
    }
  }
}

// Unknown mask of the whole fine box (computed while the TMA copies are in flight).
__device__ __forceinline__ void box_mask(const DevGeom& G, const GridDesc& g, uint8_t* uk, int fx0, int fy0) {
  for (int r = threadIdx.y; r < MLEV_TMA_FBH; r += blockDim.y)
    for (int c = threadIdx.x; c < MLEV_TMA_FBW; c += blockDim.x)
      uk[r * MLEV_TMA_FBW + c] = is_unknown(G, g, fx0 + c, fy0 + r);
}

template <typename T>
struct FusedSmem {  // byte offsets inside the dynamic shared memory (128-byte aligned arrays)
  static constexpr int FBOX = MLEV_TMA_FBW * MLEV_TMA_FBH;
  static constexpr int CBOX = MLEV_TMA_CBW * MLEV_TMA_CBH;
  static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
  static constexpr size_t xs = 0;
  static constexpr size_t fs = al(xs + FBOX * sizeof(T));
  static constexpr size_t xc = al(fs + FBOX * sizeof(T));
  static constexpr size_t uk = al(xc + CBOX * sizeof(T));
  static constexpr size_t total = al(uk + FBOX);
};

template <typename T, int KK, int NU>
__global__ void __launch_bounds__(256) k_mg_down(DevGeom G, const Tile* __restrict__ tiles, T* X, T* F, T omega) {
  constexpr int HALO = 2 * NU + 2;
  constexpr int RW = FT + 2 * HALO;
  constexpr int SW = MLEV_TMA_FBW, OX = MLEV_TMA_FOX - HALO, OY = MLEV_TMA_FOY - HALO;
  using L = FusedSmem<T>;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ unsigned long long bar;
  unsigned char* sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);  // TMA destinations: 128-byte aligned
  T* xs = reinterpret_cast<T*>(sm + L::xs);
  T* fs = reinterpret_cast<T*>(sm + L::fs);
  uint8_t* uk = sm + L::uk;
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const GridDesc& gc = G.grids[t.grid + 1];
  const int rx0 = t.x0 - HALO, ry0 = t.y0 - HALO;
  const int fx0 = t.x0 - MLEV_TMA_FOX, fy0 = t.y0 - MLEV_TMA_FOY;
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  if (lead) mbar_init(&bar);
  __syncthreads();
  if (lead) {
    const void* mx = grid_map(G, g, 0);
    const void* mf = grid_map(G, g, 1);
    tmap_acquire(mx);
    tmap_acquire(mf);
    mbar_expect_tx(&bar, 2u * L::FBOX * sizeof(T));
    tma_load_2d(xs, mx, fx0, fy0, &bar);
    tma_load_2d(fs, mf, fx0, fy0, &bar);
  }
  box_mask(G, g, uk, fx0, fy0);
  mbar_wait0(&bar, G.status);
  __syncthreads();
  for (int s = 0; s < 2 * NU; ++s) {
    tile_half_sweep<T, KK>(G, g, xs, fs, uk, OX, OY, rx0, ry0, s + 1, RW - 2 - s, s & 1, omega);
    __syncthreads();
  }
  {  // residual in place where the restriction needs it (0 off the unknowns)
    const int lo = 2 * NU + 1, hi = RW - 2 - 2 * NU;
    for (int b = lo + threadIdx.y; b <= hi; b += blockDim.y)
      for (int a = lo + threadIdx.x; a <= hi; a += blockDim.x) {
        const int q = (b + OY) * SW + a + OX;
        if (!uk[q]) {
          fs[q] = (T)0;
          continue;
        }
        const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + rx0 + a, g.oy + ry0 + b);
        fs[q] -= (T)(w.e + w.w + w.n + w.s) * xs[q] - (T)w.e * xs[q + 1] - (T)w.w * xs[q - 1] -
                 (T)w.n * xs[q + SW] - (T)w.s * xs[q - SW];
      }
  }
  __syncthreads();
  for (int bb = threadIdx.y; bb < FT; bb += blockDim.y)
    for (int aa = threadIdx.x; aa < FT; aa += blockDim.x) {
      const int i = t.x0 + aa, j = t.y0 + bb, q = (bb + MLEV_TMA_FOY) * SW + aa + MLEV_TMA_FOX;
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
      const int q = (2 * J - fy0) * SW + (2 * I - fx0);
      F[gc.off + cc] =
          fs[q] + (T)0.5 * (fs[q + 1] + fs[q - 1] + fs[q + SW] + fs[q - SW] + fs[q + SW + 1] + fs[q - SW - 1]);
    }
}

template <typename T, int KK, int NU>
__global__ void __launch_bounds__(256) k_mg_up(DevGeom G, const Tile* __restrict__ tiles, T* X, const T* __restrict__ F,
                                               T omega) {
  constexpr int HALO = 2 * NU;
  constexpr int RW = FT + 2 * HALO;
  constexpr int SW = MLEV_TMA_FBW, OX = MLEV_TMA_FOX - HALO, OY = MLEV_TMA_FOY - HALO;
  constexpr int CW = MLEV_TMA_CBW;
  using L = FusedSmem<T>;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ unsigned long long bar;
  unsigned char* sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);  // TMA destinations: 128-byte aligned
  T* xs = reinterpret_cast<T*>(sm + L::xs);
  T* fs = reinterpret_cast<T*>(sm + L::fs);
  T* xc = reinterpret_cast<T*>(sm + L::xc);
  uint8_t* uk = sm + L::uk;
  const Tile t = tiles[blockIdx.x];
  const GridDesc& g = G.grids[t.grid];
  const GridDesc& gc = G.grids[t.grid + 1];
  const int rx0 = t.x0 - HALO, ry0 = t.y0 - HALO;
  const int fx0 = t.x0 - MLEV_TMA_FOX, fy0 = t.y0 - MLEV_TMA_FOY;
  const int cx0 = (t.x0 >> 1) - MLEV_TMA_COX, cy0 = (t.y0 >> 1) - MLEV_TMA_COY;
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  if (lead) mbar_init(&bar);
  __syncthreads();
  if (lead) {
    const void* mx = grid_map(G, g, 0);
    const void* mf = grid_map(G, g, 1);
    const void* mc = grid_map(G, gc, 2);
    tmap_acquire(mx);
    tmap_acquire(mf);
    tmap_acquire(mc);
    mbar_expect_tx(&bar, (2u * L::FBOX + L::CBOX) * sizeof(T));
    tma_load_2d(xs, mx, fx0, fy0, &bar);
    tma_load_2d(fs, mf, fx0, fy0, &bar);
    tma_load_2d(xc, mc, cx0, cy0, &bar);
  }
  box_mask(G, g, uk, fx0, fy0);
  mbar_wait0(&bar, G.status);
  __syncthreads();
  // x += P x_c on the region (exact P1 interpolation on the SW-NE mesh)
  for (int b = threadIdx.y; b < RW; b += blockDim.y)
    for (int a = threadIdx.x; a < RW; a += blockDim.x) {
      const int q = (b + OY) * SW + a + OX;
      if (!uk[q]) continue;
      const int i = rx0 + a, j = ry0 + b;
      const int c = ((j >> 1) - cy0) * CW + ((i >> 1) - cx0);
      T v;
      if (!(i & 1) && !(j & 1)) v = xc[c];
      else if ((i & 1) && !(j & 1)) v = (T)0.5 * (xc[c] + xc[c + 1]);
      else if (!(i & 1) && (j & 1)) v = (T)0.5 * (xc[c] + xc[c + CW]);
      else v = (T)0.5 * (xc[c] + xc[c + CW + 1]);
      xs[q] += v;
    }
  __syncthreads();
  for (int s = 0; s < 2 * NU; ++s) {
    tile_half_sweep<T, KK>(G, g, xs, fs, uk, OX, OY, rx0, ry0, s + 1, RW - 2 - s, 1 - (s & 1), omega);
    __syncthreads();
  }
  for (int bb = threadIdx.y; bb < FT; bb += blockDim.y)
    for (int aa = threadIdx.x; aa < FT; aa += blockDim.x) {
      const int i = t.x0 + aa, j = t.y0 + bb, q = (bb + MLEV_TMA_FOY) * SW + aa + MLEV_TMA_FOX;
      if (i <= g.nx && j <= g.ny && uk[q]) X[g.off + (long long)j * g.pitch + i] = xs[q];
    }
}

// tiles[b].grid = the job's grid at the first tail depth; its coarser grids follow it.
template <typename T, int KK>
__global__ void __launch_bounds__(512, KK == MLEV_KAPPA_PER_FINE_ELEM ? 2 : 3) k_mg_tail(DevGeom G, const Tile* __restrict__ tiles, T* X, T* F,
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
    tail_restrict<T, KK>(G, lv[d], lv[d + 1], pre >= 1 && omega == (T)1);
  }
  if (jinv)
    tail_direct<T>(lv[nlev - 1], jinv, fbuf);
  else
    tail_smooth<T, KK>(G, lv[nlev - 1], csweeps, false, omega);
  for (int d = nlev - 2; d >= 0; --d) {
    tail_prolong<T>(lv[d], lv[d + 1], post >= 1 && omega == (T)1);
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
  return FusedSmem<T>::total + 128;  // + room to align the base to 128 bytes
}
template <typename T, int NU>
size_t up_smem() {
  return FusedSmem<T>::total + 128;
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
