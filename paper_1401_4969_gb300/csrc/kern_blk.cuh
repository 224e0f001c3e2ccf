// In-block multigrid: one thread block runs a whole V-cycle (or its lower part) on the
// grids of one job. Used by the level-1 eigensolver (grids in global memory) and by the
// multigrid tail kernel (grids copied into shared memory; the descriptors passed here
// then point into shared memory through their off / pitch fields).
#pragma once

#include "kern_common.cuh"

namespace mlev {

template <typename T, int KK>
__device__ void blk_smooth(const DevGeom& G, const GridDesc& g, T* X, const T* F, int sweeps, bool reverse, T omega) {
  const int W = g.nx + 1, nn = W * (g.ny + 1);
  T* x = X + g.off;
  for (int s = 0; s < sweeps; ++s)
    for (int cc = 0; cc < 2; ++cc) {
      const int color = reverse ? 1 - cc : cc;
      for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const int j = q / W, i = q - j * W;
        if (((i + j) & 1) != color || !is_unknown(G, g, i, j)) continue;
        const long long c = (long long)j * g.pitch + i;
        const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
        const T v = F[g.off + c] + (T)w.e * x[c + 1] + (T)w.w * x[c - 1] + (T)w.n * x[c + g.pitch] +
                    (T)w.s * x[c - g.pitch];
        x[c] += omega * (v / (T)(w.e + w.w + w.n + w.s) - x[c]);
      }
      __syncthreads();
    }
}

template <typename T, int KK>
__device__ __forceinline__ T blk_res(const DevGeom& G, const GridDesc& g, const T* X, const T* F, int i, int j) {
  if (!is_unknown(G, g, i, j)) return (T)0;
  const long long c = (long long)j * g.pitch + i;
  const EW<T> w = edge_weights_t<T, KK>(G.kap, g.problem, g.level, g.ox + i, g.oy + j);
  return F[g.off + c] - apply_k<T, T>(X + g.off, c, g.pitch, w);
}

template <typename T, int KK>
__device__ void blk_restrict(const DevGeom& G, const GridDesc& gf, const GridDesc& gc, T* X, T* F) {
  const int W = gc.nx + 1, nn = W * (gc.ny + 1);
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int J = q / W, I = q - J * W;
    const long long cc = (long long)J * gc.pitch + I;
    X[gc.off + cc] = (T)0;
    if (!is_unknown(G, gc, I, J)) continue;
    const int i = 2 * I, j = 2 * J;
    const T half = blk_res<T, KK>(G, gf, X, F, i + 1, j) + blk_res<T, KK>(G, gf, X, F, i - 1, j) +
                   blk_res<T, KK>(G, gf, X, F, i, j + 1) + blk_res<T, KK>(G, gf, X, F, i, j - 1) +
                   blk_res<T, KK>(G, gf, X, F, i + 1, j + 1) + blk_res<T, KK>(G, gf, X, F, i - 1, j - 1);
    F[gc.off + cc] = blk_res<T, KK>(G, gf, X, F, i, j) + (T)0.5 * half;
  }
  __syncthreads();
}

template <typename T>
__device__ void blk_prolong(const DevGeom& G, const GridDesc& gf, const GridDesc& gc, T* X) {
  const int W = gf.nx + 1, nn = W * (gf.ny + 1);
  const T* xc = X + gc.off;
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int j = q / W, i = q - j * W;
    if (!is_unknown(G, gf, i, j)) continue;
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
  __syncthreads();
}

// Exact coarsest solve x = A^{-1} f with the job's dense inverse (interior nodes of the
// window in row-major order; see k_coarse_inverse). `fbuf` holds nd values of scratch.
template <typename T>
__device__ void blk_direct(const DevGeom& G, const GridDesc& g, T* X, const T* F, const T* inv, T* fbuf) {
  const int nx1 = g.nx - 1, ny1 = g.ny - 1, nd = nx1 * ny1;
  for (int r = threadIdx.x; r < nd; r += blockDim.x) {
    const int j = r / nx1 + 1, i = r - (j - 1) * nx1 + 1;
    fbuf[r] = is_unknown(G, g, i, j) ? F[g.off + (long long)j * g.pitch + i] : (T)0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < nd; r += nw) {  // one warp per row of the inverse
    T acc = (T)0;
    for (int c = lane; c < nd; c += 32) acc += inv[r * nd + c] * fbuf[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int j = r / nx1 + 1, i = r - (j - 1) * nx1 + 1;
      X[g.off + (long long)j * g.pitch + i] = is_unknown(G, g, i, j) ? acc : (T)0;
    }
  }
  __syncthreads();
}

// V-cycle over grids[0 .. nlev-1] (finest first). The coarsest grid is solved with the
// dense inverse `inv` when given (fbuf: scratch of its size), else by csweeps sweeps.
template <typename T, int KK>
__device__ void blk_vcycle(const DevGeom& G, const GridDesc* grids, int nlev, T* X, T* F, int pre, int post, int csweeps,
                           T omega, const T* inv, T* fbuf = nullptr) {
  for (int d = 0; d + 1 < nlev; ++d) {
    blk_smooth<T, KK>(G, grids[d], X, F, pre, false, omega);
    blk_restrict<T, KK>(G, grids[d], grids[d + 1], X, F);
  }
  if (inv)
    blk_direct<T>(G, grids[nlev - 1], X, F, inv, fbuf);
  else
    blk_smooth<T, KK>(G, grids[nlev - 1], X, F, csweeps, false, omega);
  for (int d = nlev - 2; d >= 0; --d) {
    blk_prolong<T>(G, grids[d], grids[d + 1], X);
    blk_smooth<T, KK>(G, grids[d], X, F, post, true, omega);
  }
}

}  // namespace mlev
